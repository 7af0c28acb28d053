"""Block-sparse (U(1) x U(1)) mode on the GPU against the symmetric oracle.

The GPU zip-up runs the rSVD sector by sector in the charge of the cut bond and
truncates once over all sectors, like ``oracle.symmetric``; both draw the same
Omega (a sector's sketch is the dense sketch's rows of that sector's columns).
The lattice (3x4, D=2, Hubbard PEPO, seed 5) has its degenerate singular-value
clusters away from chi = 4, 6, 12, so the kept subspace is unique and FP64 runs
must agree to 1e-9 on ln|<psi|O|psi>|.
"""
import numpy as np
import pytest

from oracle import boundary as B
from oracle import symmetric as S
from synth import lattice as L
from synth import u1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fp():
    import torch
    from paper_2511_01039_gb300 import fpeps
    torch.cuda.set_device(0)
    fpeps.lib()
    return fpeps


def _case(layer):
    Lx, Ly, D, seed = 3, 4, 2, 5
    peps, ch = u1.u1_peps(Lx, Ly, D, seed)
    qpeps = [[u1.peps_leg_charges(ch, Lx, Ly, r, c) for c in range(Ly)] for r in range(Lx)]
    ham = L.hubbard_hamiltonian(Lx, Ly, seed)
    W, qW = L.fsm_pepo(ham), u1.hubbard_pepo_charges(ham)
    if layer == 1:
        Wl, qWl = W, qW
    else:
        z = np.zeros((1, 2), dtype=np.int64)
        Wl, qWl = L.identity_pepo(Lx, Ly, 4), [[(z, z, z, z)] * Ly for _ in range(Lx)]
    return peps, qpeps, W, qW, Wl, qWl


def _gpu_sweep(fp, peps, qpeps, W, qW, *, chi, prec, layer, exact, oversample=4):
    env = fp.Env(peps, W, D=2, p=4, w=6, chi=chi, prec=prec, seed=5, charges=fp.pack_charges(qpeps, qW))
    try:
        for r in range(3):
            fp.fpeps_absorb_row(env.h, r, layer)
            if r == 1:
                fp.fpeps_compress_rsvd(env.h, fp.params(oversample, 2, 0, 0, int(exact)))
        return fp.fpeps_sweep_value(env.h)
    finally:
        env.close()


@pytest.mark.parametrize("layer", [0, 1])
@pytest.mark.parametrize("exact", [True, False])
@pytest.mark.parametrize("chi", [4, 6, 12])
def test_u1_zipup_matches_symmetric_oracle(fp, chi, exact, layer):
    peps, qpeps, W, qW, Wl, qWl = _case(layer)
    prm = B.RsvdParams(oversample=4, power_iters=2, n_fit=0, exact_svd=exact)
    sn_o, ln_o = S.contract_u1(peps, qpeps, Wl, qWl, chi, prm, seed=5, layer=layer)
    sg, lg = _gpu_sweep(fp, peps, qpeps, W, qW, chi=chi, prec="f64", layer=layer, exact=exact)
    assert sg == sn_o
    assert abs(lg - ln_o) < 1e-9


def test_u1_zipup_tf32x3(fp):
    """Split-precision products (3xTF32): FP32-class agreement with the FP64 oracle."""
    peps, qpeps, W, qW, Wl, qWl = _case(1)
    prm = B.RsvdParams(oversample=4, power_iters=2, n_fit=0)
    sn_o, ln_o = S.contract_u1(peps, qpeps, Wl, qWl, 6, prm, seed=5, layer=1)
    sg, lg = _gpu_sweep(fp, peps, qpeps, W, qW, chi=6, prec="tf32x3", layer=1, exact=False)
    assert sg == sn_o
    assert abs(lg - ln_o) < 1e-4


@pytest.mark.parametrize("chi", [4, 12])
def test_u1_cbe_fit_matches_symmetric_oracle(fp, chi):
    """Zip-up plus the sector-wise CBE fit (Fig. 3-5), same sketches on both sides."""
    peps, qpeps, W, qW, Wl, qWl = _case(1)
    prm = B.RsvdParams(oversample=4, power_iters=2, n_fit=1, chi_tilde=2)
    sn_o, ln_o = S.contract_u1(peps, qpeps, Wl, qWl, chi, prm, seed=5, layer=1)
    env = fp.Env(peps, W, D=2, p=4, w=6, chi=chi, prec="f64", seed=5, charges=fp.pack_charges(qpeps, qW))
    try:
        for r in range(3):
            fp.fpeps_absorb_row(env.h, r, 1)
            if r == 1:
                fp.fpeps_compress_rsvd(env.h, fp.params(4, 2, 2, 1, 0))
        sg, lg = fp.fpeps_sweep_value(env.h)
    finally:
        env.close()
    assert sg == sn_o
    assert abs(lg - ln_o) < 1e-9


def test_u1_expect_public_api(fp):
    """<H> through fpeps_expect (operator and norm sweeps, zip-up + CBE fit) in the
    charge-sector mode; at chi = 12 every cut of both layers lies between distinct
    values or at the full rank."""
    peps, qpeps, W, qW, _, _ = _case(1)
    prm = B.RsvdParams(oversample=4, power_iters=2, n_fit=1, chi_tilde=2)
    e_o, (sn_o, ln_o), (sd_o, ld_o) = S.expectation_u1(peps, qpeps, W, qW, 12, prm, seed=5)
    env = fp.Env(peps, W, D=2, p=4, w=6, chi=12, prec="f64", seed=5, charges=fp.pack_charges(qpeps, qW))
    try:
        val, sn, ln = env.expect(fp.params(4, 2, 2, 1, 0))
    finally:
        env.close()
    assert sn == sn_o                       # sign and ln|.| of <psi|H|psi>
    assert abs(ln - ln_o) < 1e-9
    assert abs(val - e_o) <= 1e-9 * abs(e_o)


def test_u1_checkpoint_carries_bond_charges(fp):
    """A 4-row lattice in the charge-sector mode: the sweep stopped after row 1, its boundary
    exported (with the bond charges) and imported into a fresh env, then rows 2 and 3, gives the
    uninterrupted sweep's value; a dense env refuses the charged checkpoint."""
    Lx, Ly, D, seed = 4, 4, 2, 5
    peps, ch = u1.u1_peps(Lx, Ly, D, seed)
    qpeps = [[u1.peps_leg_charges(ch, Lx, Ly, r, c) for c in range(Ly)] for r in range(Lx)]
    ham = L.hubbard_hamiltonian(Lx, Ly, seed)
    W, qW = L.fsm_pepo(ham), u1.hubbard_pepo_charges(ham)
    prm = fp.params(4, 2, 2, 1, 0)

    def new_env():
        return fp.Env(peps, W, D=D, p=4, w=6, chi=8, prec="f64", seed=seed, charges=fp.pack_charges(qpeps, qW))

    env = new_env()
    try:
        for r in range(Lx):
            fp.fpeps_absorb_row(env.h, r, 1)
            if 0 < r < Lx - 1:
                fp.fpeps_compress_rsvd(env.h, prm)
            if r == 1:
                blob = fp.fpeps_export_boundary(env.h)
        ref = fp.fpeps_sweep_value(env.h)
    finally:
        env.close()
    env = new_env()
    try:
        fp.fpeps_import_boundary(env.h, blob, 2, 1)
        for r in range(2, Lx):
            fp.fpeps_absorb_row(env.h, r, 1)
            if r < Lx - 1:
                fp.fpeps_compress_rsvd(env.h, prm)
        got = fp.fpeps_sweep_value(env.h)
    finally:
        env.close()
    assert got[0] == ref[0]
    assert abs(got[1] - ref[1]) < 1e-12
    dense = fp.Env(peps, W, D=D, p=4, w=6, chi=8, prec="f64", seed=seed)
    try:
        with pytest.raises(fp.FpepsError) as ei:
            fp.fpeps_import_boundary(dense.h, blob, 2, 1)
        assert ei.value.status == 1   # FPEPS_ERR_ARG
    finally:
        dense.close()
