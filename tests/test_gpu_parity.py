"""GPU path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Tolerances: the FP64 path runs the oracle's algorithm in double precision and
must agree to 1e-8 relative on <psi|O|psi> (the bar for the FP64 mode); the
FP32 path is held to 1e-4 on the small lattices here (FP32 unit roundoff
6e-8, amplified through ~O(10) chained factorisations and truncations).
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import boundary as B
from oracle import network as N
from synth import lattice as L

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def fp():
    import torch
    from paper_2511_01039_gb300 import fpeps
    torch.cuda.set_device(0)
    fpeps.lib()
    return fpeps


def _rel(a, b):
    return abs(a / b - 1.0)


def _env(fp, peps, pepo, *, D, w, chi, prec, seed):
    return fp.Env(peps, pepo, D=D, p=4, w=w, chi=chi, prec=prec, seed=seed)


@pytest.mark.parametrize("kind", ["identity", "dense2", "fsm2", "fsm4"])
@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f32", 1e-4), ("tf32x3", 1e-4)])
def test_c1_3x3_exact_against_brute_force(fp, kind, prec, tol):
    """3x3, D=2, chi >= the largest rank of any Theta_c: the exact regime (pin (a))."""
    peps = L.random_peps(3, 3, 2, 4, seed=0)
    if kind == "identity":
        pepo, w, chi = L.identity_pepo(3, 3, 4), 1, 16
    elif kind == "dense2":
        pepo, w, chi = L.dense_pepo(3, 3, 4, 2, seed=1), 2, 64
    elif kind == "fsm2":
        pepo, w, chi = L.fsm_pepo(L.random_hamiltonian(3, 3, 4, 0, seed=1)), 2, 64
    else:
        pepo, w, chi = L.fsm_pepo(L.random_hamiltonian(3, 3, 4, 2, seed=1)), 4, 256
    num, den = N.brute_force_expectation(peps, pepo)
    env = _env(fp, peps, pepo, D=2, w=w, chi=chi, prec=prec, seed=9)
    prm = fp.params(oversample=10, power_iters=0, n_fit=1, exact_svd=1)
    val, sn, ln = env.expect(prm)
    sd, ld = env.norm(prm)
    env.close()
    assert _rel(sn * math.exp(ln), num) < tol
    assert _rel(sd * math.exp(ld), den) < tol
    assert _rel(val, num / den) < 2 * tol


# 3xTF32 tolerance = FP32 tolerance x 12: a 3xTF32 product carries up to 3 * 2^-22
# relative error (the TF32 rounding of each operand's lo part and the dropped
# lo * lo term) against 2^-24 for one FP32 operation
TF32X3_OVER_F32 = 12


@pytest.mark.parametrize("prec,tol", [("f64", 1e-9), ("f32", 1e-5), ("tf32x3", 1e-5 * TF32X3_OVER_F32)])
@pytest.mark.parametrize("n_fit", [0, 1, 2, 3])
def test_truncated_4x4_matches_oracle_algorithm(fp, prec, tol, n_fit):
    """Truncated regime (chi=12 < exact bonds): same algorithm, same Omega, both sides.

    The PEPS has decaying bond weights, so the kept and discarded singular values
    are separated; with the flat spectra of a plain random PEPS the kept subspace is
    near-degenerate and FP32-level perturbations move the result by a fraction of the
    truncation error itself (test_c2_against_stored_oracle covers that case)."""
    peps = L.decaying_peps(4, 4, 2, 4, seed=3)
    pepo = L.fsm_pepo(L.random_hamiltonian(4, 4, 4, 2, seed=3))
    prm_o = B.RsvdParams(oversample=6, power_iters=2, n_fit=n_fit)
    sn_o, ln_o = B.contract(peps, pepo, 12, prm_o, seed=5, layer=1)
    env = _env(fp, peps, pepo, D=2, w=4, chi=12, prec=prec, seed=5)
    # operator sweep through the row-level ABI
    for r in range(4):
        fp.fpeps_absorb_row(env.h, r, 1)
        if 0 < r < 3:
            st = fp.fpeps_compress_rsvd(env.h, fp.params(6, 2, 0, n_fit, 0))
            assert st.alg_flops > 0 and st.seconds > 0
    sg, lg = fp.fpeps_sweep_value(env.h)
    env.close()
    assert sg == sn_o
    assert abs(lg - ln_o) < tol


@pytest.mark.parametrize("prec,tol", [("f64", 1e-11), ("tf32x3", 1e-5)])
def test_apply_theta_small_sites(fp, prec, tol):
    """One Theta_c application on every site of an interior row (ragged edge dims)."""
    peps = L.random_peps(4, 4, 3, 4, seed=11)
    pepo = L.fsm_pepo(L.random_hamiltonian(4, 4, 4, 2, seed=11))
    T, _ = B.first_row_boundary(peps[0], pepo[0])
    env = _env(fp, peps, pepo, D=3, w=4, chi=40, prec=prec, seed=5)
    fp.fpeps_absorb_row(env.h, 0, 1)
    fp.fpeps_absorb_row(env.h, 1, 1)
    g = np.random.default_rng(1)
    for c in range(4):
        A, W = peps[1][c], pepo[1][c]
        t, tp = T[c].shape[0], T[c].shape[2]
        dL, dR, dD = B.bdim(A, W, 0), B.bdim(A, W, 2), B.bdim(A, W, 3)
        el = g.standard_normal((7, t, dL))
        x = g.standard_normal((5, tp, dR))
        y = env.apply_theta(c, el, x, dD)
        yo = np.moveaxis(B.theta(el, T[c], A, W, np.moveaxis(x, 0, -1)), -1, 0)
        assert np.abs(y - yo).max() <= tol * np.abs(yo).max(), c
    env.close()


@pytest.mark.parametrize("prec,tol", [("f64", 1e-11), ("f32", 1e-5), ("tf32x3", 1e-5), ("bf16x3", 1e-4)])
def test_site_maps_all_ops_against_oracle(fp, prec, tol):
    """The four site maps of an interior row (Theta, Theta^T, and the right-environment map and its
    transpose of the fit) on every site, element by element against the oracle's theta, theta_t,
    theta_r and theta_r_t; and the adjoint identities <Y, Theta X> = <Theta^T Y, X>,
    <Z, ThetaR X> = <ThetaR^T Z, X> on the GPU results. D=5 with chi=150 puts the environment
    products (K = t * |L| up to 150 * 100) on the tensor cores in the split modes."""
    peps = L.random_peps(4, 4, 5, 4, seed=21)
    pepo = L.fsm_pepo(L.random_hamiltonian(4, 4, 4, 2, seed=21))
    T, _ = B.first_row_boundary(peps[0], pepo[0])
    env = _env(fp, peps, pepo, D=5, w=4, chi=150, prec=prec, seed=5)
    fp.fpeps_absorb_row(env.h, 0, 1)
    fp.fpeps_absorb_row(env.h, 1, 1)
    g = np.random.default_rng(3)
    for c in range(4):
        A, W = peps[1][c], pepo[1][c]
        t, tp = T[c].shape[0], T[c].shape[2]
        dL, dR, dD = B.bdim(A, W, 0), B.bdim(A, W, 2), B.bdim(A, W, 3)
        a, k = 9, 6
        el = g.standard_normal((a, t, dL))
        er = g.standard_normal((a, tp, dR))
        x0 = g.standard_normal((k, tp, dR))
        y1 = g.standard_normal((k, a, dD))
        x2 = g.standard_normal((k, dD, a))
        z3 = g.standard_normal((k, t, dL))
        outs = [env.apply_theta_op(0, c, el, x0, (a, dD)), env.apply_theta_op(1, c, el, y1, (tp, dR)),
                env.apply_theta_op(2, c, er, x2, (t, dL)), env.apply_theta_op(3, c, er, z3, (dD, a))]
        col = lambda v: np.moveaxis(v, 0, -1)
        refs = [B.theta(el, T[c], A, W, col(x0)), B.theta_t(el, T[c], A, W, col(y1)),
                B.theta_r(er, T[c], A, W, col(x2)), B.theta_r_t(er, T[c], A, W, col(z3))]
        for op, (o, r) in enumerate(zip(outs, refs)):
            r = np.moveaxis(r, -1, 0)
            assert o.shape == r.shape, (op, c)
            assert np.abs(o - r).max() <= tol * np.abs(r).max(), (op, c)
        # adjoint pairs on the GPU's own outputs (fresh vectors of the matching shapes)
        ip = lambda u, v: float(np.sum(u.astype(np.float64) * v.astype(np.float64)))
        lhs, rhs = ip(y1, outs[0]), ip(env.apply_theta_op(1, c, el, y1, (tp, dR)), x0)
        assert abs(lhs - rhs) <= 10 * tol * (abs(lhs) + np.linalg.norm(y1) * np.linalg.norm(outs[0])), c
        lhs, rhs = ip(z3, outs[2]), ip(env.apply_theta_op(3, c, er, z3, (dD, a)), x2)
        assert abs(lhs - rhs) <= 10 * tol * (abs(lhs) + np.linalg.norm(z3) * np.linalg.norm(outs[2])), c
    env.close()


@pytest.mark.parametrize("n_fit", [2, 3])
@pytest.mark.parametrize("prec,tol", [("f64", 1e-9), ("tf32x3", 1e-4)])
def test_further_fit_passes_match_oracle(fp, n_fit, prec, tol):
    """n_fit passes of the CBE fit, each after the first starting from the previous one
    re-canonicalised left to right: kept spectra of every bond after the last pass, the row's
    log-scale and the boundary shapes against the oracle's absorb_row (truncated regime,
    D=3, chi=20; the decaying PEPS separates kept from discarded singular values)."""
    peps = L.decaying_peps(4, 4, 3, 4, seed=7)
    pepo = L.fsm_pepo(L.random_hamiltonian(4, 4, 4, 2, seed=7))
    T, _ = B.first_row_boundary(peps[0], pepo[0])
    prm_o = B.RsvdParams(oversample=6, power_iters=2, n_fit=n_fit)
    res = B.absorb_row(T, peps[1], pepo[1], 20, prm_o, seed=5, layer=1, row=1)
    env = _env(fp, peps, pepo, D=3, w=4, chi=20, prec=prec, seed=5)
    fp.fpeps_absorb_row(env.h, 0, 1)
    fp.fpeps_absorb_row(env.h, 1, 1)
    st = fp.fpeps_compress_rsvd(env.h, fp.params(6, 2, 0, n_fit, 0))
    assert abs(st.log_scale - res.log_scale) < tol
    for c in range(3):
        sv = np.array(fp.fpeps_bond_spectrum(env.h, 1, c))
        ref = np.asarray(res.fit_spectra[c])
        assert sv.shape == ref.shape, c
        assert np.abs(sv - ref).max() <= tol * ref.max(), c
    for c in range(4):
        assert fp.fpeps_boundary_shape(env.h, c) == res.T[c].shape
    env.close()


@pytest.mark.parametrize("prec,tol", [("f64", 1e-9), ("tf32x3", 1e-3)])
def test_independent_environments_of_one_handle(fp, prec, tol):
    """n_envs = 3 over one lattice, swept row by row in interleaved order (select 0, 1, 2 for
    every row): environment e gives the oracle's sweep with environment index e in its sketch
    counters, and the three values differ (independent sketches at a truncation that the
    sketch decides: oversampling 2, no power iteration; the oracle's three values lie 2.5e-3 and
    3.8e-3 apart in ln|value|)."""
    peps = L.decaying_peps(4, 4, 2, 4, seed=3)
    pepo = L.fsm_pepo(L.random_hamiltonian(4, 4, 4, 2, seed=3))
    prm_o = B.RsvdParams(oversample=2, power_iters=0, n_fit=1)
    env = fp.Env(peps, pepo, D=2, p=4, w=4, chi=10, prec=prec, seed=5, n_envs=3)
    try:
        for r in range(4):
            for e in range(3):
                env.select(e)
                fp.fpeps_absorb_row(env.h, r, 1)
                if 0 < r < 3:
                    fp.fpeps_compress_rsvd(env.h, fp.params(2, 0, 0, 1, 0))
        got = []
        for e in (2, 0, 1):
            env.select(e)
            got.append((e, fp.fpeps_sweep_value(env.h)))
        with pytest.raises(fp.FpepsError):
            env.select(3)
    finally:
        env.close()
    for e, (sg, lg) in got:
        so, lo = B.contract(peps, pepo, 10, prm_o, seed=5, layer=1, env=e)
        assert sg == so, e
        assert abs(lg - lo) < tol, e
    logs = sorted(v[1] for _, v in got)
    assert logs[1] - logs[0] > 1e-3 and logs[2] - logs[1] > 1e-3


@pytest.mark.parametrize("Lx,Ly,prec,tol", [(1, 1, "f64", 1e-10), (1, 2, "f64", 1e-10), (1, 3, "f64", 1e-10),
                                            (2, 1, "f64", 1e-10), (2, 3, "f64", 1e-10), (3, 1, "f64", 1e-10),
                                            (3, 2, "f64", 1e-10), (2, 3, "tf32x3", 1e-5), (3, 2, "tf32x3", 1e-5)])
def test_degenerate_lattice_shapes_against_brute_force(fp, Lx, Ly, prec, tol):
    """The method's degenerate cases through the public fpeps_expect: one row (closed at once
    against the trivial boundary), two rows (row 0 exact, then closed: no compression), one
    column (every Theta_c has a single column), two columns (zip-up of one site plus the last
    site); D=2, FSM PEPO with two hopping channels, chi above every bond. The split-precision
    mode runs the shapes whose sites the 3x3 tests already send to the tensor-core sandwich."""
    peps = L.random_peps(Lx, Ly, 2, 4, seed=4)
    pepo = L.fsm_pepo(L.random_hamiltonian(Lx, Ly, 4, 2, seed=4))
    num, den = N.brute_force_expectation(peps, pepo)
    env = _env(fp, peps, pepo, D=2, w=4, chi=16, prec=prec, seed=2)
    try:
        val, sn, ln = env.expect(fp.params(10, 0, 0, 1, 1))
    finally:
        env.close()
    assert abs(val / (num / den) - 1) < tol
    assert sn == (1 if num >= 0 else -1)


def test_zip_spectrum_and_apply_theta_match_oracle(fp):
    peps = L.random_peps(4, 4, 2, 4, seed=4)
    pepo = L.fsm_pepo(L.random_hamiltonian(4, 4, 4, 2, seed=4))
    T, _ = B.first_row_boundary(peps[0], pepo[0])
    prm_o = B.RsvdParams(oversample=6, power_iters=2, n_fit=1)
    res = B.absorb_row(T, peps[1], pepo[1], 12, prm_o, seed=5, layer=1, row=1)
    env = _env(fp, peps, pepo, D=2, w=4, chi=12, prec="f64", seed=5)
    fp.fpeps_absorb_row(env.h, 0, 1)
    fp.fpeps_absorb_row(env.h, 1, 1)
    # one Theta application at site 1 with a random left environment
    g = np.random.default_rng(0)
    A, W = peps[1][1], pepo[1][1]
    t, tp = T[1].shape[0], T[1].shape[2]
    dL, dR, dD = B.bdim(A, W, 0), B.bdim(A, W, 2), B.bdim(A, W, 3)
    el = g.standard_normal((5, t, dL))
    x = g.standard_normal((3, tp, dR))
    y = env.apply_theta(1, el, x, dD)
    yo = B.theta(el, T[1], A, W, np.moveaxis(x, 0, -1))            # [a, Dn, k]
    assert np.allclose(np.moveaxis(y, 0, -1), yo, rtol=1e-11, atol=1e-13 * np.abs(yo).max())
    fp.fpeps_compress_rsvd(env.h, fp.params(6, 2, 0, 1, 0))
    for c in range(3):
        sv = np.array(fp.fpeps_bond_spectrum(env.h, 0, c))
        assert np.allclose(sv, res.zip_spectra[c], rtol=1e-9, atol=1e-12 * sv.max())
    for c in range(3):
        sv = np.array(fp.fpeps_bond_spectrum(env.h, 1, c))
        assert np.allclose(sv, res.fit_spectra[c], rtol=1e-9, atol=1e-12 * sv.max())
    # boundary shapes follow the oracle's
    for c in range(4):
        assert fp.fpeps_boundary_shape(env.h, c) == res.T[c].shape
    env.close()


def test_checkpoint_roundtrip_and_state_errors(fp):
    peps = L.random_peps(4, 3, 2, 4, seed=6)
    pepo = L.fsm_pepo(L.random_hamiltonian(4, 3, 4, 2, seed=6))
    env = _env(fp, peps, pepo, D=2, w=4, chi=10, prec="f64", seed=2)
    prm = fp.params(5, 1, 0, 1, 0)
    fp.fpeps_absorb_row(env.h, 0, 1)
    with pytest.raises(fp.FpepsError) as ei:
        fp.fpeps_absorb_row(env.h, 2, 1)          # out of order
    assert ei.value.status == 2
    fp.fpeps_absorb_row(env.h, 1, 1)
    with pytest.raises(fp.FpepsError):
        fp.fpeps_absorb_row(env.h, 2, 1)          # compress pending
    fp.fpeps_compress_rsvd(env.h, prm)
    blob = fp.fpeps_export_boundary(env.h)
    fp.fpeps_absorb_row(env.h, 2, 1)
    fp.fpeps_compress_rsvd(env.h, prm)
    fp.fpeps_absorb_row(env.h, 3, 1)
    v1 = fp.fpeps_sweep_value(env.h)
    fp.fpeps_import_boundary(env.h, blob, 2, 1)
    fp.fpeps_absorb_row(env.h, 2, 1)
    fp.fpeps_compress_rsvd(env.h, prm)
    fp.fpeps_absorb_row(env.h, 3, 1)
    v2 = fp.fpeps_sweep_value(env.h)
    assert v1[0] == v2[0] and abs(v1[1] - v2[1]) < 1e-12
    with pytest.raises(fp.FpepsError) as ei:
        fp.fpeps_compress_rsvd(env.h, prm)        # nothing staged
    assert ei.value.status == 2
    env.close()


def test_product_state_closed_form_on_gpu(fp):
    peps, vecs = L.product_peps(5, 4, 3, 4, seed=8)
    ham = L.random_hamiltonian(5, 4, 4, 2, seed=8)
    env = _env(fp, peps, L.fsm_pepo(ham), D=3, w=4, chi=20, prec="f64", seed=2)
    val, sn, ln = env.expect(fp.params(4, 1, 0, 1, 0))
    env.close()
    assert abs(val - N.product_state_energy(vecs, ham)) < 1e-9 * max(1.0, abs(val))


@pytest.mark.parametrize("decay,prec,tol", [
    (False, "f64", 1e-8),
    # flat random-PEPS spectra: FP32 perturbations shift the near-degenerate kept
    # subspace; the deviation is bounded by the truncation error (~1% here), not by FP32
    (False, "f32", 2e-2), (False, "tf32x3", 2e-2),
    # separated spectra: FP32-class agreement
    (True, "f64", 1e-8), (True, "f32", 1e-5), (True, "tf32x3", 1e-5 * TF32X3_OVER_F32),
    # 3xBF16 (boundary and environment GEMMs): 3 * 2^-16 per product, 64x the 3xTF32 bound
    (False, "bf16x3", 2e-2), (True, "bf16x3", 1e-5 * TF32X3_OVER_F32 * 64)])
def test_c2_against_stored_oracle(fp, decay, prec, tol):
    """4x4, D=4, w=4, chi=64 truncated; oracle values written by tests/golden/make_golden.py."""
    path = os.path.join(HERE, "golden", "c2_fsm_decay_seed0.json" if decay else "c2_fsm_seed0.json")
    gold = json.load(open(path))
    peps = (L.decaying_peps if decay else L.random_peps)(4, 4, 4, 4, seed=gold["peps_seed"])
    pepo = L.fsm_pepo(L.random_hamiltonian(4, 4, 4, 2, seed=gold["ham_seed"]))
    env = _env(fp, peps, pepo, D=4, w=4, chi=64, prec=prec, seed=gold["sketch_seed"])
    val, sn, ln = env.expect(fp.params(10, 2, 0, 1, 0))
    sd, ld = env.norm(fp.params(10, 2, 0, 1, 0))
    env.close()
    assert sn == gold["num_sign"] and sd == gold["den_sign"]
    assert abs(ln - gold["num_log"]) < tol
    assert abs(ld - gold["den_log"]) < tol


@pytest.mark.parametrize("prec,tol", [("f64", 1e-9), ("tf32x3", 1e-5 * TF32X3_OVER_F32)])
def test_k_column_slicing_matches_oracle(fp, monkeypatch, prec, tol):
    """The Theta applications slice their O(chi^2 (DwD)^2) intermediates over the sketch
    columns (chunks of FPEPS_CHUNK_ELEMS elements). A small budget forces several chunks
    (kc < k) in every application, as the 8x8 chi=500 row does (kc = 46 of 510); the result
    must still equal the oracle's, and in FP64 the unsliced run to rounding."""
    peps = L.decaying_peps(4, 4, 2, 4, seed=3)
    pepo = L.fsm_pepo(L.random_hamiltonian(4, 4, 4, 2, seed=3))
    prm_o = B.RsvdParams(oversample=6, power_iters=2, n_fit=1)
    sn_o, ln_o = B.contract(peps, pepo, 12, prm_o, seed=5, layer=1)

    def run(budget):
        if budget:
            monkeypatch.setenv("FPEPS_CHUNK_ELEMS", str(budget))
        else:
            monkeypatch.delenv("FPEPS_CHUNK_ELEMS", raising=False)
        env = _env(fp, peps, pepo, D=2, w=4, chi=12, prec=prec, seed=5)
        for r in range(4):
            fp.fpeps_absorb_row(env.h, r, 1)
            if 0 < r < 3:
                fp.fpeps_compress_rsvd(env.h, fp.params(6, 2, 0, 1, 0))
        v = fp.fpeps_sweep_value(env.h)
        env.close()
        return v

    # per vector, an application holds t * max(U R, L Dn) <= 12 * 16 * 16 = 3072 elements per
    # intermediate here, so 3 * 3072 gives chunks of at most 3 of the 18 sketch columns
    sg, lg = run(3 * 3072)
    assert sg == sn_o and abs(lg - ln_o) < tol
    s0, l0 = run(None)
    assert s0 == sg
    if prec == "f64":
        assert abs(lg - l0) < 1e-11


@pytest.mark.parametrize("prec,tol", [("f64", 1e-8), ("tf32x3", 1e-5 * TF32X3_OVER_F32)])
def test_k_column_slicing_c2_stored_oracle(fp, monkeypatch, prec, tol):
    """C2 (4x4, D=4, chi=64, decaying PEPS) with chunks of 4 sketch columns of 74."""
    gold = json.load(open(os.path.join(HERE, "golden", "c2_fsm_decay_seed0.json")))
    peps = L.decaying_peps(4, 4, 4, 4, seed=gold["peps_seed"])
    pepo = L.fsm_pepo(L.random_hamiltonian(4, 4, 4, 2, seed=gold["ham_seed"]))
    # t * max(U R, L Dn) <= 64 * 64 * 64 elements per vector
    monkeypatch.setenv("FPEPS_CHUNK_ELEMS", str(4 * 64 * 64 * 64))
    env = _env(fp, peps, pepo, D=4, w=4, chi=64, prec=prec, seed=gold["sketch_seed"])
    val, sn, ln = env.expect(fp.params(10, 2, 0, 1, 0))
    env.close()
    assert sn == gold["num_sign"]
    assert abs(ln - gold["num_log"]) < tol


C3ROW = os.path.join(HERE, "golden", "c3_row2_seed0.json")


def _c3_row2(fp, prec):
    """Row 2 of the 6x6, D=6, w=4, chi=256 lattice absorbed into the stored seeded boundary:
    (log-scale, zip-up spectra, fit spectra) of the GPU path."""
    from paper_2511_01039_gb300 import workloads as WL
    gold = json.load(open(C3ROW))
    peps, pepo, bnd = L.interior_row_inputs(gold["Lx"], gold["Ly"], gold["D"], gold["chi"], gold["row"], gold["K"],
                                            gold["input_seed"])
    env = _env(fp, peps, pepo, D=gold["D"], w=gold["K"] + 2, chi=gold["chi"], prec=prec, seed=gold["sketch_seed"])
    fp.fpeps_import_boundary(env.h, WL.boundary_blob(bnd, gold["row"], 1, 8 if prec == "f64" else 4), gold["row"], 1)
    fp.fpeps_absorb_row(env.h, gold["row"], 1)
    st = fp.fpeps_compress_rsvd(env.h, fp.params(10, 2, 0, 1, 0))
    nb = gold["Ly"] - 1
    zs = [np.array(fp.fpeps_bond_spectrum(env.h, 0, c)) for c in range(nb)]
    fs = [np.array(fp.fpeps_bond_spectrum(env.h, 1, c)) for c in range(nb)]
    env.close()
    return gold, st.log_scale, zs, fs


def _spec_err(got, ref):
    """Largest deviation of a kept spectrum, relative to its largest value."""
    ref = np.asarray(ref)
    assert got.shape == ref.shape
    return float(np.max(np.abs(got - ref)) / ref.max())


@pytest.mark.skipif(not os.path.exists(C3ROW), reason="stored C3 row not written (tests/golden/make_golden.py --c3row)")
@pytest.mark.parametrize("prec,tol", [("f64", 1e-8), ("f32", 5e-5), ("tf32x3", 5e-5), ("bf16x3", 1e-4)])
def test_c3_row2_against_stored_oracle(fp, prec, tol):
    """6x6, D=6, w=4 (Hubbard-shaped FSM), chi=256: row 2 absorbed into a seeded boundary MPS by
    the zip-up rSVD and one CBE fit pass (Sec. IV), against the FP64 oracle's stored result:
    the row's log-scale and the kept spectrum of every bond after the zip-up and after the fit.
    FP64 must agree to 1e-8. Measured: FP32 6e-8 / 3.5e-7 / up to 1.1e-5 (log-scale, zip, fit),
    3xTF32 1.5e-6 / 5.3e-6 / 4.7e-6, 3xBF16 3.3e-6 / 3.5e-6 / 2.5e-5; the bounds leave a factor
    of four or more (the fit is a variational step whose result moves with every rounding of
    the zip-up it starts from)."""
    gold, ls, zs, fs = _c3_row2(fp, prec)
    errs = {"log_scale": abs(ls - gold["log_scale"]),
            "zip": max(_spec_err(z, r) for z, r in zip(zs, gold["zip_spectra"])),
            "fit": max(_spec_err(f, r) for f, r in zip(fs, gold["fit_spectra"]))}
    print(f"C3 row 2 {prec}: {errs}")
    assert errs["log_scale"] < tol
    assert errs["zip"] < tol
    assert errs["fit"] < tol


@pytest.mark.skipif(not os.path.exists(C3ROW), reason="stored C3 row not written (tests/golden/make_golden.py --c3row)")
@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
def test_c3_row2_repeatable(fp, prec):
    """The same C3 row twice in one process on the tensor-core path. A pair GEMM whose converters
    read a stage before its fill had landed gave run-to-run differences of 1e-4 on the log-scale
    and 1e-3 on the fit spectra. Without it, 3xTF32 runs agree to ~1e-8; 3xBF16 runs in one
    process have differed by up to 4.4e-6 on the log-scale (its error against FP64 is 3.2e-6),
    while fresh processes reproduce each other: the bound for 3xBF16 is 1e-5."""
    _, ls1, zs1, fs1 = _c3_row2(fp, prec)
    _, ls2, zs2, fs2 = _c3_row2(fp, prec)
    tf = prec == "tf32x3"
    assert abs(ls1 - ls2) < (1e-6 if tf else 1e-5)
    assert max(_spec_err(a, b) for a, b in zip(zs1, zs2)) < (1e-5 if tf else 3e-5)
    assert max(_spec_err(a, b) for a, b in zip(fs1, fs2)) < (5e-5 if tf else 2e-4)
