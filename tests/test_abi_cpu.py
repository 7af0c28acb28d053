"""Host-side checks of the C-ABI library: it builds for sm_103a, loads, and exports
every symbol that include/fpeps.h declares. No compute calls (no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    from paper_2511_01039_gb300 import build
    return build.build()


def _declared():
    src = open(os.path.join(ROOT, "include", "fpeps.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fpeps_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary_calls():
    names = _declared()
    for n in ["fpeps_env_create", "fpeps_absorb_row", "fpeps_compress_rsvd", "fpeps_contract_norm", "fpeps_expect",
              "fpeps_export_boundary", "fpeps_import_boundary", "fpeps_last_error", "fpeps_env_destroy"]:
        assert n in names


def test_library_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(built)
    for n in _declared():
        assert hasattr(lib, n), n


def test_binding_signatures_cover_header(built):
    from paper_2511_01039_gb300 import fpeps
    assert set(_declared()) <= set(fpeps.SIGNATURES)
    assert fpeps.fpeps_version().startswith("fpeps-gb300")


def test_create_rejects_bad_arguments_without_gpu(built):
    """Argument validation happens before any CUDA call."""
    from paper_2511_01039_gb300 import fpeps
    out = ctypes.c_void_p()
    cfg = fpeps.fpeps_config(0, 3, 2, 4, 1, 8, 0, 0, 0, 1)
    st = fpeps.lib().fpeps_env_create(ctypes.byref(cfg), 1, None, None, 0, None, None, ctypes.byref(out))
    assert st == 1 and not out.value
    cfg = fpeps.fpeps_config(3, 3, 2, 4, 1, 8, 0, 0, 1, 1)       # charge sectors without charges
    st = fpeps.lib().fpeps_env_create(ctypes.byref(cfg), 1, None, None, 0, None, None, ctypes.byref(out))
    assert st == 1
    q = (ctypes.c_int32 * 4)()
    cfg = fpeps.fpeps_config(3, 3, 2, 4, 1, 8, 0, 0, 0, 1)       # charges without charge sectors
    st = fpeps.lib().fpeps_env_create(ctypes.byref(cfg), 1, None, q, 0, None, None, ctypes.byref(out))
    assert st == 1
    cfg = fpeps.fpeps_config(3, 3, 2, 4, 1, 8, 0, 0, 2, 1)       # unknown symmetry
    st = fpeps.lib().fpeps_env_create(ctypes.byref(cfg), 1, None, None, 0, None, None, ctypes.byref(out))
    assert st == 1
    for n_envs in (0, -1, 1025):                                  # environments: 1 .. FPEPS_MAX_ENVS
        cfg = fpeps.fpeps_config(3, 3, 2, 4, 1, 8, 0, 0, 0, n_envs)
        st = fpeps.lib().fpeps_env_create(ctypes.byref(cfg), 1, None, None, 0, None, None, ctypes.byref(out))
        assert st == 1 and not out.value
    cfg = fpeps.fpeps_config(3, 3, 2, 4, 1, 8, 9, 0, 0, 1)       # bad precision enum
    st = fpeps.lib().fpeps_env_create(ctypes.byref(cfg), 1, None, None, 0, None, None, ctypes.byref(out))
    assert st == 1
    assert fpeps.lib().fpeps_absorb_row(None, 0, 0) == 1
    assert fpeps.lib().fpeps_env_select(None, 0) == 1
    assert fpeps.lib().fpeps_last_error(None) == b"env is NULL"
    fpeps.lib().fpeps_env_destroy(None)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2511_01039_gb300 import fpeps
    monkeypatch.setattr(fpeps, "_lib", None)
    monkeypatch.setattr(fpeps, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(fpeps.FpepsError):
        fpeps.lib()


def test_pack_charges_layout():
    """Charge marshalling follows the header: PEPS sites (legs l,u,r,d, dim pairs each),
    then PEPO sites, row-major, int32."""
    import numpy as np
    from paper_2511_01039_gb300 import fpeps
    from synth import lattice as L
    from synth import u1
    Lx, Ly, D = 3, 4, 2
    peps, ch = u1.u1_peps(Lx, Ly, D, 1)
    qpeps = [[u1.peps_leg_charges(ch, Lx, Ly, r, c) for c in range(Ly)] for r in range(Lx)]
    ham = L.hubbard_hamiltonian(Lx, Ly, 1)
    W, qW = L.fsm_pepo(ham), u1.hubbard_pepo_charges(ham)
    q = fpeps.pack_charges(qpeps, qW)
    assert q.dtype == np.int32
    n_a = sum(2 * sum(peps[r][c].shape[:4]) for r in range(Lx) for c in range(Ly))
    n_w = sum(2 * sum(W[r][c].shape[:4]) for r in range(Lx) for c in range(Ly))
    assert q.size == n_a + n_w
    # first site: legs l, u, r, d in order, each (dim, 2) flattened
    ql, qu, qr, qd = qpeps[0][0]
    head = np.concatenate([ql.reshape(-1), qu.reshape(-1), qr.reshape(-1), qd.reshape(-1)])
    assert np.array_equal(q[:head.size], head)
    assert fpeps.pack_charges(qpeps).size == n_a
