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
    cfg = fpeps.fpeps_config(3, 3, 2, 4, 1, 8, 0, 0, 0, 2)       # batched environments not built
    st = fpeps.lib().fpeps_env_create(ctypes.byref(cfg), 1, None, None, 0, None, None, ctypes.byref(out))
    assert st == 7
    cfg = fpeps.fpeps_config(3, 3, 2, 4, 1, 8, 3, 0, 0, 1)       # 3xBF16 not built
    st = fpeps.lib().fpeps_env_create(ctypes.byref(cfg), 1, None, None, 0, None, None, ctypes.byref(out))
    assert st == 7
    cfg = fpeps.fpeps_config(3, 3, 2, 4, 1, 8, 9, 0, 0, 1)       # bad precision enum
    st = fpeps.lib().fpeps_env_create(ctypes.byref(cfg), 1, None, None, 0, None, None, ctypes.byref(out))
    assert st == 1
    assert fpeps.lib().fpeps_absorb_row(None, 0, 0) == 1
    assert fpeps.lib().fpeps_last_error(None) == b"env is NULL"
    fpeps.lib().fpeps_env_destroy(None)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2511_01039_gb300 import fpeps
    monkeypatch.setattr(fpeps, "_lib", None)
    monkeypatch.setattr(fpeps, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(fpeps.FpepsError):
        fpeps.lib()
