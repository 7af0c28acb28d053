"""Thin ctypes binding of libfpeps (include/fpeps.h): argument marshalling only.

Every step of the contraction runs in the library's CUDA kernels; this module
only converts Python/PyTorch arguments to the C ABI. It raises if the native
library is missing: there is no fallback implementation.

PyTorch supplies device memory (through the allocator callback, backed by the
caching allocator) and the CUDA stream.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libfpeps.so")

F64, F32, TF32X3, BF16X3 = 0, 1, 2, 3
PRECISIONS = {"f64": F64, "f32": F32, "tf32x3": TF32X3, "bf16x3": BF16X3}
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_STATE", 3: "ERR_OOM", 4: "ERR_CUDA", 5: "ERR_NUMERIC", 6: "ERR_TIMEOUT",
          7: "ERR_UNSUPPORTED"}


class fpeps_config(C.Structure):
    _fields_ = [("Lx", C.c_int32), ("Ly", C.c_int32), ("D", C.c_int32), ("p", C.c_int32), ("w", C.c_int32),
                ("chi", C.c_int32), ("prec", C.c_int), ("seed", C.c_uint64), ("symmetry", C.c_int32),
                ("n_envs", C.c_int32)]


class fpeps_rsvd_params(C.Structure):
    _fields_ = [("oversample", C.c_int32), ("power_iters", C.c_int32), ("chi_tilde", C.c_int32),
                ("n_fit", C.c_int32), ("exact_svd", C.c_int32)]


class fpeps_stats(C.Structure):
    _fields_ = [("seconds", C.c_double), ("alg_flops", C.c_double), ("log_scale", C.c_double),
                ("trunc_err_est", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class fpeps_allocator(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN)]


class FpepsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None

# symbol name -> (restype, argtypes)
SIGNATURES = {
    "fpeps_env_create": (C.c_int, [C.POINTER(fpeps_config), C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                                   C.c_void_p, C.POINTER(fpeps_allocator), C.POINTER(C.c_void_p)]),
    "fpeps_absorb_row": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32]),
    "fpeps_compress_rsvd": (C.c_int, [C.c_void_p, C.POINTER(fpeps_rsvd_params), C.POINTER(fpeps_stats)]),
    "fpeps_sweep_value": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int32)]),
    "fpeps_contract_norm": (C.c_int, [C.c_void_p, C.POINTER(fpeps_rsvd_params), C.POINTER(C.c_double),
                                      C.POINTER(C.c_int32)]),
    "fpeps_expect": (C.c_int, [C.c_void_p, C.POINTER(fpeps_rsvd_params), C.POINTER(C.c_double),
                               C.POINTER(C.c_double), C.POINTER(C.c_int32)]),
    "fpeps_export_boundary": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_size_t)]),
    "fpeps_import_boundary": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_int32, C.c_int32]),
    "fpeps_last_error": (C.c_char_p, [C.c_void_p]),
    "fpeps_env_select": (C.c_int, [C.c_void_p, C.c_int32]),
    "fpeps_theta_block_tasks": (C.c_int, [C.c_int32] + [C.c_void_p, C.c_int32] * 7 +
                                [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_int32)]),
    "fpeps_env_destroy": (None, [C.c_void_p]),
    "fpeps_boundary_shape": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                       C.POINTER(C.c_int32)]),
    "fpeps_bond_spectrum": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.POINTER(C.c_double),
                                      C.POINTER(C.c_int32)]),
    "fpeps_apply_theta": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p,
                                    C.c_void_p]),
    "fpeps_apply_theta_op": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_int32,
                                       C.c_void_p, C.c_void_p]),
    "fpeps_gemm_f32": (C.c_int, [C.c_int32, C.c_int64, C.c_int64, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p,
                                 C.c_int64, C.c_void_p, C.c_void_p]),
    "fpeps_svd_f64": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "fpeps_svd_f64_noalloc": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "fpeps_launch_count": (C.c_int64, []),
    "fpeps_selftest_wait_timeout": (C.c_int, [C.c_void_p]),
    "fpeps_profile": (C.c_int, [C.c_int32]),
    "fpeps_profile_read": (C.c_int, [C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                     C.POINTER(C.c_double)]),
    "fpeps_version": (C.c_char_p, []),
}


def lib():
    """Load libfpeps.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise FpepsError(-1, f"native library missing: {LIB_PATH} (run __graft_entry__.build())")
        _lib = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(_lib, name)
            fn.restype = res
            fn.argtypes = args
    return _lib


def _check(env, st):
    if st != 0:
        msg = lib().fpeps_last_error(env).decode() if env else ""
        raise FpepsError(st, msg)


class TorchAllocator:
    """fpeps_allocator backed by torch's caching allocator (one uint8 tensor per block)."""

    def __init__(self, device):
        import torch
        self.torch = torch
        self.device = device
        self.live = {}
        self._a = ALLOC_FN(self._alloc)
        self._f = FREE_FN(self._free)
        self.struct = fpeps_allocator(None, self._a, self._f)

    def _alloc(self, ctx, nbytes, stream):
        try:
            t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device=self.device)
        except RuntimeError:
            return None
        p = t.data_ptr()
        self.live[p] = t
        return p

    def _free(self, ctx, ptr, stream):
        self.live.pop(ptr, None)


# ------------------------------------------------------------------ same-name wrappers
def fpeps_env_create(cfg: fpeps_config, peps, pepo, dtype_in: int, stream_handle: int, allocator=None,
                     charges=None):
    """peps/pepo: device pointers (int) or torch tensors; charges: None or a contiguous
    int32 numpy array in the layout of the C header (cfg.symmetry must be 1); returns
    the env handle (c_void_p)."""
    import numpy as np
    out = C.c_void_p()
    pp = peps.data_ptr() if hasattr(peps, "data_ptr") else peps
    wp = (pepo.data_ptr() if hasattr(pepo, "data_ptr") else pepo) if pepo is not None else None
    al = C.byref(allocator.struct) if allocator is not None else None
    qp = None
    if charges is not None:
        charges = np.ascontiguousarray(charges, dtype=np.int32)
        qp = charges.ctypes.data
    st = lib().fpeps_env_create(C.byref(cfg), pp, wp, qp, dtype_in, stream_handle, al, C.byref(out))
    _check(None, st)
    return out


def fpeps_absorb_row(env, row: int, layer: int):
    _check(env, lib().fpeps_absorb_row(env, row, layer))


def fpeps_compress_rsvd(env, params: fpeps_rsvd_params):
    st = fpeps_stats()
    _check(env, lib().fpeps_compress_rsvd(env, C.byref(params), C.byref(st)))
    return st


def fpeps_sweep_value(env):
    la, sg = C.c_double(), C.c_int32()
    _check(env, lib().fpeps_sweep_value(env, C.byref(la), C.byref(sg)))
    return sg.value, la.value


def fpeps_contract_norm(env, params: fpeps_rsvd_params):
    la, sg = C.c_double(), C.c_int32()
    _check(env, lib().fpeps_contract_norm(env, C.byref(params), C.byref(la), C.byref(sg)))
    return sg.value, la.value


def fpeps_expect(env, params: fpeps_rsvd_params):
    v, la, sg = C.c_double(), C.c_double(), C.c_int32()
    _check(env, lib().fpeps_expect(env, C.byref(params), C.byref(v), C.byref(la), C.byref(sg)))
    return v.value, sg.value, la.value


def fpeps_export_boundary(env) -> bytes:
    n = C.c_size_t(0)
    _check(env, lib().fpeps_export_boundary(env, None, C.byref(n)))
    buf = (C.c_char * n.value)()
    _check(env, lib().fpeps_export_boundary(env, buf, C.byref(n)))
    return bytes(buf)


def fpeps_import_boundary(env, blob: bytes, next_row: int, layer: int):
    buf = C.create_string_buffer(blob, len(blob))
    _check(env, lib().fpeps_import_boundary(env, buf, len(blob), next_row, layer))


def fpeps_theta_block_tasks(qa, qt, qu, qtp, ql, qr, qd, q, op=0):
    """Task table of the block-sparse Theta_c (op 0) or Theta_c^T (op 1) application to sector q
    (host only): a list of (step, terms, output-block charges, flops per vector)."""
    import numpy as np
    legs = [np.ascontiguousarray(np.asarray(x).reshape(-1, 2), dtype=np.int32) for x in (qa, qt, qu, qtp, ql, qr, qd)]
    qs = np.ascontiguousarray(np.asarray(q).reshape(2), dtype=np.int32)
    args = []
    for x in legs:
        args += [x.ctypes.data, len(x)]
    n = C.c_int32(0)
    _check(None, lib().fpeps_theta_block_tasks(op, *args, qs.ctypes.data, None, None, C.byref(n)))
    tab = np.zeros((max(n.value, 1), 8), dtype=np.int32)
    fl = np.zeros(max(n.value, 1))
    _check(None, lib().fpeps_theta_block_tasks(op, *args, qs.ctypes.data, tab.ctypes.data, fl.ctypes.data,
                                               C.byref(n)))
    out = []
    for i in range(n.value):
        step, terms = int(tab[i, 0]), int(tab[i, 1])
        pairs = [(int(tab[i, 2 + 2 * j]), int(tab[i, 3 + 2 * j])) for j in range(3 if step < 3 else 2)]
        out.append((step, terms, tuple(pairs), float(fl[i])))
    return out


def fpeps_env_select(env, e: int):
    _check(env, lib().fpeps_env_select(env, e))


def fpeps_last_error(env) -> str:
    return lib().fpeps_last_error(env).decode()


def fpeps_env_destroy(env):
    lib().fpeps_env_destroy(env)


def fpeps_boundary_shape(env, c: int):
    a, b, d = C.c_int32(), C.c_int32(), C.c_int32()
    _check(env, lib().fpeps_boundary_shape(env, c, C.byref(a), C.byref(b), C.byref(d)))
    return a.value, b.value, d.value


def fpeps_bond_spectrum(env, which: int, c: int):
    n = C.c_int32(0)
    _check(env, lib().fpeps_bond_spectrum(env, which, c, None, C.byref(n)))
    arr = (C.c_double * max(n.value, 1))()
    _check(env, lib().fpeps_bond_spectrum(env, which, c, arr, C.byref(n)))
    return [arr[i] for i in range(n.value)]


def fpeps_apply_theta(env, c: int, el, x, dn: int, elem_bytes: int):
    """Theta_c of the staged row on host vectors: el [a, t, L], x [k, t', R] -> y [k, a, dn] (numpy)."""
    import numpy as np
    dt = np.float64 if elem_bytes == 8 else np.float32
    el = np.ascontiguousarray(el, dtype=dt)
    x = np.ascontiguousarray(x, dtype=dt)
    a, k = el.shape[0], x.shape[0]
    y = np.zeros((k, a, dn), dtype=dt)
    _check(env, lib().fpeps_apply_theta(env, c, a, el.ctypes.data, k, x.ctypes.data, y.ctypes.data))
    return y


def fpeps_apply_theta_op(env, op: int, c: int, envt, x, out_shape, elem_bytes: int):
    """Site map `op` of the staged row (0: Theta, 1: Theta^T, 2: ThetaR, 3: ThetaR^T) on host
    vectors x [k, ...] with the environment envt [a, bond, bundle]; returns out [k, *out_shape]."""
    import numpy as np
    dt = np.float64 if elem_bytes == 8 else np.float32
    envt = np.ascontiguousarray(envt, dtype=dt)
    x = np.ascontiguousarray(x, dtype=dt)
    k = x.shape[0]
    y = np.zeros((k,) + tuple(out_shape), dtype=dt)
    _check(env, lib().fpeps_apply_theta_op(env, op, c, envt.shape[0], envt.ctypes.data, k, x.ctypes.data,
                                           y.ctypes.data))
    return y


def fpeps_gemm_f32(mode: int, A, B, C, K=None, stream_handle: int = 0):
    """C = A[:, :K] @ B[:, :K].T for torch CUDA float32 tensors (unit inner stride); C [M,N] contiguous."""
    M = A.shape[0]
    K = A.shape[1] if K is None else K
    N = B.shape[0]
    _check(None, lib().fpeps_gemm_f32(mode, M, N, K, A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0),
                                      C.data_ptr(), stream_handle))


def fpeps_svd_f64(M, stream_handle: int = 0):
    """SVD of a square torch float64 CUDA matrix (row-major view of the column-major argument is handled here)."""
    import torch
    k = M.shape[0]
    Mc = M.t().contiguous()             # column-major storage
    U = torch.empty_like(Mc)
    V = torch.empty_like(Mc)
    s = torch.empty(k, dtype=torch.float64, device=M.device)
    _check(None, lib().fpeps_svd_f64(Mc.data_ptr(), k, U.data_ptr(), s.data_ptr(), V.data_ptr(), stream_handle))
    return U.t(), s, V.t()


def fpeps_svd_f64_noalloc(M, stream_handle: int = 0):
    """fpeps_svd_f64 without device allocation in the library (k <= 256)."""
    import torch
    k = M.shape[0]
    Mc = M.t().contiguous()
    U = torch.empty_like(Mc)
    V = torch.empty_like(Mc)
    s = torch.empty(k, dtype=torch.float64, device=M.device)
    _check(None, lib().fpeps_svd_f64_noalloc(Mc.data_ptr(), k, U.data_ptr(), s.data_ptr(), V.data_ptr(),
                                             stream_handle))
    return U.t(), s, V.t()


PROF_KINDS = {0: "gemm_tc_tf32x3", 1: "gemm_simt", 2: "sandwich", 3: "gram", 4: "factor", 5: "sketch"}


def fpeps_launch_count() -> int:
    return lib().fpeps_launch_count()


def fpeps_selftest_wait_timeout(stream_handle: int = 0) -> int:
    """Run the GEMM with its loads withheld; returns the status (ERR_TIMEOUT = the bounded waits worked)."""
    return lib().fpeps_selftest_wait_timeout(stream_handle)


def fpeps_profile(enable: bool):
    _check(None, lib().fpeps_profile(int(enable)))


def fpeps_profile_read(kind: int):
    n, ms, fl, by = C.c_int64(), C.c_double(), C.c_double(), C.c_double()
    _check(None, lib().fpeps_profile_read(kind, C.byref(n), C.byref(ms), C.byref(fl), C.byref(by)))
    return {"launches": n.value, "ms": ms.value, "flops": fl.value, "bytes": by.value}


def fpeps_version() -> str:
    return lib().fpeps_version().decode()


# ------------------------------------------------------------------ convenience
class Env:
    """An fpeps environment on the current CUDA device and stream.

    peps / pepo: lists of lists of site tensors (numpy or torch), packed and copied
    to the device once; ``prec`` one of 'f64', 'f32', 'tf32x3', 'bf16x3'.
    """

    def __init__(self, peps, pepo, *, D, p, w, chi, prec="f64", seed=0, stream=None, use_torch_allocator=True,
                 charges=None, n_envs=1):
        import numpy as np
        import torch
        self.torch = torch
        Lx, Ly = len(peps), len(peps[0])
        self.dev = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream or torch.cuda.current_stream(self.dev)
        dt = torch.float64
        pk = torch.cat([torch.as_tensor(np.asarray(t), dtype=dt).reshape(-1) for row in peps for t in row]).to(self.dev)
        wk = None
        if pepo is not None:
            wk = torch.cat([torch.as_tensor(np.asarray(t), dtype=dt).reshape(-1) for row in pepo for t in row]).to(self.dev)
        self.cfg = fpeps_config(Lx, Ly, D, p, w, chi, PRECISIONS[prec], seed, 1 if charges is not None else 0,
                                n_envs)
        self.elem = 8 if prec == "f64" else 4
        self.alloc = TorchAllocator(self.dev) if use_torch_allocator else None
        torch.cuda.synchronize(self.dev)
        self.h = fpeps_env_create(self.cfg, pk, wk, 0, self.stream.cuda_stream, self.alloc, charges)
        del pk, wk

    def close(self):
        if getattr(self, "h", None):
            fpeps_env_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def select(self, e):
        """Make environment e of the handle the one later calls act on."""
        fpeps_env_select(self.h, e)

    def norm(self, params):
        return fpeps_contract_norm(self.h, params)

    def expect(self, params):
        return fpeps_expect(self.h, params)

    def apply_theta(self, c, el, x, dn):
        """One Theta_c application of the staged row (diagnostic): el [a,t,L], x [k,t',R] -> y [k,a,dn]."""
        return fpeps_apply_theta(self.h, c, el, x, dn, self.elem)

    def apply_theta_op(self, op, c, envt, x, out_shape):
        """One site map of the staged row (diagnostic; layouts of fpeps_apply_theta_op)."""
        return fpeps_apply_theta_op(self.h, op, c, envt, x, out_shape, self.elem)


def pack_charges(qpeps, qpepo=None):
    """Leg charges in the layout of fpeps_env_create: qpeps[r][c] (and qpepo[r][c])
    = (q_l, q_u, q_r, q_d), each an (dim, 2) integer array; PEPS sites first."""
    import numpy as np
    parts = [np.asarray(q, dtype=np.int32).reshape(-1) for row in qpeps for site in row for q in site]
    if qpepo is not None:
        parts += [np.asarray(q, dtype=np.int32).reshape(-1) for row in qpepo for site in row for q in site]
    return np.concatenate(parts)


def params(oversample=10, power_iters=2, chi_tilde=0, n_fit=1, exact_svd=0) -> fpeps_rsvd_params:
    return fpeps_rsvd_params(oversample, power_iters, chi_tilde, n_fit, int(exact_svd))
