"""Kernel-level parity through the C ABI (fpeps_gemm_f32): the tensor-core
3xTF32 GEMM and the CUDA-core FP32 GEMM against an FP64 evaluation of the same
product, on ragged shapes that span several tiles. Products with M <= 128 run on
single CTAs (128x128 tiles), larger ones on CTA pairs (256x192 tiles); M = 129
and 257 leave most rows of a pair's second CTA outside the matrix, and N = 260,
300, 2000, 4097 (or N < 192) leave a partial last column tile of a pair."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fp():
    import torch
    from paper_2511_01039_gb300 import fpeps
    torch.cuda.set_device(0)
    fpeps.lib()
    return fpeps


@pytest.mark.parametrize("M,N,K,pad", [(300, 260, 100, 0), (128, 128, 32, 0), (1000, 2000, 512, 4),
                                       (4100, 700, 1000, 12), (130, 4097, 36, 0), (500, 432, 108000, 0),
                                       (260, 300, 4100, 8), (500, 60, 108000, 0), (64, 256, 1000, 0),
                                       (1, 9, 40, 0), (3000, 7, 500, 4), (129, 300, 2000, 0),
                                       (257, 64, 33, 3)])
@pytest.mark.parametrize("mode", ["tf32x3", "f32", "bf16x3"])
def test_gemm_against_fp64(fp, M, N, K, pad, mode):
    import torch
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N)
    A = torch.randn(M, K + pad, device="cuda", generator=g)
    B = torch.randn(N, K + pad, device="cuda", generator=g)
    C = torch.full((M, N), float("nan"), device="cuda")
    fp.fpeps_gemm_f32(fp.PRECISIONS[mode], A, B, C, K=K)
    ref = (A[:, :K].double() @ B[:, :K].double().T)
    scale = (A[:, :K].double().abs() @ B[:, :K].double().abs().T)
    err = ((C.double() - ref).abs() / scale).max().item()
    # 3xTF32: products exact to ~2^-21 relative, FP32 accumulation; 3xBF16: each product carries
    # up to 3 * 2^-16 relative error (the BF16 rounding of the lo parts and the dropped lo * lo)
    bf = mode == "bf16x3"
    assert err < (1e-4 if bf else 4e-6), err
    # relative to the result itself (random signs: |C| ~ sqrt(K) |a||b|): long K must not drift
    # (one FP32 TMEM accumulator over K = 108000 drifted to ~1e-3; K slices of 2048 keep it FP32-class)
    rel = ((C.double() - ref).abs().max() / ref.abs().max()).item()
    # FP32-class bound: u * sqrt(K) with u = 2^-24 (plain FP32 accumulation is ~2e-5 at K = 1e5);
    # 3xBF16: the per-product bound, random signs
    assert rel < (5e-4 if bf else max(1e-5, 1e-7 * K ** 0.5)), rel
    assert torch.isfinite(C).all()


def test_gemm_tc_rejects_unsupported_shapes(fp):
    """K below one 32-wide k-box, or rows not 16-byte aligned (TMA strides)."""
    import torch
    for K, ld in [(16, 16), (34, 34)]:
        A = torch.randn(64, ld, device="cuda")
        B = torch.randn(256, ld, device="cuda")
        C = torch.empty(64, 256, device="cuda")
        with pytest.raises(fp.FpepsError) as ei:
            fp.fpeps_gemm_f32(fp.TF32X3, A, B, C, K=K)
        assert ei.value.status == 7


@pytest.mark.parametrize("k", [7, 64, 97, 200, 511, 1024])
def test_svd_f64_against_lapack(fp, k):
    """One-sided Jacobi (single block for k <= 96; above, whole-GPU cooperative over blocks of
    two columns, with a dummy block for odd block counts (k = 97) and a one-column block for
    odd k) vs numpy's SVD."""
    import numpy as np
    import torch
    g = np.random.default_rng(k)
    A0 = g.standard_normal((k, k)) @ np.diag(np.logspace(0, -6, k)) @ g.standard_normal((k, k))
    # the path factorises R^T of a thin QR (Jacobi preconditioned by QR)
    A = np.linalg.qr(A0)[1].T.copy()
    M = torch.tensor(A, device="cuda")
    U, s, V = fp.fpeps_svd_f64(M)
    s_ref = np.linalg.svd(A, compute_uv=False)
    # relative accuracy of the small values is limited by the reference's own ~eps*sigma_max
    assert np.allclose(s.cpu().numpy(), s_ref, rtol=1e-7, atol=1e-13 * s_ref[0])
    Un, Vn = U.cpu().numpy(), V.cpu().numpy()
    assert np.allclose((Un * s.cpu().numpy()) @ Vn.T, A, atol=1e-12 * s_ref[0])
    assert np.allclose(Vn.T @ Vn, np.eye(k), atol=1e-12)


def test_bounded_waits_time_out_and_context_survives(fp):
    """Failure detection without a GPU fault: the GEMM runs with its TMA loads
    withheld (on a single CTA and on a CTA pair), every mbarrier wait runs out
    after its bound (~1 s), the kernel reports ERR_TIMEOUT through its error word,
    and the next products on the same context are correct."""
    import torch
    assert fp.fpeps_selftest_wait_timeout() == 6      # FPEPS_ERR_TIMEOUT
    g = torch.Generator(device="cuda").manual_seed(3)
    for M in (100, 300):
        A = torch.randn(M, 64, device="cuda", generator=g)
        B = torch.randn(200, 64, device="cuda", generator=g)
        C = torch.empty(M, 200, device="cuda")
        fp.fpeps_gemm_f32(fp.TF32X3, A, B, C)
        ref = A.double() @ B.double().T
        assert ((C.double() - ref).abs().max() / ref.abs().max()).item() < 1e-5
