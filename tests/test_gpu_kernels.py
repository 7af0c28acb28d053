"""Kernel-level parity through the C ABI (fpeps_gemm_f32): the tensor-core
3xTF32 GEMM and the CUDA-core FP32 GEMM against an FP64 evaluation of the same
product, on ragged shapes that span several 128x128x32 tiles."""
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
                                       (4100, 700, 1000, 12), (130, 4097, 36, 0)])
@pytest.mark.parametrize("mode", ["tf32x3", "f32"])
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
    # 3xTF32: products exact to ~2^-21 relative, FP32 accumulation
    assert err < 4e-6, err
    assert torch.isfinite(C).all()


def test_gemm_tc_rejects_unsupported_shapes(fp):
    import torch
    A = torch.randn(64, 32, device="cuda")
    B = torch.randn(256, 32, device="cuda")
    C = torch.empty(64, 256, device="cuda")
    with pytest.raises(fp.FpepsError) as ei:
        fp.fpeps_gemm_f32(fp.TF32X3, A, B, C)
    assert ei.value.status == 7


@pytest.mark.parametrize("k", [7, 64, 200, 511])
def test_svd_f64_against_lapack(fp, k):
    """One-sided Jacobi (single block for k <= 96, whole-GPU cooperative above) vs numpy's SVD."""
    import numpy as np
    import torch
    g = np.random.default_rng(k)
    A = g.standard_normal((k, k)) @ np.diag(np.logspace(0, -6, k)) @ g.standard_normal((k, k))
    M = torch.tensor(A, device="cuda")
    U, s, V = fp.fpeps_svd_f64(M)
    s_ref = np.linalg.svd(A, compute_uv=False)
    assert np.allclose(s.cpu().numpy(), s_ref, rtol=1e-10, atol=1e-13 * s_ref[0])
    Un, Vn = U.cpu().numpy(), V.cpu().numpy()
    assert np.allclose((Un * s.cpu().numpy()) @ Vn.T, A, atol=1e-12 * s_ref[0])
    assert np.allclose(Vn.T @ Vn, np.eye(k), atol=1e-12)
