"""The scratch-free SVD entry point (fpeps_svd_f64_noalloc) against the
allocating one (fpeps_svd_f64), through the C ABI.

It is meant for callers that cannot allocate device memory during the call;
its working storage is a fixed array inside the library that every call
reuses. Two calls in a row with different inputs must each reproduce the
allocating entry point, and sizes beyond the fixed array must be refused.
This file is collected last so that a stop at the first failure has already
run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fp():
    import torch
    from paper_2511_01039_gb300 import fpeps
    torch.cuda.set_device(0)
    fpeps.lib()
    return fpeps


def _case(k, seed):
    g = np.random.default_rng(seed)
    A0 = g.standard_normal((k, k)) @ np.diag(np.logspace(0, -5, k)) @ g.standard_normal((k, k))
    return np.linalg.qr(A0)[1].T.copy()     # the path factorises R^T of a thin QR


# one-block and whole-GPU Jacobi; 256 is the largest k the array holds (its counter area ends
# exactly at the end of the array)
@pytest.mark.parametrize("k", [64, 200, 256])
def test_noalloc_svd_matches_allocating_svd_twice(fp, k):
    import torch
    for seed in (1, 2):                    # two calls in a row: the shared array is reused
        M = torch.tensor(_case(k, seed + k), device="cuda")
        U0, s0, V0 = fp.fpeps_svd_f64(M)
        U1, s1, V1 = fp.fpeps_svd_f64_noalloc(M)
        s0n = s0.cpu().numpy()
        assert np.allclose(s1.cpu().numpy(), s0n, rtol=1e-12, atol=1e-14 * s0n[0])
        assert np.allclose(V1.cpu().numpy(), V0.cpu().numpy(), atol=1e-10)
        assert np.allclose(U1.cpu().numpy(), U0.cpu().numpy(), atol=1e-10)
        A = M.cpu().numpy()
        assert np.allclose((U1.cpu().numpy() * s1.cpu().numpy()) @ V1.cpu().numpy().T, A, atol=1e-12 * s0n[0])


def test_noalloc_svd_rejects_k_beyond_its_array(fp):
    import torch
    M = torch.eye(257, dtype=torch.float64, device="cuda")
    with pytest.raises(fp.FpepsError) as ei:
        fp.fpeps_svd_f64_noalloc(M)
    assert ei.value.status == 1
