"""Full-size parity on sampled outputs (8x8, D=6, w=6 Hubbard FSM PEPO, chi=500,
and the 6x6, D=6, w=4, chi=256 configuration).

The oracle cannot run a whole chi=500 row in a test, but it can apply
Theta_c of the central site to a few vectors: the GPU path (tensor-core GEMMs
and sandwich, launch configuration of the benchmark) applies the same matrix
through fpeps_apply_theta and the results are compared element by element.
"""
import numpy as np
import pytest

from oracle import boundary as B

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tol", [("tf32x3", 1e-5), ("f32", 5e-5)])
@pytest.mark.parametrize("workload", ["C4", "C3"])
def test_central_site_theta_full_size(prec, tol, workload):
    """C4: 8x8, D=6, w=6, chi=500 (row 4); C3: 6x6, D=6, w=4, chi=256 (row 2): Theta_c on two
    vectors and Theta_c^T on two vectors."""
    import torch
    from paper_2511_01039_gb300 import fpeps as fp
    from paper_2511_01039_gb300 import workloads as WL
    torch.cuda.set_device(0)
    w = WL.hubbard_row(**getattr(WL, workload))
    env = fp.Env(w.peps, w.pepo, D=w.D, p=w.p, w=w.w, chi=w.chi, prec=prec, seed=1)
    fp.fpeps_import_boundary(env.h, WL.boundary_blob(w.boundary, w.row, 1, 4), w.row, 1)
    fp.fpeps_absorb_row(env.h, w.row, 1)
    c = w.Ly // 2 - 1
    A, W, T = w.peps[w.row][c], w.pepo[w.row][c], w.boundary[c]
    t, tp = T.shape[0], T.shape[2]
    dL, dR, dD = B.bdim(A, W, 0), B.bdim(A, W, 2), B.bdim(A, W, 3)
    g = np.random.default_rng(7)
    el = g.standard_normal((w.chi, t, dL)).astype(np.float32)
    x = g.standard_normal((2, tp, dR)).astype(np.float32)
    y = env.apply_theta(c, el, x, dD)
    # the transpose map on two vectors of the output space (the first step of every subspace iteration)
    yin = g.standard_normal((2, w.chi, dD)).astype(np.float32)
    z = env.apply_theta_op(1, c, el, yin, (tp, dR))
    env.close()
    f64 = lambda v: v.astype(np.float32).astype(np.float64)
    yo = B.theta(f64(el), f64(T), f64(A), f64(W), np.moveaxis(x, 0, -1).astype(np.float64))
    yo = np.moveaxis(yo, -1, 0)
    # inputs rounded to FP32 on both sides; the environment GEMM sums K = t * |L| = 108000 terms
    err = np.abs(y - yo).max() / np.abs(yo).max()
    assert err < tol, err
    zo = np.moveaxis(B.theta_t(f64(el), f64(T), f64(A), f64(W), np.moveaxis(yin, 0, -1).astype(np.float64)), -1, 0)
    err_t = np.abs(z - zo).max() / np.abs(zo).max()
    assert err_t < tol, err_t
