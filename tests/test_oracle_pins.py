"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself:
  * a library known-answer test (Philox raw words from numpy),
  * brute-force state vectors and term-by-term Hamiltonians (pin a),
  * an exact contraction in a different order (pin b),
  * closed forms for product states (pin c),
  * exact SVDs when the sketch covers the full rank (pin d),
  * Eckart-Young, isometry (canonical form) and projector identities.
"""
import math

import numpy as np
import pytest

from oracle import boundary as B
from oracle import network as N
from oracle.philox import gaussian_sketch, philox4x64_10
from synth import lattice as L


# ---------------------------------------------------------------- Philox KAT
@pytest.mark.parametrize("key,ctr", [((0, 0), (0, 0, 0, 0)),
                                     ((0x1234567890ABCDEF, 0xFEDCBA9876543210), (5, 6, 7, 8)),
                                     ((2 ** 64 - 1, 17), (2 ** 64 - 3, 2 ** 63, 1, 2 ** 64 - 1))])
def test_philox_matches_numpy_raw(key, ctr):
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(ctr, dtype=np.uint64))
    raw = bg.random_raw(8)
    c = list(ctr)
    outs = []
    for _ in range(2):
        # numpy increments the 256-bit counter before each block of four words
        c[0] = (c[0] + 1) % 2 ** 64
        carry = c[0] == 0
        i = 1
        while carry and i < 4:
            c[i] = (c[i] + 1) % 2 ** 64
            carry = c[i] == 0
            i += 1
        w = philox4x64_10(tuple(np.array([x], dtype=np.uint64) for x in c), key)
        outs.extend(int(x[0]) for x in w)
    assert outs == [int(x) for x in raw]


def test_gaussian_sketch_moments_and_determinism():
    om = gaussian_sketch(4000, 50, seed=7, layer=0, stage=0, site=3, row=2)
    assert abs(om.mean()) < 0.01 and abs(om.var() - 1) < 0.01
    assert abs(((om ** 4).mean()) - 3) < 0.05            # Gaussian fourth moment
    om2 = gaussian_sketch(4000, 50, seed=7, layer=0, stage=0, site=3, row=2)
    assert np.array_equal(om, om2)
    om3 = gaussian_sketch(4000, 50, seed=7, layer=0, stage=1, site=3, row=2)
    assert np.corrcoef(om.ravel(), om3.ravel())[0, 1] < 0.01
    # a sub-block is the same numbers (element (i,j) depends only on i, j and the tags)
    assert np.array_equal(gaussian_sketch(100, 7, seed=7, layer=0, stage=0, site=3, row=2), om[:100, :7])


# ------------------------------------------------------- PEPO / brute force
@pytest.mark.parametrize("Lx,Ly,K", [(3, 3, 0), (3, 3, 2), (2, 3, 4), (3, 2, 1)])
def test_fsm_pepo_equals_term_by_term(Lx, Ly, K):
    peps = L.random_peps(Lx, Ly, 2, 4, seed=11)
    ham = L.random_hamiltonian(Lx, Ly, 4, K, seed=5) if K != 4 else L.hubbard_hamiltonian(Lx, Ly, seed=5, K=4)
    pepo = L.fsm_pepo(ham)
    assert pepo[min(1, Lx - 1)][0].shape[2] == K + 2 or Ly == 1
    num, den = N.brute_force_expectation(peps, pepo)
    psi = N.psi_vector(peps)
    assert den == pytest.approx(psi @ psi, rel=1e-13)
    assert num == pytest.approx(psi @ N.apply_terms(psi, ham), rel=1e-11, abs=1e-14 * abs(den))


def test_fsm_interior_channel_counts():
    ham = L.hubbard_hamiltonian(5, 5, seed=0, K=4)
    W = L.fsm_pepo(ham)[2][2]
    ch = L.pepo_channels(W)
    assert len(ch) == 3 + 4 * 4
    assert len({(l, d) for (l, u, r, d) in ch}) == 2 + 2 * 4


def test_columnwise_exact_equals_brute_force():
    peps = L.random_peps(3, 3, 2, 4, seed=2)
    pepo = L.dense_pepo(3, 3, 4, 2, seed=3)
    num, _ = N.brute_force_expectation(peps, pepo)
    assert N.exact_columnwise(peps, pepo) == pytest.approx(num, rel=1e-11)


def test_product_state_brute_force_closed_form():
    peps, vecs = L.product_peps(3, 3, 2, 4, seed=4)
    ham = L.random_hamiltonian(3, 3, 4, 2, seed=4)
    num, den = N.brute_force_expectation(peps, L.fsm_pepo(ham))
    assert den == pytest.approx(1.0, abs=1e-13)
    assert num == pytest.approx(N.product_state_energy(vecs, ham), rel=1e-12)


# ------------------------------------------------------ the boundary method
def _value(sign, log):
    return sign * math.exp(log)


@pytest.mark.parametrize("pepo_kind,chi", [("identity", 16), ("dense2", 64), ("fsm2", 64), ("fsm4", 256)])
def test_boundary_equals_brute_force_3x3(pepo_kind, chi):
    """Pin (a): 3x3, D=2, exact-rank sketch and chi >= the largest rank of any Theta_c
    (B^2 for bundle B = D w D at the middle site): the boundary method reproduces <psi|O|psi>."""
    peps = L.random_peps(3, 3, 2, 4, seed=0)
    if pepo_kind == "identity":
        pepo = L.identity_pepo(3, 3, 4)
    elif pepo_kind == "dense2":
        pepo = L.dense_pepo(3, 3, 4, 2, seed=1)
    elif pepo_kind == "fsm2":
        pepo = L.fsm_pepo(L.random_hamiltonian(3, 3, 4, 0, seed=1))
    else:
        pepo = L.fsm_pepo(L.random_hamiltonian(3, 3, 4, 2, seed=1))
    num, _ = N.brute_force_expectation(peps, pepo)
    for n_fit in (0, 1, 2):
        prm = B.RsvdParams(exact_svd=True, n_fit=n_fit, power_iters=0)
        s, lv = B.contract(peps, pepo, chi, prm, seed=9, layer=1)
        assert _value(s, lv) == pytest.approx(num, rel=1e-10)


def test_boundary_untruncated_4x4_equals_columnwise():
    """Pin (b): chi = 64 = largest bond of a 4x4, D=2, w=2 lattice: no truncation, any order agrees."""
    peps = L.random_peps(4, 4, 2, 4, seed=3)
    pepo = L.fsm_pepo(L.random_hamiltonian(4, 4, 4, 0, seed=3))
    ex = N.exact_columnwise(peps, pepo)
    for n_fit in (0, 1, 2):
        s, lv = B.contract(peps, pepo, 64, B.RsvdParams(n_fit=n_fit), seed=1, layer=1)
        assert _value(s, lv) == pytest.approx(ex, rel=1e-10)


@pytest.mark.parametrize("Lx,Ly,D,chi", [(4, 4, 3, 20), (5, 3, 2, 12)])
def test_product_state_closed_form_by_boundary(Lx, Ly, D, chi):
    """Pin (c): rank-1 bonds, rank-deficient sketches: norm 1 and the closed-form energy."""
    peps, vecs = L.product_peps(Lx, Ly, D, 4, seed=8)
    ham = L.random_hamiltonian(Lx, Ly, 4, 2, seed=8)
    prm = B.RsvdParams(oversample=4, power_iters=1, n_fit=1)
    s, lv = B.contract(peps, L.identity_pepo(Lx, Ly, 4), chi, prm, seed=2, layer=0)
    assert _value(s, lv) == pytest.approx(1.0, rel=1e-10)
    s, lv = B.contract(peps, L.fsm_pepo(ham), chi, prm, seed=2, layer=1)
    assert _value(s, lv) == pytest.approx(N.product_state_energy(vecs, ham), rel=1e-9)


def _site_setup(seed=0, D=2, w_K=2):
    """A middle site of a 4x4 lattice with a random boundary and a random left environment."""
    peps = L.random_peps(4, 4, D, 4, seed=seed)
    pepo = L.fsm_pepo(L.random_hamiltonian(4, 4, 4, w_K, seed=seed))
    A, W = peps[1][1], pepo[1][1]
    g = np.random.default_rng(seed)
    dU = B.bdim(A, W, 1)
    dL = B.bdim(A, W, 0)
    T = g.standard_normal((5, dU, 6))
    EL = g.standard_normal((3, 5, dL))
    return EL, T, A, W


def test_orth_full_rank_is_lapack_thin_qr():
    """Thin QR of Sec. IV: for full-rank Y the factor is LAPACK's Householder Q
    with diag(R) > 0 (unique), so the column order and nesting are those of QR."""
    g = np.random.default_rng(11)
    Y = g.standard_normal((60, 12)) @ np.diag(np.logspace(0, -5, 12))
    Qh, R = np.linalg.qr(Y)
    Qh = Qh * np.where(np.diag(R) < 0, -1.0, 1.0)[None, :]
    assert np.allclose(B.orth(Y), Qh, atol=1e-12)


def test_orth_dependent_columns_become_zero():
    """A column in the span of the ones before it (exactly, or zero) gives a zero
    column in place; the others are the QR factor of the independent columns,
    and the non-zero columns span range(Y)."""
    g = np.random.default_rng(12)
    X = g.standard_normal((40, 6))
    Y = np.column_stack([X[:, 0], X[:, 1], X[:, 0] - 3 * X[:, 1], X[:, 2], np.zeros(40), X[:, 3],
                         X[:, 2] * 1e-2, X[:, 4]])
    Q = B.orth(Y)
    zero = np.abs(Q).sum(axis=0) == 0
    assert zero.tolist() == [False, False, True, False, True, False, True, False]
    ind = Y[:, ~zero]
    Qh, R = np.linalg.qr(ind)
    Qh = Qh * np.where(np.diag(R) < 0, -1.0, 1.0)[None, :]
    assert np.allclose(Q[:, ~zero], Qh, atol=1e-12)
    assert np.allclose(Q @ (Q.T @ Y), Y, atol=1e-12)
    # a wide matrix has no thin QR in this reading (callers handle that case)
    with pytest.raises(ValueError):
        B.orth(np.ones((3, 4)))


def test_rsvd_equals_exact_svd_when_sketch_covers_rank():
    """Pin (d): with k >= rank(Theta) the rSVD spectrum and subspace are exact."""
    EL, T, A, W = _site_setup()
    th = B.form_theta(EL, T, A, W)
    rows, cols = th.shape
    sv = np.linalg.svd(th, compute_uv=False)
    rank = int((sv > 1e-12 * sv[0]).sum())
    k = min(rows, cols)
    assert k >= rank
    tp, dR = T.shape[2], B.bdim(A, W, 2)
    a, dDn = EL.shape[0], B.bdim(A, W, 3)
    om = gaussian_sketch(cols, k, seed=3, layer=0, stage=0, site=1, row=1)
    ap = lambda X: B.theta(EL, T, A, W, X.reshape(tp, dR, -1)).reshape(rows, -1)
    apt = lambda Y: B.theta_t(EL, T, A, W, Y.reshape(a, dDn, -1)).reshape(cols, -1)
    Q, ub, s, vt = B.rsvd(ap, apt, om, q=1)
    assert np.allclose(s[:rank], sv[:rank], rtol=1e-12, atol=1e-12 * sv[0])
    # principal angles between the leading left subspaces are zero
    U, _, _ = np.linalg.svd(th)
    P = (Q @ ub[:, :rank]).T @ U[:, :rank]
    assert np.allclose(np.linalg.svd(P, compute_uv=False), 1.0, atol=1e-10)
    # transpose map is the transpose
    X = np.random.default_rng(1).standard_normal((cols, 3))
    Yv = np.random.default_rng(2).standard_normal((rows, 3))
    assert np.allclose(ap(X), th @ X) and np.allclose(apt(Yv), th.T @ Yv)


def test_rsvd_eckart_young_lower_bound():
    EL, T, A, W = _site_setup(seed=4, D=2, w_K=2)
    th = B.form_theta(EL, T, A, W)
    rows, cols = th.shape
    sv = np.linalg.svd(th, compute_uv=False)
    chi = 10
    om = gaussian_sketch(cols, chi + 5, seed=1, layer=0, stage=0, site=0, row=0)
    Q, ub, s, vt = B.rsvd(lambda X: th @ X, lambda Y: th.T @ Y, om, q=2)
    Uk = Q @ ub[:, :chi]
    err = np.linalg.norm(th - Uk @ (Uk.T @ th))
    opt = math.sqrt((sv[chi:] ** 2).sum())
    assert err >= opt * (1 - 1e-12)
    assert err <= 2.0 * opt                    # q = 2 subspace iteration is near-optimal here
    assert np.all(s[:chi] <= sv[:chi] * (1 + 1e-12))   # Ritz values never exceed the true ones


def test_zipup_and_fit_canonical_forms():
    peps = L.random_peps(4, 4, 2, 4, seed=6)
    pepo = L.fsm_pepo(L.random_hamiltonian(4, 4, 4, 2, seed=6))
    T, _ = B.first_row_boundary(peps[0], pepo[0])
    prm = B.RsvdParams(oversample=5, power_iters=1)
    N_, ELs, _, sp = B.zipup(T, peps[1], pepo[1], 12, prm, seed=0, layer=1, row=1)
    for c, n in enumerate(N_[:-1]):
        m = n.reshape(-1, n.shape[2])
        assert np.allclose(m.T @ m, np.eye(m.shape[1]), atol=1e-12)
        w = gaussian_sketch(m.shape[0], 1, seed=0, layer=1, stage=2, site=c, row=1)[:, 0]
        assert np.all(w @ m >= 0)                # sign gauge
    newT, _, _ = B.cbe_fit(T, peps[1], pepo[1], N_, ELs, 12, prm, seed=0, layer=1, row=1)
    for c, n in enumerate(newT[1:], start=1):
        m = n.reshape(n.shape[0], -1)
        assert np.allclose(m @ m.T, np.eye(m.shape[0]), atol=1e-12)
        w = gaussian_sketch(m.shape[1], 1, seed=0, layer=1, stage=2, site=c, row=1)[:, 0]
        assert np.all(m @ w >= 0)
    assert abs(np.linalg.norm(newT[0]) - 1) < 1e-12


def test_cbe_two_cluster_subtraction_equals_explicit_projectors():
    """Fig. 5: Theta2s(Omega) - Theta2s(P Omega), then the left projector, equals P_L^perp Theta2s P_R^perp Omega."""
    g = np.random.default_rng(0)
    m, n, a = 30, 24, 5
    th2 = g.standard_normal((m, n))
    V = np.linalg.qr(g.standard_normal((n, a)))[0].T          # orthonormal rows (right isometry)
    Nl = np.linalg.qr(g.standard_normal((m, a)))[0]           # orthonormal columns (left isometry)
    om = g.standard_normal((n, 7))
    y = th2 @ om - th2 @ (V.T @ (V @ om))
    y = y - Nl @ (Nl.T @ y)
    explicit = (np.eye(m) - Nl @ Nl.T) @ th2 @ (np.eye(n) - V.T @ V) @ om
    assert np.allclose(y, explicit, atol=1e-12)


def test_cbe_fit_improves_truncated_fidelity():
    """The fit is expected (not guaranteed) to beat the zip-up; here it must on a clear case."""
    peps = L.random_peps(4, 4, 3, 4, seed=1)
    pepo = L.identity_pepo(4, 4, 4)
    ex = N.exact_columnwise(peps, pepo)
    s0, l0 = B.contract(peps, pepo, 8, B.RsvdParams(n_fit=0, oversample=4), seed=1, layer=0)
    s1, l1 = B.contract(peps, pepo, 8, B.RsvdParams(n_fit=1, oversample=4), seed=1, layer=0)
    e0 = abs(_value(s0, l0) / ex - 1)
    e1 = abs(_value(s1, l1) / ex - 1)
    assert e1 < e0
