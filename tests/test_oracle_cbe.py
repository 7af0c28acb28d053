"""Pins of the oracle's CBE expansion step (Sec. IV, Fig. 3-5) in the truncated regime.

The fit's expansion takes the truncated complement of
A = P_L^perp Theta2s P_R^perp, where Theta2s is the two-site matrix of the bond
(c-1, c). The oracle applies A without forming it (two-cluster subtraction of
Fig. 5 on top of the layered sandwich). Here everything is formed explicitly
and densely, independently of the oracle's maps:

  * the site sandwich C[L, U, R, Dn] = sum_{p,p'} A[.., p] W[.., p, p'] A[.., p'],
  * Theta2s = EL . T_{c-1} . C_{c-1} . T_c . C_c . ER as one matrix,
  * the projectors I - V^T V and I - N N^T as matrices,

and the oracle's expansion vectors and fitted spectra are checked against
numpy.linalg.svd of those matrices:

  (i)   with a sketch covering the rank, the expansion vectors span the top
        singular subspace of the explicit A (principal angles), its singular
        values equal the oracle's;
  (ii)  with chi_tilde covering the whole complement, V' spans the whole
        bond space and the kept spectrum of the fitted bond equals the exact
        SVD of the explicit Theta2s (Eckart-Young optimal truncation);
  (iii) planted mistakes (the tangent projector in place of its complement,
        on either side; the right projector missing from the transpose; the
        CBE width not clipped to the complement) each fail (i) or (ii).

Dropping the left projector altogether is not a mistake these pins (or any
exact-arithmetic pin) can see: N_{c-1}^T Theta2s is the centre tensor, whose
row space is V, so P_L Theta2s P_R^perp vanishes identically; that identity is
checked on the explicit matrices instead.
"""
import numpy as np
import pytest

from oracle import boundary as B
from synth import lattice as L


def _sandwich_dense(A, W):
    """C[(l,lw,l'), (u,uw,u'), (r,rw,r'), (d,dw,d')]: ket, PEPO, bra; bra fastest."""
    c = np.einsum("lurdp,LURDpq,wxyzq->lLwuUxrRydDz", A, W, A)
    dims = [A.shape[i] * W.shape[i] * A.shape[i] for i in range(4)]
    return c.reshape(dims)


def _two_site_dense(EL, Tl, Al, Wl, Tc, Ac, Wc, ER):
    """Explicit Theta2s: rows (a_{c-2}, Dn_{c-1}), columns (Dn_c, a_c), last index fastest."""
    C1 = _sandwich_dense(Al, Wl)
    C2 = _sandwich_dense(Ac, Wc)
    m = np.einsum("atL,tUs,LUPd,sVz,PVRD,bzR->adDb", EL, Tl, C1, Tc, C2, ER, optimize=True)
    return m.reshape(m.shape[0] * m.shape[1], m.shape[2] * m.shape[3])


def _run_fit(chi, chi_tilde, oversample, seed=2, D=2, K=2, Ly=4, dense=False):
    """Zip-up + CBE fit of row 1 of a 4 x Ly lattice (FSM PEPO with K hopping channels,
    or a dense random w=2 PEPO); returns the trace, the fitted spectra and the inputs."""
    peps = L.random_peps(4, Ly, D, 4, seed=seed)
    if dense:
        pepo = L.dense_pepo(4, Ly, 4, 2, seed=seed)
    else:
        pepo = L.fsm_pepo(L.random_hamiltonian(4, Ly, 4, K, seed=seed))
    T, _ = B.first_row_boundary(peps[0], pepo[0])
    prm = B.RsvdParams(oversample=oversample, power_iters=1, chi_tilde=chi_tilde)
    N_, ELs, _, _ = B.zipup(T, peps[1], pepo[1], chi, prm, seed=seed, layer=1, row=1)
    trace = []
    _, _, spectra = B.cbe_fit(T, peps[1], pepo[1], N_, ELs, chi, prm, seed=seed, layer=1, row=1, trace=trace)
    return trace, spectra, T, peps[1], pepo[1]


def _theta2s(tr, T, Arow, Wrow):
    c = tr["c"]
    return _two_site_dense(tr["EL"], T[c - 1], Arow[c - 1], Wrow[c - 1], T[c], Arow[c], Wrow[c], tr["ER"])


def check_complement_subspace(chi=6, chi_tilde=4):
    """(i): exact sketches; the expansion vectors are the top right singular vectors of
    the explicit P_L^perp Theta2s P_R^perp. Returns the number of bonds checked."""
    trace, _, T, Arow, Wrow = _run_fit(chi, chi_tilde, oversample=400)
    checked = 0
    for tr in trace:
        ct = tr["ct"]
        if ct <= 0:
            continue
        th = _theta2s(tr, T, Arow, Wrow)
        V, Nl = tr["V"], tr["Nlm"]
        assert th.shape == (tr["rows_a"], tr["cols_a"])
        A = (np.eye(th.shape[0]) - Nl @ Nl.T) @ th @ (np.eye(th.shape[1]) - V.T @ V)
        _, sv, vt = np.linalg.svd(A)
        assert tr["k"] >= int((sv > 1e-12 * sv[0]).sum())          # the sketch covers rank(A)
        r = min(len(tr["sigma_a"]), len(sv))
        assert np.allclose(tr["sigma_a"][:r], sv[:r], rtol=1e-9, atol=1e-11 * sv[0])
        # principal angles between the expansion and the exact top-ct subspace
        assert sv[ct - 1] - sv[ct] > 1e-3 * sv[0], "no gap at the cut: pick another seed"
        cos = np.linalg.svd(tr["Vtil"] @ vt[:ct].T, compute_uv=False)
        assert np.allclose(cos, 1.0, atol=1e-8)
        # expansion vectors are orthogonal to V and the expanded basis is orthonormal
        assert np.abs(tr["Vtil"] @ V.T).max() < 1e-10
        assert np.allclose(tr["Vp"] @ tr["Vp"].T, np.eye(tr["Vp"].shape[0]), atol=1e-10)
        checked += 1
    return checked


def check_full_complement_is_optimal(chi=6, chi_tilde=200, **kw):
    """(ii): the CBE width covers the rank of the explicit P_L^perp Theta2s P_R^perp, so
    V' contains the row space of Theta2s and the fitted spectrum is the exact top-chi
    spectrum of Theta2s (Eckart-Young). Returns the number of bonds checked."""
    trace, spectra, T, Arow, Wrow = _run_fit(chi, chi_tilde, oversample=400, **kw)
    checked = 0
    for tr in trace:
        th = _theta2s(tr, T, Arow, Wrow)
        V, Nl, Vp = tr["V"], tr["Nlm"], tr["Vp"]
        A = (np.eye(th.shape[0]) - Nl @ Nl.T) @ th @ (np.eye(th.shape[1]) - V.T @ V)
        sa = np.linalg.svd(A, compute_uv=False)
        rank_a = int((sa > 1e-10 * sa[0]).sum()) if sa[0] > 0 else 0
        assert tr["ct"] >= rank_a, "the CBE width must cover the complement here"
        assert np.linalg.norm(th - (th @ Vp.T) @ Vp) <= 1e-10 * np.linalg.norm(th)
        sv = np.linalg.svd(th, compute_uv=False)
        keep = len(tr["spectrum"])
        assert keep == min(chi, th.shape[0], th.shape[1])
        assert np.allclose(tr["spectrum"], sv[:keep], rtol=1e-9, atol=1e-12 * sv[0])
        assert np.allclose(spectra[tr["c"] - 1], sv[:keep], rtol=1e-9, atol=1e-12 * sv[0])
        checked += 1
    return checked


def test_cbe_explicit_two_site_matches_oracle_maps():
    """The dense Theta2s of this file equals the oracle's layered two-site map on the
    basis of the centre's columns (so (i) and (ii) compare like with like)."""
    trace, _, T, Arow, Wrow = _run_fit(6, 4, oversample=400)
    tr = trace[1]
    c = tr["c"]
    th = _theta2s(tr, T, Arow, Wrow)
    dDn = B.bdim(Arow[c], Wrow[c], 3)
    a_c = tr["cols_a"] // dDn
    X = np.random.default_rng(0).standard_normal((tr["cols_a"], 3))
    z = B.theta_r(tr["ER"], T[c], Arow[c], Wrow[c], X.reshape(dDn, a_c, -1))
    y = B.theta(tr["EL"], T[c - 1], Arow[c - 1], Wrow[c - 1], z).reshape(tr["rows_a"], -1)
    assert np.allclose(y, th @ X, rtol=1e-11, atol=1e-12 * np.abs(y).max())


def test_cbe_complement_is_top_subspace_of_explicit_projected_matrix():
    assert check_complement_subspace() >= 2


@pytest.mark.parametrize("kw", [dict(chi=6, chi_tilde=4), dict(chi=4, chi_tilde=3, Ly=5, dense=True)])
def test_left_isometry_maps_two_site_matrix_to_the_centre(kw):
    """N_{c-1}^T Theta2s is the centre tensor at c (the zip-up remainder EL_c = N^T Theta_{c-1}
    and the right environment of the fit meet there), so its rows lie in span(V) and
    P_L Theta2s P_R^perp = 0: in exact arithmetic the left projector of A acts as the
    identity on Theta2s P_R^perp, and dropping it cannot change any value (it only
    removes rounding in that direction). Checked on the explicit matrices."""
    trace, _, T, Arow, Wrow = _run_fit(oversample=400, **kw)
    for tr in trace:
        th = _theta2s(tr, T, Arow, Wrow)
        V, Nl = tr["V"], tr["Nlm"]
        centre = Nl.T @ th
        assert np.linalg.norm(centre - (centre @ V.T) @ V) <= 1e-10 * np.linalg.norm(th)


@pytest.mark.parametrize("kw", [dict(chi=6), dict(chi=4, Ly=5, dense=True)])
def test_cbe_full_complement_gives_exact_truncation(kw):
    assert check_full_complement_is_optimal(**kw) >= 3


# ---------------------------------------------------------------- planted mistakes
def _ops_left_tangent_instead_of_complement(two_site, two_site_t, V, Nlm):
    def a(X):
        y = two_site(X) - two_site(V.T @ (V @ X))
        return Nlm @ (Nlm.T @ y)

    def at(Y):
        z = two_site_t(Nlm @ (Nlm.T @ Y))
        return z - V.T @ (V @ z)
    return a, at


def _ops_tangent_instead_of_complement(two_site, two_site_t, V, Nlm):
    def a(X):
        y = two_site(V.T @ (V @ X))
        return y - Nlm @ (Nlm.T @ y)

    def at(Y):
        z = two_site_t(Y) - two_site_t(Nlm @ (Nlm.T @ Y))
        return V.T @ (V @ z)
    return a, at


def _ops_transpose_without_right_projector(two_site, two_site_t, V, Nlm):
    def a(X):
        y = two_site(X) - two_site(V.T @ (V @ X))
        return y - Nlm @ (Nlm.T @ y)

    def at(Y):
        return two_site_t(Y) - two_site_t(Nlm @ (Nlm.T @ Y))
    return a, at


@pytest.mark.parametrize("wrong", [_ops_left_tangent_instead_of_complement, _ops_tangent_instead_of_complement,
                                   _ops_transpose_without_right_projector])
def test_planted_projector_mistakes_are_caught(monkeypatch, wrong):
    monkeypatch.setattr(B, "cbe_operator", wrong)
    with pytest.raises(AssertionError):
        check_complement_subspace()


def test_unclipped_cbe_width_is_caught(monkeypatch):
    """chi_tilde clipped to the full matrix instead of the complement: the expanded
    basis would exceed the bond space (a wide thin QR) or overlap V."""
    monkeypatch.setattr(B, "cbe_width", lambda chi_t, rows_a, nl, cols_a, nr: min(chi_t, rows_a, cols_a))
    with pytest.raises((AssertionError, ValueError)):
        check_full_complement_is_optimal()
