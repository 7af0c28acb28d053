"""Pins of the oracle's second and later fit passes (n_fit > 1, Sec. IV / Fig. 3): the
left-to-right re-canonicalisation between passes, and the passes themselves.

Everything here is checked against quantities formed independently of the oracle's
layered maps: the boundary MPS and the exactly absorbed row contracted into full
vectors over the physical bundles, and the left environments contracted site by site
with the dense sandwich C[L, U, R, Dn] (one einsum per site).

  * recanonicalize keeps the state: the MPS before and after agree as vectors; every
    new site but the last is a left isometry;
  * its left environments equal the explicit contraction of the rows above with the
    new isometries (in any regime);
  * untruncated, two passes give back the exactly absorbed row;
  * a second and a third pass move the compressed row closer to the exactly absorbed
    row (a variational fit; the distance falls from pass to pass on these cases);
  * the exact regimes with n_fit = 2 are in test_oracle_pins.py (brute force, 3x3;
    column-wise exact, 4x4).
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


def _mps_vector(F):
    """Contract an MPS [a_{c-1}, Dn_c, a_c] (end bonds 1) into one vector over (Dn_0, ..)."""
    v = F[0].reshape(-1, F[0].shape[2])
    for f in F[1:]:
        v = np.einsum("xa,aDb->xDb", v, f).reshape(-1, f.shape[2])
    return v.reshape(-1)


def _exact_row(T, Arow, Wrow):
    """The row absorbed into the boundary without truncation, as one vector over (Dn_0, ..)."""
    v = np.ones((1, 1, 1))   # [physical so far, t, L]
    for c in range(len(T)):
        C = _sandwich_dense(Arow[c], Wrow[c])
        v = np.einsum("xtL,tUs,LURD->xDsR", v, T[c], C, optimize=True)
        v = v.reshape(-1, v.shape[2], v.shape[3])
    return v.reshape(-1)


def _explicit_envs(T, Arow, Wrow, N):
    """EL_{c+1}[a_c, t', R] = sum over the sites <= c of N x T x C (dense), normalised."""
    E = np.ones((1, 1, 1))
    out = [E]
    for c in range(len(T) - 1):
        C = _sandwich_dense(Arow[c], Wrow[c])
        E = np.einsum("atL,tUs,LURD,aDb->bsR", E, T[c], C, N[c], optimize=True)
        E = E / np.linalg.norm(E)
        out.append(E)
    return out


def _row_setup(seed, D=2, K=2, Ly=4):
    peps = L.random_peps(4, Ly, D, 4, seed=seed)
    pepo = L.fsm_pepo(L.random_hamiltonian(4, Ly, 4, K, seed=seed))
    T, _ = B.first_row_boundary(peps[0], pepo[0])
    return T, peps[1], pepo[1]


@pytest.mark.parametrize("seed,chi", [(1, 8), (2, 6)])
def test_recanonicalize_keeps_state_and_gives_left_isometries(seed, chi):
    T, Arow, Wrow = _row_setup(seed)
    prm = B.RsvdParams(oversample=4, power_iters=1)
    N, ELs, _, _ = B.zipup(T, Arow, Wrow, chi, prm, seed=seed, layer=1, row=1)
    F, _, _ = B.cbe_fit(T, Arow, Wrow, N, ELs, chi, prm, seed=seed, layer=1, row=1)
    N2, ELs2 = B.recanonicalize(T, Arow, Wrow, F)
    assert np.allclose(_mps_vector(N2), _mps_vector(F), atol=1e-12)
    assert abs(np.linalg.norm(_mps_vector(F)) - 1) < 1e-12
    for n in N2[:-1]:
        m = n.reshape(-1, n.shape[2])
        g = m.T @ m
        live = np.diag(g) > 0.5                      # numerically dependent columns are zero
        assert np.allclose(g, np.diag(live.astype(float)), atol=1e-12)
    for got, ref in zip(ELs2, _explicit_envs(T, Arow, Wrow, N2)):
        assert got.shape == ref.shape
        assert np.allclose(got, ref, atol=1e-12)


def test_two_fit_passes_reproduce_the_exact_row_when_untruncated():
    """chi above every bond: after two fit passes the compressed row (times its scale) is the
    exactly absorbed row, as a vector over the physical bundles."""
    T, Arow, Wrow = _row_setup(5)
    ex = _exact_row(T, Arow, Wrow)
    res = B.absorb_row(T, Arow, Wrow, 400, B.RsvdParams(oversample=6, power_iters=1, n_fit=2), seed=5, layer=1,
                       row=1)
    v = _mps_vector(res.T) * np.exp(res.log_scale)
    assert np.linalg.norm(v - ex) <= 1e-10 * np.linalg.norm(ex)


@pytest.mark.parametrize("seed,chi", [(1, 8), (2, 6), (3, 10), (4, 4)])
def test_further_fit_passes_approach_the_exact_row(seed, chi):
    """Distance of the compressed row (times its scale) to the exactly absorbed row:
    zip-up only > one fit pass > two passes >= three passes (measured here: a second
    pass gains 6-16 %, a third under 1 %)."""
    T, Arow, Wrow = _row_setup(seed)
    ex = _exact_row(T, Arow, Wrow)
    errs = []
    for n_fit in (0, 1, 2, 3):
        res = B.absorb_row(T, Arow, Wrow, chi, B.RsvdParams(oversample=4, power_iters=1, n_fit=n_fit), seed=seed,
                           layer=1, row=1)
        v = _mps_vector(res.T) * np.exp(res.log_scale)
        errs.append(np.linalg.norm(v - ex) / np.linalg.norm(ex))
    assert errs[1] < errs[0]
    assert errs[2] < errs[1] * 0.97
    assert errs[3] <= errs[2] * (1 + 1e-9)


def test_second_pass_uses_its_own_sketch_stage():
    """Pass p draws its CBE sketch at stage 1 + 16 (p - 1): the second pass's sketch differs
    from the first's, and neither collides with the zip-up's (0) or the gauge's (2)."""
    assert [B.fit_stage(p) for p in (1, 2, 3)] == [1, 17, 33]
    assert len({0, 2, B.fit_stage(1), B.fit_stage(2), B.fit_stage(3)}) == 5


def _broken_factor_not_carried(T, Arow, Wrow, F):
    """Planted mistake: each site is split by QR but the factor is dropped instead of carried."""
    Ly = len(F)
    EL = np.ones((1, 1, 1))
    N, ELs = [], [EL]
    for c in range(Ly - 1):
        X = F[c]
        a1, dDn, ac = X.shape
        Q = B.orth(X.reshape(a1 * dDn, ac))
        Nc = Q.reshape(a1, dDn, ac)
        N.append(Nc)
        el = np.moveaxis(B.theta_t(EL, T[c], Arow[c], Wrow[c], Nc), -1, 0)
        EL = el / np.linalg.norm(el)
        ELs.append(EL)
    N.append(F[Ly - 1] / np.linalg.norm(F[Ly - 1]))
    return N, ELs


def _broken_old_environments(T, Arow, Wrow, F):
    """Planted mistake: the isometries are re-canonicalised but the environments are built
    from the fitted (right-canonical) tensors instead of the new left isometries."""
    N, _ = B.recanonicalize(T, Arow, Wrow, F)
    EL = np.ones((1, 1, 1))
    ELs = [EL]
    for c in range(len(F) - 1):
        el = np.moveaxis(B.theta_t(EL, T[c], Arow[c], Wrow[c], F[c]), -1, 0)
        EL = el / np.linalg.norm(el)
        ELs.append(EL)
    return N, ELs


@pytest.mark.parametrize("broken", [_broken_factor_not_carried, _broken_old_environments])
def test_planted_recanonicalisation_mistakes_are_caught(broken):
    """Each planted mistake breaks the state-and-environment pin above on a truncated row."""
    T, Arow, Wrow = _row_setup(1)
    prm = B.RsvdParams(oversample=4, power_iters=1)
    N, ELs, _, _ = B.zipup(T, Arow, Wrow, 8, prm, seed=1, layer=1, row=1)
    F, _, _ = B.cbe_fit(T, Arow, Wrow, N, ELs, 8, prm, seed=1, layer=1, row=1)
    N2, ELs2 = broken(T, Arow, Wrow, F)
    same_state = np.allclose(_mps_vector(N2), _mps_vector(F), atol=1e-10)
    envs_ok = all(a.shape == b.shape and np.allclose(a, b, atol=1e-10)
                  for a, b in zip(ELs2, _explicit_envs(T, Arow, Wrow, N2)))
    assert not (same_state and envs_ok)
