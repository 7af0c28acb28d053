"""Pins of the U(1) x U(1) symmetric oracle (block-sparse mode: zip-up and CBE fit).

What fixes it independently of its own code:
  * the generators' tensors obey the charge rules (checked entry by entry);
  * every sandwich site conserves the bundle charge Q = q_ket - q_pepo - q_bra
    (checked on the explicit sandwich tensor of the dense network code);
  * with no truncation, <H> equals the brute-force state-vector value;
  * with truncation and exact sector SVDs, the kept spectra and the contracted
    value equal the dense oracle's exact truncated SVD (the exact SVD of a
    block-diagonal matrix is the union of its blocks' SVDs, so a wrong global
    truncation or sector bookkeeping fails);
  * the same holds for the CBE fit: exact sector SVDs reproduce the dense
    oracle's exact fit (spectra and value);
  * the new boundary tensors conserve charge with the bond charges returned,
    after the zip-up and after the fit;
  * a wrong sign in the bundle charge (a planted mistake) is caught by the
    block-diagonality check;
  * in the approximate regime (a sector's rank above the sketch width) the kept
    Ritz values never exceed the exact singular values (interlacing) and the
    kept vectors are orthonormal and sector-pure.
"""
import numpy as np
import pytest

from oracle import boundary as B
from oracle import network as NW
from oracle import symmetric as S
from synth import lattice as L
from synth import u1


def _lattice(Lx, Ly, D, seed, hubbard=True):
    peps, ch = u1.u1_peps(Lx, Ly, D, seed)
    qpeps = [[u1.peps_leg_charges(ch, Lx, Ly, r, c) for c in range(Ly)] for r in range(Lx)]
    if hubbard:
        ham = L.hubbard_hamiltonian(Lx, Ly, seed)
        W, qW = L.fsm_pepo(ham), u1.hubbard_pepo_charges(ham)
    else:
        z = np.zeros((1, 2), dtype=np.int64)
        W, qW = L.identity_pepo(Lx, Ly, 4), [[(z, z, z, z)] * Ly for _ in range(Lx)]
    return peps, ch, qpeps, W, qW


def test_generators_conserve_charge():
    Lx, Ly = 3, 4
    peps, ch, qpeps, W, qW = _lattice(Lx, Ly, 3, 2)
    for r in range(Lx):
        for c in range(Ly):
            ql, qu, qr, qd = qpeps[r][c]
            bal = u1.site_balance(ql, qu, qr, qd, u1.HUB_CHARGES)
            nz = peps[r][c] != 0
            assert nz.any()
            assert np.all(np.all(bal == ch["flux"][r][c], axis=-1)[nz])
            wl, wu, wr, wd = qW[r][c]
            assert W[r][c].shape[:4] == (len(wl), len(wu), len(wr), len(wd))
            balw = u1.site_balance(wl, wu, wr, wd, u1.HUB_CHARGES)[..., None, :] - u1.HUB_CHARGES
            assert np.all(np.all(balw == 0, axis=-1)[W[r][c] != 0])


def test_sandwich_conserves_bundle_charge():
    Lx, Ly = 3, 3
    peps, ch, qpeps, W, qW = _lattice(Lx, Ly, 3, 4)
    for r, c in [(0, 0), (1, 1), (1, 2), (2, 1)]:
        C = NW.sandwich_full(peps[r][c], W[r][c])            # [L, U, R, Dn]
        QL, QU, QR, QD = S.site_bundles(qpeps[r][c], qW[r][c])
        assert C.shape == (len(QL), len(QU), len(QR), len(QD))
        bal = QL[:, None, None, None] + QU[None, :, None, None] - QR[None, None, :, None] - QD[None, None, None, :]
        nz = C != 0
        assert nz.any()
        assert np.all(np.all(bal == 0, axis=-1)[nz])


def test_untruncated_energy_equals_brute_force():
    peps, _, qpeps, W, qW = _lattice(3, 3, 2, 0)
    e, _, _ = S.expectation_u1(peps, qpeps, W, qW, 10 ** 6, B.RsvdParams(n_fit=0, exact_svd=True), seed=0)
    num, den = NW.brute_force_expectation(peps, W)
    assert den > 0
    assert abs(e - num / den) <= 1e-10 * abs(num / den)


# The truncated comparisons need a cut between distinct singular values: a cut
# through a degenerate cluster has no unique kept subspace (the double layer has
# exact degeneracies between sectors, e.g. from ket <-> bra exchange in the norm
# network). The Hubbard case below (3x4, D=2, seed 5) has its clusters away from
# chi = 4, 6, 12 at every bond (chi = 8 would cut a fourfold cluster).
CUT_CASE = (3, 4, 2, 5)


@pytest.mark.parametrize("chi", [4, 6, 12])
def test_exact_sector_svd_equals_dense_exact_truncation(chi):
    """Truncating zip-up: sector-wise exact SVD + global truncation = dense exact SVD."""
    peps, _, qpeps, W, qW = _lattice(*CUT_CASE)
    prm = B.RsvdParams(n_fit=0, exact_svd=True)
    s_u1, l_u1, rows_u1 = S.contract_u1(peps, qpeps, W, qW, chi, prm, seed=0, layer=1, return_rows=True)
    s_d, l_d, rows_d = B.contract(peps, W, chi, prm, seed=0, layer=1, return_rows=True)
    assert s_u1 == s_d
    assert abs(l_u1 - l_d) < 1e-10
    for ru, rd in zip(rows_u1, rows_d):
        for su, sd in zip(ru.zip_spectra, rd.zip_spectra):
            m = min(len(su), len(sd))
            # the dense bond may carry extra exactly-null vectors beyond the total sector rank
            assert np.all(sd[m:] <= 1e-12 * sd[0])
            assert np.allclose(np.sort(su)[::-1][:m], sd[:m], rtol=0, atol=1e-12 * sd[0])


def test_new_boundary_conserves_charge():
    """N[c][a_{c-1}, Dn_c, a_c] is nonzero only where q_a(c-1) = Q_Dn + q_a(c)."""
    Lx, Ly = 3, 4
    peps, _, qpeps, W, qW = _lattice(Lx, Ly, 2, 5)
    bundles = [[S.site_bundles(qpeps[r][c], qW[r][c]) for c in range(Ly)] for r in range(Lx)]
    T, _ = B.first_row_boundary(peps[0], W[0])
    qT = S.first_row_charges(bundles[0])
    N, _, _, _, qN = S.zipup_u1(T, qT, peps[1], W[1], bundles[1], 16, B.RsvdParams(n_fit=0), seed=3, layer=1,
                                row=1)
    qa = np.zeros((1, 2), dtype=np.int64)
    for c in range(Ly):
        QD = bundles[1][c][3]
        bal = qa[:, None, None, :] - QD[None, :, None, :] - qN[c][None, None, :, :]
        nz = N[c] != 0
        assert nz.any()
        assert np.all(np.all(bal == 0, axis=-1)[nz])
        qa = qN[c]


def test_wrong_bundle_charge_is_caught(monkeypatch):
    """Planted mistake: the PEPO charge enters the bundle with the wrong sign."""
    peps, _, qpeps, W, qW = _lattice(3, 3, 2, 0)

    def wrong(qk, qw, qb):
        return (qk[:, None, None, :] + qw[None, :, None, :] - qb[None, None, :, :]).reshape(-1, 2)

    monkeypatch.setattr(S, "bundle_charges", wrong)
    with pytest.raises((AssertionError, ValueError)):
        S.contract_u1(peps, qpeps, W, qW, 8, B.RsvdParams(n_fit=0), seed=0, layer=1)


@pytest.mark.parametrize("chi", [4, 12])
def test_exact_sector_fit_equals_dense_exact_fit(chi):
    """CBE fit (Fig. 3-5) with exact sector SVDs = the dense oracle's exact fit (an
    oversampling beyond every rank makes the CBE sketches exact on both sides)."""
    peps, _, qpeps, W, qW = _lattice(*CUT_CASE)
    prm = B.RsvdParams(n_fit=1, exact_svd=True, chi_tilde=2, oversample=10 ** 4)
    s_u1, l_u1, rows_u1 = S.contract_u1(peps, qpeps, W, qW, chi, prm, seed=0, layer=1, return_rows=True)
    s_d, l_d, rows_d = B.contract(peps, W, chi, prm, seed=0, layer=1, return_rows=True)
    assert s_u1 == s_d
    assert abs(l_u1 - l_d) < 1e-10
    for ru, rd in zip(rows_u1, rows_d):
        for su, sd in zip(ru.fit_spectra, rd.fit_spectra):
            m = min(len(su), len(sd))
            assert np.all(sd[m:] <= 1e-12 * sd[0])
            assert np.allclose(np.sort(su)[::-1][:m], sd[:m], rtol=0, atol=1e-11 * sd[0])


def test_fitted_boundary_conserves_charge():
    """After the zip-up and the CBE fit, T[c][a_{c-1}, Dn_c, a_c] conserves charge."""
    Lx, Ly = 3, 4
    peps, _, qpeps, W, qW = _lattice(Lx, Ly, 2, 5)
    bundles = [[S.site_bundles(qpeps[r][c], qW[r][c]) for c in range(Ly)] for r in range(Lx)]
    T, _ = B.first_row_boundary(peps[0], W[0])
    qT = S.first_row_charges(bundles[0])
    prm = B.RsvdParams(n_fit=1, chi_tilde=2)
    N, ELs, _, _, qN = S.zipup_u1(T, qT, peps[1], W[1], bundles[1], 6, prm, seed=3, layer=1, row=1)
    F, _, _, qF = S.cbe_fit_u1(T, qT, peps[1], W[1], bundles[1], N, qN, ELs, 6, prm, seed=3, layer=1, row=1)
    qa = np.zeros((1, 2), dtype=np.int64)
    for c in range(Ly):
        QD = bundles[1][c][3]
        bal = qa[:, None, None, :] - QD[None, :, None, :] - qF[c][None, None, :, :]
        nz = F[c] != 0
        assert nz.any()
        assert np.all(np.all(bal == 0, axis=-1)[nz])
        qa = qF[c]


def test_sector_rsvd_ritz_values_bounded_by_exact():
    """Approximate regime (sectors wider than the sketch): every kept Ritz value is at most
    the exact singular value of the same rank (interlacing within each sector, hence
    for the sorted union), and the kept vectors are orthonormal and block-pure."""
    Lx, Ly = 3, 3
    peps, _, qpeps, W, qW = _lattice(Lx, Ly, 3, 6)
    bundles = [[S.site_bundles(qpeps[r][c], qW[r][c]) for c in range(Ly)] for r in range(Lx)]
    T, _ = B.first_row_boundary(peps[0], W[0])
    qT = S.first_row_charges(bundles[0])
    # Theta of row 1 at site 0 (trivial left environment): rows Dn_0, columns (t_0, R_0)
    Th = B.form_theta(np.ones((1, 1, 1)), T[0], peps[1][0], W[1][0])
    QD, QR = bundles[1][0][3], bundles[1][0][2]
    rowq = -QD
    colq = (qT[0][:, None, :] + QR[None, :, :]).reshape(-1, 2)
    chi, prm = 3, B.RsvdParams(n_fit=0, oversample=1, power_iters=1)
    ranks = []
    for q in S._sectors(rowq, colq):
        sv = np.linalg.svd(Th[np.ix_(np.all(rowq == q, axis=1), np.all(colq == q, axis=1))], compute_uv=False)
        ranks.append(int((sv > 1e-12 * sv.max()).sum()))
    assert max(ranks) > chi + prm.oversample          # a sector is sketched, not solved exactly
    om = lambda k: np.random.default_rng(1).standard_normal((Th.shape[1], k))
    U, s, Vt, qk, _ = S.sector_rsvd(lambda X: Th @ X, lambda Y: Th.T @ Y, rowq, colq, chi, prm, om)
    exact = np.linalg.svd(Th, compute_uv=False)[:len(s)]
    assert np.all(np.sort(s)[::-1] <= exact * (1 + 1e-12))
    live = s > 1e-12 * s.max()
    assert live.any()
    assert np.allclose(U[:, live].T @ U[:, live], np.eye(live.sum()), atol=1e-12)
    assert np.allclose(Vt[live] @ Vt[live].T, np.eye(live.sum()), atol=1e-12)
    for m in range(len(s)):
        assert np.all(U[~np.all(rowq == qk[m], axis=1), m] == 0)
        assert np.all(Vt[m, ~np.all(colq == qk[m], axis=1)] == 0)
