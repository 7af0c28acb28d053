"""U(1) x U(1) symmetric zip-up compression (oracle; test infrastructure).

Block-sparse mode of the row absorption. The paper slices its contractions by
quantum numbers (Sec. III) and runs the Hubbard model with U(1) x U(1)
symmetric tensors (Sec. V). With charge-conserving PEPS and PEPO every matrix
the compression factorises is block diagonal in the charge of the cut bond, so
the randomized SVD runs sector by sector and one global truncation keeps the
chi largest singular values over all sectors; each kept vector brings its
sector's charge onto the new bond.

This module restates that on top of the dense FP64 oracle: the matrix
applications are the dense ones of ``oracle.boundary`` (structural zeros stay
exact zeros), restricted to one sector's rows and columns by index masks, and
every restricted application checks that nothing leaks out of the sector.

Charges are pairs (N_up, N_dn) (see ``synth.u1`` for the tensors' rules):
  double-layer bundle (x, x_w, x'):   Q = q_ket - q_pepo - q_bra
    (then every sandwich site conserves Q: Q_L + Q_U = Q_R + Q_Dn)
  boundary tensor T[t, U, t']:         q_t = Q_U + q_t'
  zip-up matrix Theta_c at site c:     rows (a, Dn) carry q_a - Q_Dn,
                                       columns (t', R) carry q_t' + Q_R.

Readings where the paper is silent (listed with the other readings in the
design notes):
  * sector sketch: the rows of the dense sketch Omega (same generator, indexed
    by the global flat column index) that belong to the sector's columns, its
    first k_Q columns, k_Q = min(chi_c + oversample, rows_Q, cols_Q);
  * global truncation: each sector offers at most min(chi, rows_Q, cols_Q)
    triplets; chi_c = min(chi, sum_Q min(rows_Q, cols_Q)) triplets with the
    largest singular values are kept (ties: sector order, then index);
  * the kept vectors are ordered by sector (ascending charge), then by
    singular value, so the new bond is sector-contiguous;
  * the null test and the sign gauge are those of the dense zip-up, applied to
    the sector vectors embedded in the full row / column space;
  * the CBE fit (Fig. 3-5) runs sector by sector in the same way (see
    ``cbe_fit_u1``).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from .boundary import (NULL_TOL, RsvdParams, RowResult, bdim, close_last_row, first_row_boundary, gauge_signs,
                       orth, rsvd, theta, theta_r, theta_r_t, theta_t)
from .philox import gaussian_sketch


def bundle_charges(qk: np.ndarray, qw: np.ndarray, qb: np.ndarray) -> np.ndarray:
    """Charges of the flattened (ket, PEPO, bra) bundle, bra fastest: q_ket - q_pepo - q_bra."""
    return (qk[:, None, None, :] - qw[None, :, None, :] - qb[None, None, :, :]).reshape(-1, 2)


def site_bundles(qA, qW):
    """(Q_L, Q_U, Q_R, Q_Dn) of one sandwich site from the PEPS and PEPO leg charges."""
    return tuple(bundle_charges(qA[i], qW[i], qA[i]) for i in range(4))


def _sectors(rowq: np.ndarray, colq: np.ndarray):
    """Charges present among both the rows and the columns, ascending."""
    return sorted({tuple(x) for x in rowq.tolist()} & {tuple(x) for x in colq.tolist()})


def sector_rsvd(ap, ap_t, rowq, colq, chi: int, prm: RsvdParams, omega_of, cap_of=None):
    """rSVD of a block-diagonal matrix, sector by sector, with one global truncation.

    ap / ap_t apply the dense matrix and its transpose to column blocks;
    omega_of(k) returns the dense sketch (cols x k); cap_of(q, ri, ci) bounds the
    triplets a sector may offer (default min(chi, rows_Q, cols_Q)); the total kept is
    min(chi, sum of the caps). Returns (U, s, Vt, q, alive): the
    kept left vectors embedded in the row space (rows x chi_c), their singular
    values, the right vectors embedded in the column space (chi_c x cols), the
    sector charge of each kept triplet (chi_c x 2) and the null test of the dense
    zip-up (s^2 > NULL_TOL times the sum of s^2 over every sketched value).
    """
    rows, cols = len(rowq), len(colq)
    sec = []
    for qc in _sectors(rowq, colq):
        ri = np.flatnonzero(np.all(rowq == qc, axis=1))
        ci = np.flatnonzero(np.all(colq == qc, axis=1))
        rank = min(len(ri), len(ci))
        cap = min(chi, rank) if cap_of is None else max(0, min(chi, rank, cap_of(qc, ri, ci)))
        if cap == 0:
            continue
        k = rank if prm.exact_svd else min(cap + prm.oversample, rank)
        sec.append((qc, ri, ci, cap, k))
    if not sec:
        raise ValueError("no charge sector is shared by the rows and columns")
    omega = omega_of(max(s[4] for s in sec))
    parts = []
    for qc, ri, ci, cap, k in sec:
        out_r = np.ones(rows, dtype=bool)
        out_r[ri] = False
        out_c = np.ones(cols, dtype=bool)
        out_c[ci] = False

        def ap_s(X, ri=ri, ci=ci, out_r=out_r):
            full = np.zeros((cols, X.shape[1]))
            full[ci] = X
            Y = ap(full)
            if np.any(Y[out_r] != 0):
                raise AssertionError("matrix is not block diagonal in the given charges")
            return Y[ri]

        def ap_t_s(Y, ri=ri, ci=ci, out_c=out_c):
            full = np.zeros((rows, Y.shape[1]))
            full[ri] = Y
            Z = ap_t(full)
            if np.any(Z[out_c] != 0):
                raise AssertionError("matrix is not block diagonal in the given charges")
            return Z[ci]

        Q, ub, s, vt = rsvd(ap_s, ap_t_s, omega[ci, :k], prm.power_iters)
        parts.append((qc, ri, ci, cap, Q @ ub, s, vt))

    chi_c = min(chi, sum(p[3] for p in parts))
    cand = [(-s[j], n, j) for n, (_, _, _, cap, _, s, _) in enumerate(parts) for j in range(cap)]
    kept = sorted(sorted(cand)[:chi_c], key=lambda x: (x[1], x[2]))
    U = np.zeros((rows, chi_c))
    Vt = np.zeros((chi_c, cols))
    sv = np.zeros(chi_c)
    qk = np.zeros((chi_c, 2), dtype=np.int64)
    for m, (_, n, j) in enumerate(kept):
        qc, ri, ci, _, qu, s, vt = parts[n]
        U[ri, m] = qu[:, j]
        Vt[m, ci] = vt[j]
        sv[m] = s[j]
        qk[m] = qc
    tot = float(sum((p[5] ** 2).sum() for p in parts))
    alive = ((sv * sv > NULL_TOL * tot) & (tot > 0)).astype(np.float64)
    return U, sv, Vt, qk, alive


def sector_svd(M: np.ndarray, rowq, colq, keep_max: int):
    """Exact SVD of a block-diagonal matrix sector by sector, the keep_max largest
    triplets kept over all sectors (ordered by sector, then value). Returns
    (U, s, Wt, q, alive) embedded in the full row / column spaces."""
    rows, cols = M.shape
    parts = []
    allowed = np.zeros((rows, cols), dtype=bool)
    for qc in _sectors(rowq, colq):
        ri = np.flatnonzero(np.all(rowq == qc, axis=1))
        ci = np.flatnonzero(np.all(colq == qc, axis=1))
        allowed[np.ix_(ri, ci)] = True
        u, sv, wt = np.linalg.svd(M[np.ix_(ri, ci)], full_matrices=False)
        parts.append((qc, ri, ci, u, sv, wt))
    if np.any(M[~allowed] != 0):
        raise AssertionError("matrix is not block diagonal in the given charges")
    keep = min(keep_max, sum(len(p[4]) for p in parts))
    cand = [(-p[4][j], n, j) for n, p in enumerate(parts) for j in range(len(p[4]))]
    kept = sorted(sorted(cand)[:keep], key=lambda x: (x[1], x[2]))
    U = np.zeros((rows, keep))
    Wt = np.zeros((keep, cols))
    sv_k = np.zeros(keep)
    qk = np.zeros((keep, 2), dtype=np.int64)
    for m, (_, n, j) in enumerate(kept):
        qc, ri, ci, u, sv, wt = parts[n]
        U[ri, m] = u[:, j]
        Wt[m, ci] = wt[j]
        sv_k[m] = sv[j]
        qk[m] = qc
    tot = float(sum((p[4] ** 2).sum() for p in parts))
    alive = ((sv_k * sv_k > NULL_TOL * tot) & (tot > 0)).astype(np.float64)
    return U, sv_k, Wt, qk, alive


def zipup_u1(T, qT, Arow, Wrow, qrow, chi: int, prm: RsvdParams, *, seed: int, layer: int, row: int,
             env: int = 0):
    """Left-to-right zip-up with sector-wise rSVD (the block-sparse form of ``boundary.zipup``).

    qT[c]: charges of bond t_c (the last index of T[c]); qrow[c] = (Q_L, Q_U, Q_R, Q_Dn)
    of the row's sandwich site c. Returns (N, ELs, log_s, spectra, qN) with qN[c]
    the charges of the new bond a_c (qN[Ly-1] the trivial right edge).
    """
    Ly = len(T)
    EL = np.ones((1, 1, 1))
    qa = np.zeros((1, 2), dtype=np.int64)
    N, ELs, spectra, qN = [], [EL], [], []
    log_s = 0.0
    for c in range(Ly - 1):
        A, W = Arow[c], Wrow[c]
        a, tp = EL.shape[0], T[c].shape[2]
        dDn, dR = bdim(A, W, 3), bdim(A, W, 2)
        rows, cols = a * dDn, tp * dR
        _, _, QR, QD = qrow[c]
        rowq = (qa[:, None, :] - QD[None, :, :]).reshape(-1, 2)
        colq = (qT[c][:, None, :] + QR[None, :, :]).reshape(-1, 2)

        def ap(X, EL=EL, T=T[c], A=A, W=W, tp=tp, dR=dR, rows=rows):
            return theta(EL, T, A, W, X.reshape(tp, dR, -1)).reshape(rows, -1)

        def ap_t(Y, EL=EL, T=T[c], A=A, W=W, a=a, dDn=dDn, cols=cols):
            return theta_t(EL, T, A, W, Y.reshape(a, dDn, -1)).reshape(cols, -1)

        def omega_of(k, c=c, cols=cols):
            return gaussian_sketch(cols, k, seed=seed, layer=layer, stage=0, site=c, row=row, env=env)

        U, s, vt, qk, alive = sector_rsvd(ap, ap_t, rowq, colq, chi, prm, omega_of)
        chi_c = len(s)
        nc = U * alive[None, :]
        sg = gauge_signs(nc, 0, seed=seed, layer=layer, site=c, row=row, env=env)
        nc = nc * sg[None, :]
        el = (sg * s)[:, None] * vt
        nrm = np.linalg.norm(el)
        el /= nrm
        log_s += math.log(nrm)
        N.append(nc.reshape(a, dDn, chi_c))
        EL = el.reshape(chi_c, tp, dR)
        ELs.append(EL)
        spectra.append(s.copy())
        qN.append(qk)
        qa = qk
    c = Ly - 1
    y = theta(EL, T[c], Arow[c], Wrow[c], np.ones((1, 1, 1)))
    nrm = np.linalg.norm(y)
    N.append(y / nrm)
    log_s += math.log(nrm)
    qN.append(np.zeros((1, 2), dtype=np.int64))
    return N, ELs, log_s, spectra, qN


def cbe_fit_u1(T, qT, Arow, Wrow, qrow, N, qN, ELs, chi: int, prm: RsvdParams, *, seed: int, layer: int,
               row: int, env: int = 0):
    """Right-to-left CBE fit in the block-sparse mode (the form of ``boundary.cbe_fit``).

    Every matrix of the fit is block diagonal in the charge of the bond a_{c-1} it
    straddles: the rows of the centre tensor (their ordered Gram-Schmidt keeps
    sectors apart, the rows having disjoint supports), the CBE matrix
    A = P_L^perp Theta2s P_R^perp (sector-wise rSVD; a sector offers at most
    min(chi_tilde, rows_Q - n_Q(a_{c-1}), cols_Q - n_Q(V)) triplets and chi_tilde are
    kept over all sectors) and the fitted tensor M' (sector-wise SVD, chi kept over
    all sectors). Returns (new T, log_scale, spectra, bond charges).
    """
    Ly = len(T)
    chi_t = prm.chi_tilde if prm.chi_tilde > 0 else -(-chi // 10)
    M = N[Ly - 1]
    qright = np.zeros((1, 2), dtype=np.int64)      # charges of bond a_c (right of the centre)
    ER = np.ones((1, 1, 1))
    rs = 0.0
    rs_M = 0.0
    out = [None] * Ly
    qout = [None] * Ly
    qout[Ly - 1] = qright
    spectra = []
    zero = np.zeros((1, 2), dtype=np.int64)
    for c in range(Ly - 1, 0, -1):
        A, W = Arow[c], Wrow[c]
        Al, Wl = Arow[c - 1], Wrow[c - 1]
        a_prev, dDn, a_c = M.shape
        QD, QDl = qrow[c][3], qrow[c - 1][3]
        qa_prev = qN[c - 1]
        qa_left = qN[c - 2] if c >= 2 else zero
        colq = (QD[:, None, :] + qright[None, :, :]).reshape(-1, 2)          # (Dn_c, a_c)
        if a_prev >= dDn * a_c:
            V = np.eye(dDn * a_c)
            qV = colq
        else:
            V = orth(M.reshape(a_prev, dDn * a_c).T).T
            qV = qa_prev
        Nl = N[c - 1]
        Nlm = Nl.reshape(-1, Nl.shape[2])
        rows_a, cols_a = Nlm.shape[0], dDn * a_c
        rowq = (qa_left[:, None, :] - QDl[None, :, :]).reshape(-1, 2)        # (a_{c-2}, Dn_{c-1})
        ELl = ELs[c - 1]
        a2, dDnl = ELl.shape[0], bdim(Al, Wl, 3)

        def two_site(X, ER=ER):
            z = theta_r(ER, T[c], A, W, X.reshape(dDn, a_c, -1))
            return theta(ELl, T[c - 1], Al, Wl, z).reshape(rows_a, -1)

        def two_site_t(Y, ER=ER):
            z = theta_t(ELl, T[c - 1], Al, Wl, Y.reshape(a2, dDnl, -1))
            return theta_r_t(ER, T[c], A, W, z).reshape(cols_a, -1)

        def a_apply(X):
            y = two_site(X) - two_site(V.T @ (V @ X))
            return y - Nlm @ (Nlm.T @ y)

        def a_apply_t(Y):
            z = two_site_t(Y) - two_site_t(Nlm @ (Nlm.T @ Y))
            return z - V.T @ (V @ z)

        def cap_of(qc, ri, ci):
            n_a = int(np.all(qa_prev == qc, axis=1).sum())
            n_v = int(np.all(qV == qc, axis=1).sum())
            return min(chi_t, len(ri) - n_a, len(ci) - n_v)

        caps = [cap_of(qc, np.flatnonzero(np.all(rowq == qc, axis=1)), np.flatnonzero(np.all(colq == qc, axis=1)))
                for qc in _sectors(rowq, colq)]
        ct = min(chi_t, sum(max(0, x) for x in caps))
        if ct > 0:
            def omega_of(k, c=c):
                return gaussian_sketch(cols_a, k, seed=seed, layer=layer, stage=1, site=c, row=row, env=env)

            # as in the dense fit, the CBE sketch keeps its width chi_tilde + oversample
            # whatever exact_svd says (that setting governs the zip-up)
            cbe_prm = dataclasses.replace(prm, exact_svd=False)
            _, sa, vt, qt, alive = sector_rsvd(a_apply, a_apply_t, rowq, colq, ct, cbe_prm, omega_of, cap_of)
            vt = vt * alive[:, None]
            Vp = orth(np.hstack([V.T, vt.T])).T
            qVp = np.concatenate([qV, qt])
        else:
            Vp, qVp = V, qV
        ERp = theta_r(ER, T[c], A, W, Vp.T.reshape(dDn, a_c, -1))
        Mp = theta(ELl, T[c - 1], Al, Wl, ERp).reshape(a2 * dDnl, -1)
        u, s, wt, qk, alive = sector_svd(Mp, rowq, qVp, chi)
        wt = wt * alive[:, None]
        keep = len(s)
        nc = wt @ Vp
        sg = gauge_signs(nc, 1, seed=seed, layer=layer, site=c, row=row, env=env)
        nc = nc * sg[:, None]
        out[c] = nc.reshape(keep, dDn, a_c)
        M = ((u * s) * sg[None, :]).reshape(a2, dDnl, keep)
        er = (sg[:, None] * wt) @ ERp.reshape(-1, ERp.shape[2]).T
        nrm = np.linalg.norm(er)
        rs_M = rs
        rs += math.log(nrm)
        ER = (er / nrm).reshape(keep, ERp.shape[0], ERp.shape[1])
        spectra.append(s.copy())
        qright = qk
        qout[c - 1] = qk
    nrm = np.linalg.norm(M)
    out[0] = M / nrm
    spectra.reverse()
    return out, rs_M + math.log(nrm), spectra, qout


def first_row_charges(qrow):
    """Bond charges of the exact row-0 boundary: q_{t_c} = Q_R of site c (right edge trivial)."""
    return [qr for (_, _, qr, _) in qrow[:-1]] + [np.zeros((1, 2), dtype=np.int64)]


def contract_u1(peps, qpeps, pepo, qpepo, chi: int, prm: RsvdParams, *, seed: int, layer: int, env: int = 0,
                return_rows: bool = False):
    """<psi|O|psi> by boundary MPS with sector-wise compression: (sign, ln|value|[, rows]).

    qpeps[r][c] / qpepo[r][c]: (q_l, q_u, q_r, q_d) leg charges of the PEPS / PEPO site.
    """
    if prm.n_fit not in (0, 1):
        raise ValueError("n_fit must be 0 or 1")
    Lx, Ly = len(peps), len(peps[0])
    bundles = [[site_bundles(qpeps[r][c], qpepo[r][c]) for c in range(Ly)] for r in range(Lx)]
    rows = []
    if Lx == 1:
        T = [np.ones((1, 1, 1)) for _ in range(Ly)]
        sign, lv = close_last_row(T, peps[0], pepo[0])
        return (sign, lv, rows) if return_rows else (sign, lv)
    T, log_total = first_row_boundary(peps[0], pepo[0])
    qT = first_row_charges(bundles[0])
    for r in range(1, Lx - 1):
        N, ELs, log_s, zsp, qN = zipup_u1(T, qT, peps[r], pepo[r], bundles[r], chi, prm, seed=seed, layer=layer,
                                          row=r, env=env)
        if prm.n_fit == 1 and Ly > 1:
            N, log_s, fsp, qN = cbe_fit_u1(T, qT, peps[r], pepo[r], bundles[r], N, qN, ELs, chi, prm, seed=seed,
                                           layer=layer, row=r, env=env)
        else:
            fsp = []
        T, qT = N, qN
        log_total += log_s
        rows.append(RowResult(N, log_s, zsp, fsp))
    sign, lv = close_last_row(T, peps[Lx - 1], pepo[Lx - 1])
    log_total += lv
    return (sign, log_total, rows) if return_rows else (sign, log_total)


def expectation_u1(peps, qpeps, pepo, qpepo, chi: int, prm: RsvdParams, *, seed: int, env: int = 0):
    """<O> = <psi|O|psi> / <psi|psi>: operator sweep layer 1, norm sweep layer 0 (identity PEPO)."""
    from synth.lattice import identity_pepo  # data only
    Lx, Ly = len(peps), len(peps[0])
    p = peps[0][0].shape[4]
    zero = np.zeros((1, 2), dtype=np.int64)
    qid = [[(zero, zero, zero, zero) for _ in range(Ly)] for _ in range(Lx)]
    sn, ln = contract_u1(peps, qpeps, pepo, qpepo, chi, prm, seed=seed, layer=1, env=env)
    sd, ld = contract_u1(peps, qpeps, identity_pepo(Lx, Ly, p), qid, chi, prm, seed=seed, layer=0, env=env)
    return sn * sd * math.exp(ln - ld), (sn, ln), (sd, ld)
