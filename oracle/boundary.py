"""Boundary-MPS environment approximation with rSVD compression (oracle; test infrastructure).

Plain FP64 NumPy restatement of the row absorption the GPU path performs:

* Sec. II: rows of PEPS-PEPO-PEPS sandwiches are absorbed one by one into a
  boundary MPS whose bundles of D*w*D are compressed to a bond chi.
* Sec. IV: each compression uses a randomized SVD (Gaussian sketch Omega,
  repeated application of the matrix and its transpose, thin QR, small SVD of
  the projected matrix; Halko et al. 2011, Example 1.6), first in a left-to-
  right zip-up pass and then in a right-to-left variational fit whose bond is
  widened by controlled bond expansion (CBE, Fig. 3) before it is truncated
  back to chi. The CBE matrix A = P_L^perp Theta2s P_R^perp is applied to Omega
  without forming the orthogonal projectors: each projector is split into the
  identity minus the tangent projector and the two resulting clusters are
  contracted separately and subtracted (Fig. 5 (b)-(g)).

Conventions (all real FP64):
  T[c]  boundary tensor [t_{c-1}, U_c, t_c]          (previous environment)
  EL[c] left environment [a_{c-1}, t_{c-1}, L_c]   (new boundary x old row)
  ER[c] right environment [a_{c-1}, t_{c-1}, L_c]  (same index roles, from the right)
  N[c]  new boundary tensor [a_{c-1}, Dn_c, a_c]
Bundles (L, U, R, Dn) are flattened (ket, PEPO, bra) legs, bra fastest.

Readings where the paper is silent (each is listed with its reason in the
design notes): kept bond chi_c = min(chi, rows, cols) of the matrix factorised;
sketch width chi_c + oversampling; q power iterations with re-orthonormalisation
after every application; CBE width ceil(chi/10), clipped to the dimensions of
the complement; singular-vector signs fixed so that every kept vector x has
sum_i w_i x_i >= 0 for fixed Gaussian weights w drawn by the sketch generator
(``gauge_signs``); per-site Frobenius normalisation with the logarithms
accumulated.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .network import sandwich_apply
from .philox import gaussian_sketch


@dataclass
class RsvdParams:
    """rSVD settings (Sec. IV). Defaults follow the 4x4 and larger configurations."""
    oversample: int = 10
    power_iters: int = 2
    chi_tilde: int = 0          # 0 => ceil(chi / 10)
    n_fit: int = 1              # right-to-left CBE fit passes (0: zip-up only)
    exact_svd: bool = False     # sketch width = full rank (exact factorisation)


@dataclass
class RowResult:
    T: list                     # new boundary tensors
    log_scale: float            # ln of the scale factor taken out of the tensors
    zip_spectra: list = field(default_factory=list)
    fit_spectra: list = field(default_factory=list)


def bdim(A: np.ndarray, W: np.ndarray, leg: int) -> int:
    """Dimension of the (ket, PEPO, bra) bundle of leg 0..3 = l, u, r, d."""
    return A.shape[leg] * W.shape[leg] * A.shape[leg]


# ---------------------------------------------------------------------------
# the four matrix applications used by the compression (pattern of Fig. 2(a))
# ---------------------------------------------------------------------------

# The four maps are linear in their k input vectors (last axis); they are applied to at most
# COLS vectors at a time, which bounds the size of the intermediates (at 6x6, D=6, chi=256 a
# full-width intermediate would hold ~11 GB) without changing any vector's arithmetic.
COLS = 16


def _by_columns(fn):
    def wrapped(E, T, A, W, X):
        k = X.shape[-1]
        if k <= COLS:
            return fn(E, T, A, W, X)
        parts = [fn(E, T, A, W, X[..., j:j + COLS]) for j in range(0, k, COLS)]
        return np.concatenate(parts, axis=-1)
    wrapped.__doc__ = fn.__doc__
    wrapped.__name__ = fn.__name__
    return wrapped


@_by_columns
def theta(EL, T, A, W, X):
    """Theta_c X: X[t', R, k] -> [a, Dn, k];  Theta = EL . T . C (left environment side)."""
    G1 = np.einsum("tUs,sRk->tURk", T, X, optimize=True)
    G2 = sandwich_apply(G1, A, W, ins=("u", "r"), outs=("l", "d"))   # [t, L, Dn, k]
    return np.einsum("atL,tLDk->aDk", EL, G2, optimize=True)


@_by_columns
def theta_t(EL, T, A, W, Y):
    """Theta_c^T Y: Y[a, Dn, k] -> [t', R, k]."""
    H1 = np.einsum("atL,aDk->tLDk", EL, Y, optimize=True)
    H2 = sandwich_apply(H1, A, W, ins=("l", "d"), outs=("u", "r"))   # [t, U, R, k]
    return np.einsum("tUs,tURk->sRk", T, H2, optimize=True)


@_by_columns
def theta_r(ER, T, A, W, X):
    """Right-environment map: X[Dn, a, k] -> [t, L, k];  ER[a, t', R] is the environment to the right."""
    W1 = np.einsum("asR,Dak->sRDk", ER, X, optimize=True)
    W2 = sandwich_apply(W1, A, W, ins=("r", "d"), outs=("l", "u"))   # [t', L, U, k]
    return np.einsum("tUs,sLUk->tLk", T, W2, optimize=True)


@_by_columns
def theta_r_t(ER, T, A, W, Z):
    """Transpose of theta_r: Z[t, L, k] -> [Dn, a, k]."""
    W1 = np.einsum("tUs,tLk->sLUk", T, Z, optimize=True)
    W2 = sandwich_apply(W1, A, W, ins=("l", "u"), outs=("r", "d"))   # [t', R, Dn, k]
    return np.einsum("asR,sRDk->Dak", ER, W2, optimize=True)


def form_theta(EL, T, A, W) -> np.ndarray:
    """Explicit (a*Dn) x (t'*R) matrix Theta_c (small sizes only)."""
    tp, dR = T.shape[2], bdim(A, W, 2)
    n = tp * dR
    return theta(EL, T, A, W, np.eye(n).reshape(tp, dR, n)).reshape(-1, n)


# ---------------------------------------------------------------------------
# linear algebra steps (Sec. IV; Halko et al. Example 1.6)
# ---------------------------------------------------------------------------

# A column whose squared residual, after projecting out the columns before it,
# is at most DEP_TOL times the largest squared column norm is numerically
# dependent on them (an FP64 Gram matrix cannot resolve it) and gives a zero column.
DEP_TOL = 1e-13


def orth(Y: np.ndarray) -> np.ndarray:
    """Thin QR factor of Y (Sec. IV): columns orthonormalised in their order, so
    that span(Q[:, :j]) = span(Y[:, :j]) and each column's coefficient on its own
    direction is positive (diag(R) > 0, as LAPACK's QR with the sign fixed).

    When Y is rank deficient, a column that depends numerically on the ones
    before it (squared residual <= DEP_TOL * max squared column norm) becomes a
    zero column instead of an arbitrary completion direction, so the non-zero
    columns span exactly range(Y). Classical Gram-Schmidt, applied twice.
    """
    m, k = Y.shape
    if m < k:
        raise ValueError("orth: thin QR needs at least as many rows as columns")
    Q = np.zeros((m, k))
    if k == 0:
        return Q
    cap = DEP_TOL * float((Y * Y).sum(axis=0).max())
    for j in range(k):
        v = Y[:, j].astype(np.float64)
        v = v - Q[:, :j] @ (Q[:, :j].T @ v)
        r2 = float(v @ v)
        if not r2 > cap:
            continue
        v = v - Q[:, :j] @ (Q[:, :j].T @ v)
        Q[:, j] = v / np.sqrt(v @ v)
    return Q


# Singular vectors of a numerically zero singular value (sigma^2 <= NULL_TOL times
# the sum of all sigma^2) are not determined by the matrix; they are taken as zero,
# so that they add no bond direction.
NULL_TOL = 1e-30


def live(s: np.ndarray) -> np.ndarray:
    """1.0 for singular values above the null level, 0.0 for the rest."""
    tot = float((s * s).sum())
    return ((s * s > NULL_TOL * tot) & (tot > 0)).astype(np.float64)


def rsvd(apply, apply_t, omega: np.ndarray, q: int):
    """Randomized subspace iteration and the SVD of the projected matrix.

    Y = A Omega; Q = orth(Y); q times {Q' = orth(A^T Q); Q = orth(A Q')};
    B = Q^T A (formed as (A^T Q)^T); B = Ub S Vt.  Returns (Q, Ub, S, Vt).
    """
    Q = orth(apply(omega))
    for _ in range(q):
        Qz = orth(apply_t(Q))
        Q = orth(apply(Qz))
    bt = apply_t(Q)
    ub, s, vt = np.linalg.svd(bt.T, full_matrices=False)
    return Q, ub, s, vt


GAUGE_STAGE = 2   # sketch stage word of the gauge weights (0: zip-up, 1: CBE)


def gauge_signs(x: np.ndarray, axis: int, *, seed: int, layer: int, site: int, row: int,
                env: int = 0) -> np.ndarray:
    """Sign gauge of kept singular vectors: +1 where sum_i w_i x_i >= 0 along ``axis``,
    else -1, with fixed Gaussian weights w (the sketch generator, stage GAUGE_STAGE,
    one column over the C-order flat index). A plain entry sum can vanish exactly
    for symmetric vectors and leave the sign to rounding; generic weights cannot."""
    w = gaussian_sketch(x.shape[axis], 1, seed=seed, layer=layer, stage=GAUGE_STAGE, site=site, row=row,
                        env=env)[:, 0]
    t = np.tensordot(w, x, axes=([0], [axis]))
    return np.where(t < 0, -1.0, 1.0)


# ---------------------------------------------------------------------------
# row 0, zip-up, CBE fit, last row
# ---------------------------------------------------------------------------

def first_row_boundary(Arow, Wrow):
    """Exact boundary from row 0: T_c[L, Dn, R] = row-0 sandwich with the dimension-1 up legs dropped.

    Each tensor is scaled to unit norm; returns (T, log_scale).
    """
    T, log_s = [], 0.0
    for A, W in zip(Arow, Wrow):
        c = np.einsum("lurdp,LURDpq,wxyzq->lLwuUxrRydDz", A, W, A)
        dl, dr, dd = bdim(A, W, 0), bdim(A, W, 2), bdim(A, W, 3)
        c = c.reshape(dl, 1, dr, dd)[:, 0]            # [L, R, Dn]
        t = np.ascontiguousarray(np.transpose(c, (0, 2, 1)))   # [L, Dn, R]
        nrm = np.linalg.norm(t)
        T.append(t / nrm)
        log_s += math.log(nrm)
    return T, log_s


def zipup(T, Arow, Wrow, chi: int, prm: RsvdParams, *, seed: int, layer: int, row: int, env: int = 0):
    """Left-to-right zip-up of (row sandwiches) x (boundary T) with rSVD truncation to chi.

    Returns (N, EL, log_s, spectra): N[c] left-isometric for c < Ly-1, N[Ly-1]
    the unit-norm last tensor, EL[c] the normalised left environments.
    """
    Ly = len(T)
    EL = np.ones((1, 1, 1))
    N, ELs, spectra = [], [EL], []
    log_s = 0.0
    for c in range(Ly - 1):
        A, W = Arow[c], Wrow[c]
        a, tp = EL.shape[0], T[c].shape[2]
        dDn, dR = bdim(A, W, 3), bdim(A, W, 2)
        rows, cols = a * dDn, tp * dR
        chi_c = min(chi, rows, cols)
        k = min(rows, cols) if prm.exact_svd else min(chi_c + prm.oversample, rows, cols)
        omega = gaussian_sketch(cols, k, seed=seed, layer=layer, stage=0, site=c, row=row, env=env)

        def ap(X, EL=EL, T=T[c], A=A, W=W, tp=tp, dR=dR):
            return theta(EL, T, A, W, X.reshape(tp, dR, -1)).reshape(rows, -1)

        def ap_t(Y, EL=EL, T=T[c], A=A, W=W, a=a, dDn=dDn):
            return theta_t(EL, T, A, W, Y.reshape(a, dDn, -1)).reshape(cols, -1)

        Q, ub, s, vt = rsvd(ap, ap_t, omega, prm.power_iters)
        nc = Q @ (ub[:, :chi_c] * live(s)[None, :chi_c])
        sg = gauge_signs(nc, 0, seed=seed, layer=layer, site=c, row=row, env=env)
        nc = nc * sg[None, :]
        el = (sg * s[:chi_c])[:, None] * vt[:chi_c]
        nrm = np.linalg.norm(el)
        el /= nrm
        log_s += math.log(nrm)
        N.append(nc.reshape(a, dDn, chi_c))
        EL = el.reshape(chi_c, tp, dR)
        ELs.append(EL)
        spectra.append(s[:chi_c].copy())
    # last site: Theta has a single column
    c = Ly - 1
    y = theta(EL, T[c], Arow[c], Wrow[c], np.ones((1, 1, 1)))
    nrm = np.linalg.norm(y)
    N.append(y / nrm)
    log_s += math.log(nrm)
    return N, ELs, log_s, spectra


def cbe_operator(two_site, two_site_t, V, Nlm):
    """The CBE matrix A = P_L^perp Theta2s P_R^perp and its transpose as maps (Fig. 5).

    V (rows orthonormal) spans the row space of the centre tensor, so
    P_R^perp = I - V^T V; Nlm (columns orthonormal) is the left isometry of the
    zip-up at the left site, so P_L^perp = I - Nlm Nlm^T. Neither projector is
    formed: the right one is split into the identity minus the tangent
    projector and the two clusters Theta2s(X) and Theta2s(V^T V X) are
    contracted separately and subtracted (Fig. 5(b)-(e)); the left one is then
    applied to the result (Fig. 5(f)-(g)). The transpose runs the mirror image.
    """

    def a_apply(X):
        y = two_site(X) - two_site(V.T @ (V @ X))
        return y - Nlm @ (Nlm.T @ y)

    def a_apply_t(Y):
        z = two_site_t(Y) - two_site_t(Nlm @ (Nlm.T @ Y))
        return z - V.T @ (V @ z)

    return a_apply, a_apply_t


def cbe_width(chi_t: int, rows_a: int, n_left: int, cols_a: int, n_right: int) -> int:
    """Number of expansion vectors: chi_tilde, clipped to the dimensions of the
    complement (rows outside the left isometry's n_left columns, columns outside
    the n_right rows of V), which bound the rank of A."""
    return min(chi_t, rows_a - n_left, cols_a - n_right)


def cbe_fit(T, Arow, Wrow, N, ELs, chi: int, prm: RsvdParams, *, seed: int, layer: int, row: int,
            env: int = 0, trace: list | None = None, stage: int = 1):
    """Right-to-left variational fit with controlled bond expansion (Fig. 3-5).

    At each bond (c-1, c): V = row basis of the centre tensor at c; the
    truncated complement Vtil (top singular vectors of A = P_L^perp Theta2s
    P_R^perp, by rSVD) widens V to V' = [V; Vtil]; the expanded right
    environment and the fitted tensor M' at c-1 follow pattern 2(a); the SVD of
    M' truncates the bond back. Returns (new T, log_scale, spectra).

    ``trace`` (test hook, no effect on the result): if a list is given, one dict
    per bond is appended with the inputs and outputs of the expansion step.
    ``stage``: generator stage of the CBE sketch (pass p of the fit uses 1 + 16 (p - 1)).
    """
    Ly = len(T)
    chi_t = prm.chi_tilde if prm.chi_tilde > 0 else -(-chi // 10)
    M = N[Ly - 1]
    ER = np.ones((1, 1, 1))
    rs = 0.0
    rs_M = 0.0
    out = [None] * Ly
    spectra = []
    for c in range(Ly - 1, 0, -1):
        A, W = Arow[c], Wrow[c]
        Al, Wl = Arow[c - 1], Wrow[c - 1]
        a_prev, dDn, a_c = M.shape
        if a_prev >= dDn * a_c:
            # at least as many rows as columns: the row space is the whole (Dn a_c) space
            V = np.eye(dDn * a_c)
        else:
            V = orth(M.reshape(a_prev, dDn * a_c).T).T              # a_prev x (Dn a_c), orthonormal rows
        a_eff = V.shape[0]
        Nl = N[c - 1]
        Nlm = Nl.reshape(-1, Nl.shape[2])                           # (a_{c-2} Dn_{c-1}) x a_{c-1}
        rows_a, cols_a = Nlm.shape[0], dDn * a_c
        ct = cbe_width(chi_t, rows_a, Nlm.shape[1], cols_a, a_eff)
        ELl = ELs[c - 1]
        a2, dDnl = ELl.shape[0], bdim(Al, Wl, 3)

        def two_site(X, ER=ER):
            z = theta_r(ER, T[c], A, W, X.reshape(dDn, a_c, -1))      # [t_{c-1}, L_c, k]
            return theta(ELl, T[c - 1], Al, Wl, z).reshape(rows_a, -1)

        def two_site_t(Y, ER=ER):
            z = theta_t(ELl, T[c - 1], Al, Wl, Y.reshape(a2, dDnl, -1))
            return theta_r_t(ER, T[c], A, W, z).reshape(cols_a, -1)

        a_apply, a_apply_t = cbe_operator(two_site, two_site_t, V, Nlm)

        sa, vtil, k = np.zeros(0), np.zeros((0, cols_a)), 0
        if ct > 0:
            k = min(ct + prm.oversample, rows_a, cols_a)
            omega = gaussian_sketch(cols_a, k, seed=seed, layer=layer, stage=stage, site=c, row=row, env=env)
            _, _, sa, vt = rsvd(a_apply, a_apply_t, omega, prm.power_iters)
            vtil = (vt * live(sa)[:, None])[:ct]
            # the kept singular vectors lie in range(P_R^perp) unless A is (numerically)
            # rank deficient, when null-space vectors are arbitrary: a thin QR of
            # [V^T, Vtil^T] keeps V and makes the added rows orthogonal to it
            Vp = orth(np.hstack([V.T, vtil.T])).T
        else:
            Vp = V
        ERp = theta_r(ER, T[c], A, W, Vp.T.reshape(dDn, a_c, -1))   # [t_{c-1}, L_c, j]
        Mp = theta(ELl, T[c - 1], Al, Wl, ERp)                      # [a_{c-2}, Dn_{c-1}, j]
        u, s, wt = np.linalg.svd(Mp.reshape(a2 * dDnl, -1), full_matrices=False)
        wt = wt * live(s)[:, None]
        keep = min(chi, a2 * dDnl, Vp.shape[0])
        nc = wt[:keep] @ Vp
        sg = gauge_signs(nc, 1, seed=seed, layer=layer, site=c, row=row, env=env)
        nc = nc * sg[:, None]
        out[c] = nc.reshape(keep, dDn, a_c)
        M = ((u[:, :keep] * s[:keep]) * sg[None, :]).reshape(a2, dDnl, keep)
        er = (sg[:, None] * wt[:keep]) @ ERp.reshape(-1, ERp.shape[2]).T    # keep x (t L)
        if trace is not None:
            trace.append(dict(c=c, V=V, Nlm=Nlm, ct=ct, k=k, sigma_a=sa, Vtil=vtil, Vp=Vp, ER=ER, EL=ELl,
                              rows_a=rows_a, cols_a=cols_a, spectrum=s[:keep].copy()))
        nrm = np.linalg.norm(er)
        rs_M = rs
        rs += math.log(nrm)
        ER = (er / nrm).reshape(keep, ERp.shape[0], ERp.shape[1])
        spectra.append(s[:keep].copy())
    nrm = np.linalg.norm(M)
    out[0] = M / nrm
    spectra.reverse()
    return out, rs_M + math.log(nrm), spectra


def fit_stage(p: int) -> int:
    """Generator stage of the CBE sketch of fit pass p = 1, 2, ... (stage 0 is the zip-up's
    sketch, stage 2 the sign gauge's weights)."""
    return 1 + 16 * (p - 1)


def recanonicalize(T, Arow, Wrow, F):
    """Left-to-right gauge sweep of a fitted boundary before another right-to-left
    fit pass (Sec. IV: the fit of a bond needs the sites to its left in left-canonical
    form, and the fit pass leaves them right-canonical).

    F[0] is the unit-norm first tensor and F[c > 0] right isometries [a_{c-1}, Dn, a_c].
    Each site, with the triangular factor of the site before it multiplied in, is
    split by a thin QR; Q is the new left isometry and the factor moves right. The
    left environment of the next site is the product of the rows above with the new
    isometry, EL_{c+1} = (Theta_c^T N_c)^T (the same pattern 2(a) as the zip-up's
    remainder), normalised by its Frobenius norm (the fit takes its scale from the
    first site, whose environment is exactly 1). Returns (N, ELs) in the form the
    zip-up returns them: N[c] left isometries for c < Ly-1, N[Ly-1] the unit-norm
    last tensor, ELs[c] the left environment of site c.
    """
    Ly = len(F)
    R = np.ones((1, 1))
    EL = np.ones((1, 1, 1))
    N, ELs = [], [EL]
    for c in range(Ly - 1):
        X = np.einsum("ab,bDc->aDc", R, F[c])
        a1, dDn, ac = X.shape
        Xm = X.reshape(a1 * dDn, ac)
        Q = orth(Xm)
        R = Q.T @ Xm                                      # X = Q R (Q spans the range of X)
        Nc = Q.reshape(a1, dDn, ac)
        N.append(Nc)
        z = theta_t(EL, T[c], Arow[c], Wrow[c], Nc)       # [t', R, a_c]
        el = np.moveaxis(z, -1, 0)
        EL = el / np.linalg.norm(el)
        ELs.append(EL)
    X = np.einsum("ab,bDc->aDc", R, F[Ly - 1])
    N.append(X / np.linalg.norm(X))
    return N, ELs


def absorb_row(T, Arow, Wrow, chi: int, prm: RsvdParams, *, seed: int, layer: int, row: int,
               env: int = 0) -> RowResult:
    """One interior row: zip-up rSVD compression, then n_fit CBE fit passes (each pass
    after the first starts from the previous one, re-canonicalised left to right)."""
    N, ELs, log_s, zsp = zipup(T, Arow, Wrow, chi, prm, seed=seed, layer=layer, row=row, env=env)
    if prm.n_fit == 0 or len(T) == 1:
        return RowResult(N, log_s, zsp, [])
    newT, log_f, fsp = cbe_fit(T, Arow, Wrow, N, ELs, chi, prm, seed=seed, layer=layer, row=row, env=env)
    for p in range(2, prm.n_fit + 1):
        N, ELs = recanonicalize(T, Arow, Wrow, newT)
        newT, log_f, fsp = cbe_fit(T, Arow, Wrow, N, ELs, chi, prm, seed=seed, layer=layer, row=row, env=env,
                                   stage=fit_stage(p))
    return RowResult(newT, log_f, zsp, fsp)


def close_last_row(T, Arow, Wrow):
    """Exact contraction of the last row against the boundary: (sign, ln|value|)."""
    v = np.ones((1, 1, 1))
    log_s = 0.0
    Ly = len(T)
    for c in range(Ly):
        z = theta_t(v, T[c], Arow[c], Wrow[c], np.ones((1, 1, 1)))   # [t', R, 1]
        if c < Ly - 1:
            nrm = np.linalg.norm(z)
            log_s += math.log(nrm)
            v = (z / nrm).reshape(1, z.shape[0], z.shape[1])
        else:
            val = float(z.reshape(-1)[0])
    sign = 1 if val >= 0 else -1
    return sign, (log_s + math.log(abs(val))) if val != 0 else -math.inf


def contract(peps, pepo, chi: int, prm: RsvdParams, *, seed: int, layer: int, env: int = 0,
             return_rows: bool = False):
    """<psi|O|psi> by boundary MPS: (sign, ln|value|[, per-row results])."""
    Lx, Ly = len(peps), len(peps[0])
    rows = []
    if Lx == 1:
        T = [np.ones((1, 1, 1)) for _ in range(Ly)]
        sign, lv = close_last_row(T, peps[0], pepo[0])
        return (sign, lv, rows) if return_rows else (sign, lv)
    T, log_total = first_row_boundary(peps[0], pepo[0])
    for r in range(1, Lx - 1):
        res = absorb_row(T, peps[r], pepo[r], chi, prm, seed=seed, layer=layer, row=r, env=env)
        T = res.T
        log_total += res.log_scale
        rows.append(res)
    sign, lv = close_last_row(T, peps[Lx - 1], pepo[Lx - 1])
    log_total += lv
    return (sign, log_total, rows) if return_rows else (sign, log_total)


def expectation(peps, pepo, chi: int, prm: RsvdParams, *, seed: int, env: int = 0):
    """<O> = <psi|O|psi> / <psi|psi>: operator sweep uses layer 1, norm sweep layer 0."""
    from synth.lattice import identity_pepo  # data only
    p = peps[0][0].shape[4]
    sn, ln = contract(peps, pepo, chi, prm, seed=seed, layer=1, env=env)
    sd, ld = contract(peps, identity_pepo(len(peps), len(peps[0]), p), chi, prm, seed=seed, layer=0, env=env)
    return sn * sd * math.exp(ln - ld), (sn, ln), (sd, ld)
