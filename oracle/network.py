"""PEPS-PEPO-PEPS network pieces in plain FP64 NumPy (oracle side; test infrastructure).

* ``sandwich_apply`` - contract one block of vectors through the sandwich C of a
  site (paper Sec. II, Fig. 1: ket A, PEPO W, bra A; Sec. III: C is the
  sandwich of a PEPS, a PEPO and an adjoint PEPS tensor). Real data, so the
  adjoint PEPS is A itself.
* ``psi_vector`` / ``brute_force_expectation`` - exact state vector of a small
  lattice and <psi|O|psi> from it (pin (a)).
* ``apply_terms`` - H|psi> applied term by term from a Hamiltonian's term list,
  independent of any PEPO tensor (pins the finite-state-machine PEPO).
* ``exact_columnwise`` - exact contraction of <psi|O|psi> column by column
  (the transposed order of the row-wise boundary method), no truncation.
"""
from __future__ import annotations

import numpy as np

# einsum letters: ket legs, PEPO legs, bra legs
_KET = {"l": "l", "u": "u", "r": "r", "d": "d"}
_PEPO = {"l": "L", "u": "U", "r": "R", "d": "D"}
_BRA = {"l": "w", "u": "x", "r": "y", "d": "z"}


def bundle(leg: str) -> str:
    """einsum letters of the (ket, PEPO, bra) bundle on one side of a site, bra fastest."""
    return _KET[leg] + _PEPO[leg] + _BRA[leg]


def sandwich_apply(G: np.ndarray, A: np.ndarray, W: np.ndarray, ins, outs) -> np.ndarray:
    """Contract the sandwich C = A (x) W (x) A of one site with a block G.

    G has shape [t, X, Y, k] where X, Y are the flattened (ket, PEPO, bra)
    bundles of legs ``ins = (x, y)`` (each one of 'l','u','r','d').
    Returns [t, V, Z, k] with V, Z the bundles of legs ``outs = (v, z)``:

      out[t, V, Z, k] = sum_{X, Y} G[t, X, Y, k] C[..X..Y..V..Z..]

    where C[(l,lw,l'),(u,uw,u'),(r,rw,r'),(d,dw,d')]
          = sum_{p,p'} A[l,u,r,d,p] W[lw,uw,rw,dw,p,p'] A[l',u',r',d',p'].
    """
    x, y = ins
    v, z = outs
    li = {"l": 0, "u": 1, "r": 2, "d": 3}
    perm = [li[x], li[y], li[v], li[z]]
    Ar = A.transpose(perm + [4])            # ket / bra roles [x, y, v, z, p]
    Wr = W.transpose(perm + [4, 5])         # PEPO roles [xw, yw, vw, zw, p, p']
    nx, ny, nv, nz, p = Ar.shape
    nxw, nyw, nvw, nzw = Wr.shape[:4]
    t, gx, gy, k = G.shape
    assert gx == nx * nxw * nx and gy == ny * nyw * ny, (G.shape, Ar.shape, Wr.shape)
    # layer by layer, PEPO indices kept separate (Sec. III): ket, then PEPO, then bra.
    # ket: sum over (x, y)
    g = G.reshape(t, nx, nxw, nx, ny, nyw, ny, k).transpose(0, 2, 3, 5, 6, 7, 1, 4)
    g = g.reshape(-1, nx * ny) @ Ar.reshape(nx * ny, nv * nz * p)          # [t,xw,x',yw,y',k,v,z,p]
    # PEPO: sum over (xw, yw, p)
    g = g.reshape(t, nxw, nx, nyw, ny, k, nv, nz, p).transpose(0, 2, 4, 5, 6, 7, 1, 3, 8)
    wm = Wr.transpose(0, 1, 4, 2, 3, 5).reshape(nxw * nyw * p, nvw * nzw * p)
    g = g.reshape(-1, nxw * nyw * p) @ wm                                    # [t,x',y',k,v,z,vw,zw,p']
    # bra: sum over (x', y', p')
    g = g.reshape(t, nx, ny, k, nv, nz, nvw, nzw, p).transpose(0, 3, 4, 5, 6, 7, 1, 2, 8)
    bm = Ar.transpose(0, 1, 4, 2, 3).reshape(nx * ny * p, nv * nz)
    g = g.reshape(-1, nx * ny * p) @ bm                                      # [t,k,v,z,vw,zw,v',z']
    g = g.reshape(t, k, nv, nz, nvw, nzw, nv, nz).transpose(0, 2, 4, 6, 3, 5, 7, 1)
    return np.ascontiguousarray(g).reshape(t, nv * nvw * nv, nz * nzw * nz, k)


def sandwich_full(A: np.ndarray, W: np.ndarray) -> np.ndarray:
    """Explicit sandwich tensor C[L, U, R, Dn] (bundles flattened) for small sites."""
    c = np.einsum("lurdp,LURDpq,wxyzq->lLwuUxrRydDz", A, W, A)
    dl, du, dr, dd = (A.shape[i] * W.shape[i] * A.shape[i] for i in range(4))
    return c.reshape(dl, du, dr, dd)


# ---------------------------------------------------------------------------
# brute force on small lattices
# ---------------------------------------------------------------------------

def psi_vector(grid) -> np.ndarray:
    """Exact state vector psi(s_00, s_01, ..., s_{Lx-1,Ly-1}) (row-major sites).

    One einsum over the whole grid of site tensors [l, u, r, d, p]; every bond
    gets its own letter, open-boundary legs (dimension 1) are summed trivially.
    """
    import string
    Lx, Ly = len(grid), len(grid[0])
    pool = iter(string.ascii_letters)
    hb = [[next(pool) for _ in range(Ly + 1)] for _ in range(Lx)]     # hb[r][c]: left leg of column c
    vb = [[next(pool) for _ in range(Ly)] for _ in range(Lx + 1)]     # vb[r][c]: up leg of row r
    ph = [[next(pool) for _ in range(Ly)] for _ in range(Lx)]
    terms = []
    for r in range(Lx):
        for c in range(Ly):
            terms.append(hb[r][c] + vb[r][c] + hb[r][c + 1] + vb[r + 1][c] + ph[r][c])
    out = "".join(ph[r][c] for r in range(Lx) for c in range(Ly))
    # absorb sites one at a time in row-major order; a bond letter shared by the
    # running tensor and the next site is summed, every other letter stays open
    acc, acc_l = grid[0][0], terms[0]
    for idx in range(1, Lx * Ly):
        t, tl = grid[idx // Ly][idx % Ly], terms[idx]
        keep = "".join(ch for ch in acc_l + tl if (ch in acc_l) != (ch in tl))
        acc = np.einsum(f"{acc_l},{tl}->{keep}", acc, t)
        acc_l = keep
    # remaining open letters: the physical legs and the dimension-1 boundary legs
    acc = np.einsum(f"{acc_l}->{out}", acc)
    return acc.reshape(-1)


def pepo_times_peps(peps, pepo):
    """Site-wise product (W psi): tensors [(l,lw),(u,uw),(r,rw),(d,dw), p'] of bond D*w."""
    out = []
    for arow, wrow in zip(peps, pepo):
        row = []
        for a, w in zip(arow, wrow):
            t = np.einsum("lurdp,LURDpq->lLuUrRdDq", a, w)
            s = t.shape
            row.append(t.reshape(s[0] * s[1], s[2] * s[3], s[4] * s[5], s[6] * s[7], s[8]))
        out.append(row)
    return out


def brute_force_expectation(peps, pepo):
    """(<psi|O|psi>, <psi|psi>) from the exact vectors psi and O psi (O as a PEPO)."""
    psi = psi_vector(peps)
    opsi = psi_vector(pepo_times_peps(peps, pepo))
    return float(psi @ opsi), float(psi @ psi)


def apply_terms(psi: np.ndarray, ham) -> np.ndarray:
    """H psi for H = sum_i h_i + sum_<ij> sum_k t^k_ij X^k_i Y^k_j, term by term."""
    Lx, Ly, p = ham.Lx, ham.Ly, ham.p
    n = Lx * Ly
    v = psi.reshape((p,) * n)
    out = np.zeros_like(v)

    def site(r, c):
        return r * Ly + c

    def apply1(x, op, s):
        return np.moveaxis(np.tensordot(op, x, axes=([1], [s])), 0, s)

    for r in range(Lx):
        for c in range(Ly):
            out += apply1(v, ham.onsite[r][c], site(r, c))
    for k in range(ham.K):
        for r in range(Lx):
            for c in range(Ly):
                if c + 1 < Ly:
                    out += ham.t_h[k, r, c] * apply1(apply1(v, ham.Y[k], site(r, c + 1)), ham.X[k], site(r, c))
                if r + 1 < Lx:
                    out += ham.t_v[k, r, c] * apply1(apply1(v, ham.Y[k], site(r + 1, c)), ham.X[k], site(r, c))
    return out.reshape(-1)


def product_state_energy(vecs, ham) -> float:
    """Closed form <psi|H|psi> for a normalised product state psi = (x) v_i."""
    Lx, Ly = ham.Lx, ham.Ly
    e = sum(vecs[r][c] @ ham.onsite[r][c] @ vecs[r][c] for r in range(Lx) for c in range(Ly))
    for k in range(ham.K):
        for r in range(Lx):
            for c in range(Ly):
                xv = vecs[r][c] @ ham.X[k] @ vecs[r][c]
                if c + 1 < Ly:
                    e += ham.t_h[k, r, c] * xv * (vecs[r][c + 1] @ ham.Y[k] @ vecs[r][c + 1])
                if r + 1 < Lx:
                    e += ham.t_v[k, r, c] * xv * (vecs[r + 1][c] @ ham.Y[k] @ vecs[r + 1][c])
    return float(e)


# ---------------------------------------------------------------------------
# exact contraction in the transposed order (columns), no truncation
# ---------------------------------------------------------------------------

def exact_columnwise(peps, pepo) -> float:
    """<psi|O|psi> by absorbing columns left to right into an exact (untruncated) MPS.

    The column boundary E[b_0, (l-bundle of column c, row 0..Lx-1) ...] is kept
    as a dense vector over the left bundles of the current column; cost grows
    like (D w D)^Lx, so this is for small lattices only.
    """
    Lx, Ly = len(peps), len(peps[0])
    sand = [[sandwich_full(peps[r][c], pepo[r][c]) for c in range(Ly)] for r in range(Lx)]
    # E over the right bundles of the absorbed columns: shape [R_0, R_1, ..., R_{Lx-1}]
    E = np.ones([1] * Lx)
    for c in range(Ly):
        # absorb column c: contract E[L_0..L_{Lx-1}] with C[L_r, U_r, R_r, D_r] down the column
        cur = E.reshape(E.shape + (1,))  # trailing vertical bond (up leg of row 0) = 1
        # cur legs: [L_0..L_{Lx-1}, vert]; contract row by row
        for r in range(Lx):
            C = sand[r][c]  # [L, U, R, Dn]
            # cur: [R_0..R_{r-1}, L_r, ..., L_{Lx-1}, vert]
            cur = np.moveaxis(cur, r, -2)  # bring L_r next to vert
            shp = cur.shape
            m = cur.reshape(-1, shp[-2] * shp[-1])  # [(rest), (L_r, vert=U_r)]
            Cm = C.reshape(C.shape[0] * C.shape[1], C.shape[2] * C.shape[3])
            res = (m @ Cm).reshape(shp[:-2] + (C.shape[2], C.shape[3]))  # [..., R_r, Dn_r]
            cur = np.moveaxis(res, -2, r)
        E = cur.reshape(cur.shape[:-1])
    return float(E.reshape(-1)[0])
