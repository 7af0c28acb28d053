"""Seeded U(1) x U(1) charged inputs: charge-conserving PEPS and the charge labels
of the Hubbard FSM PEPO legs (data and bookkeeping only).

The paper's Hubbard runs use U(1)_spin x U(1)_charge symmetric tensors (Sec. V).
Here a charge is the pair (N_up, N_dn), an equivalent basis of the same group
(S^z = (N_up - N_dn)/2, N = N_up + N_dn). Every leg carries a charge per index;
a tensor is charge conserving when each nonzero entry satisfies

  PEPS  A[l,u,r,d,p]:      q_l + q_u + q_p = q_r + q_d + f_site
  PEPO  W[l,u,r,d,p,p']:   q_l + q_u + q_p = q_r + q_d + q_p'

(l, u and the ket physical index flow in; r, d and the bra physical index flow
out; f_site is a fixed charge per PEPS site, like a dimension-1 charged leg).
Open-boundary legs have dimension 1 and charge (0, 0).

This module contains none of the contraction or compression arithmetic; it only
draws tensors and records charges. Random data come from
``numpy.random.Generator(numpy.random.Philox(seed))``.
"""
from __future__ import annotations

import numpy as np

from .lattice import HUB_DIM, _rng, bond_dims

# charges (N_up, N_dn) of the Hubbard basis |0>, |up>, |dn>, |up dn>
HUB_CHARGES = np.array([[0, 0], [1, 0], [0, 1], [1, 1]], dtype=np.int64)

# candidate sector charges of a virtual bond
_BOND_CHARGES = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, -1], [1, -1], [-1, 1]],
                         dtype=np.int64)


def bond_charges(g: np.random.Generator, D: int) -> np.ndarray:
    """Charges of a virtual bond of dimension D: sectors of 1-3 indices with
    distinct charges, listed sector by sector. Returns a (D, 2) int array."""
    if D == 1:
        return np.zeros((1, 2), dtype=np.int64)
    sizes = []
    left = D
    while left > 0:
        s = int(g.integers(1, min(3, left) + 1))
        sizes.append(s)
        left -= s
    pick = g.permutation(len(_BOND_CHARGES))[:len(sizes)]
    return np.concatenate([np.repeat(_BOND_CHARGES[i][None, :], s, axis=0) for i, s in zip(pick, sizes)])


def site_balance(ql, qu, qr, qd, qp) -> np.ndarray:
    """q_l + q_u + q_p - q_r - q_d over the index grid [l, u, r, d, p, 2]."""
    return (ql[:, None, None, None, None, :] + qu[None, :, None, None, None, :]
            + qp[None, None, None, None, :, :] - qr[None, None, :, None, None, :]
            - qd[None, None, None, :, None, :])


def u1_peps(Lx: int, Ly: int, D: int, seed: int, dtype=np.float64):
    """Charge-conserving random PEPS on the Hubbard basis (p = 4).

    Returns (peps, charges): charges["h"][r][c] labels the bond between (r, c) and
    (r, c+1) (c < Ly-1), charges["v"][r][c] the bond between (r, c) and (r+1, c)
    (r < Lx-1), charges["flux"][r][c] the site charge f, charges["phys"] the
    physical charges. The fluxes come from one seeded reference configuration (an
    index on every bond, a basis state on every site): f is the balance of that
    configuration at each site, so the configuration is allowed everywhere and the
    state does not vanish. Entries are N(0,1) where a site's balance equals f and
    zero elsewhere; each site is scaled to unit Frobenius norm.
    """
    g = _rng(seed, 11)
    h = [[bond_charges(g, D) for _ in range(Ly - 1)] for _ in range(Lx)]
    v = [[bond_charges(g, D) for _ in range(Ly)] for _ in range(Lx - 1)]
    ref_h = g.integers(0, D, size=(Lx, max(Ly - 1, 1)))
    ref_v = g.integers(0, D, size=(max(Lx - 1, 1), Ly))
    ref_p = g.integers(0, HUB_DIM, size=(Lx, Ly))
    zero = np.zeros((1, 2), dtype=np.int64)
    peps, flux = [], []
    for r in range(Lx):
        row, frow = [], []
        for c in range(Ly):
            ql = h[r][c - 1] if c > 0 else zero
            qr = h[r][c] if c < Ly - 1 else zero
            qu = v[r - 1][c] if r > 0 else zero
            qd = v[r][c] if r < Lx - 1 else zero
            il = ref_h[r, c - 1] if c > 0 else 0
            ir = ref_h[r, c] if c < Ly - 1 else 0
            iu = ref_v[r - 1, c] if r > 0 else 0
            idn = ref_v[r, c] if r < Lx - 1 else 0
            f = ql[il] + qu[iu] + HUB_CHARGES[ref_p[r, c]] - qr[ir] - qd[idn]
            mask = np.all(site_balance(ql, qu, qr, qd, HUB_CHARGES) == f, axis=-1)
            a = g.standard_normal(bond_dims(Lx, Ly, r, c, D) + (HUB_DIM,)) * mask
            a /= np.linalg.norm(a)
            row.append(a.astype(dtype))
            frow.append(f)
        peps.append(row)
        flux.append(frow)
    return peps, {"h": h, "v": v, "flux": flux, "phys": HUB_CHARGES}


def peps_leg_charges(ch, Lx: int, Ly: int, r: int, c: int):
    """(q_l, q_u, q_r, q_d) of PEPS site (r, c)."""
    zero = np.zeros((1, 2), dtype=np.int64)
    return (ch["h"][r][c - 1] if c > 0 else zero, ch["v"][r - 1][c] if r > 0 else zero,
            ch["h"][r][c] if c < Ly - 1 else zero, ch["v"][r][c] if r < Lx - 1 else zero)


def operator_shift(op: np.ndarray) -> np.ndarray:
    """Charge change q(p') - q(p) of an operator with matrix <p'|op|p> on the Hubbard
    basis; every nonzero element must agree (else the operator is not charged)."""
    nz = np.argwhere(op != 0)
    shifts = {tuple(HUB_CHARGES[pp] - HUB_CHARGES[p]) for pp, p in nz}
    if len(shifts) != 1:
        raise ValueError("operator does not carry a definite charge")
    return np.array(shifts.pop(), dtype=np.int64)


def hubbard_pepo_charges(ham):
    """Charges of the legs of ``synth.lattice.fsm_pepo(ham)``, site by site.

    Horizontal bond states N, D carry (0, 0) and the pending state X^k minus the shift
    of X^k (the charge that Y^k, placed further on, gives back); vertical bonds of
    columns c < Ly-1 carry I = (0, 0), X^k = minus the shift of X^k and (0, 0) for the
    padding index; the spine column's vertical bonds use the
    horizontal encoding. Boundary legs keep the selected state's charge. Returns
    [r][c] -> (q_l, q_u, q_r, q_d).
    """
    Lx, Ly, K = ham.Lx, ham.Ly, ham.K
    w = K + 2
    dk = [operator_shift(x) for x in ham.X]
    horiz = np.zeros((w, 2), dtype=np.int64)
    vert = np.zeros((w, 2), dtype=np.int64)
    for k in range(K):
        horiz[2 + k] = -dk[k]
        vert[1 + k] = -dk[k]
    N, Dn, I = 0, 1, 0
    out = []
    for r in range(Lx):
        row = []
        for c in range(Ly):
            spine = c == Ly - 1
            qv = horiz if spine else vert
            ql = horiz[N:N + 1] if c == 0 else horiz
            qu = (horiz[N:N + 1] if spine else vert[I:I + 1]) if r == 0 else qv
            qr = horiz[N:N + 1] if spine else horiz
            qd = (horiz[Dn:Dn + 1] if spine else vert[I:I + 1]) if r == Lx - 1 else qv
            row.append((ql, qu, qr, qd))
        out.append(row)
    return out

