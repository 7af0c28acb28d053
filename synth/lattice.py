"""Seeded synthetic inputs for finite-PEPS / PEPO contraction.

This module generates *data only*: PEPS site tensors, PEPO site tensors and the
Hamiltonian term lists they encode, plus synthetic boundary MPSs of a given
bond profile. It contains none of the contraction, compression or
factorisation arithmetic of the method; both the FP64 oracle and the GPU path
consume what it produces.

Index conventions (paper Sec. II, Fig. 1: ket PEPS, PEPO, bra PEPS):
  PEPS site  A[l, u, r, d, p]          open-boundary legs have dimension 1
  PEPO site  W[l, u, r, d, p, p']      p meets the ket, p' meets the bra
  Boundary   T[t, U, t']               U = (u, u_w, u') bundle, u' fastest

Sites are stored row-major: tensors[r][c], r = 0..Lx-1 top to bottom,
c = 0..Ly-1 left to right.

Random data come from ``numpy.random.Generator(numpy.random.Philox(seed))``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Local basis of a Hubbard site: |0>, |up>, |dn>, |up dn>  (p = 4, paper Sec. V).
HUB_DIM = 4


def _rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=np.array([int(seed) & 0xFFFFFFFFFFFFFFFF, int(stream)], dtype=np.uint64)))


def bond_dims(Lx: int, Ly: int, r: int, c: int, D: int):
    """(Dl, Du, Dr, Dd) of site (r, c) on an open Lx x Ly lattice."""
    return (1 if c == 0 else D, 1 if r == 0 else D, 1 if c == Ly - 1 else D, 1 if r == Lx - 1 else D)


def random_peps(Lx: int, Ly: int, D: int, p: int, seed: int, dtype=np.float64):
    """PEPS with i.i.d. N(0,1) entries drawn site-major, each site scaled to unit Frobenius norm."""
    g = _rng(seed, 1)
    out = []
    for r in range(Lx):
        row = []
        for c in range(Ly):
            shp = bond_dims(Lx, Ly, r, c, D) + (p,)
            a = g.standard_normal(shp)
            a /= np.linalg.norm(a)
            row.append(a.astype(dtype))
        out.append(row)
    return out


def decaying_peps(Lx: int, Ly: int, D: int, p: int, seed: int, dtype=np.float64):
    """Random PEPS whose virtual index i carries weight exp(-i/2) on every bond leg.

    Mimics the decaying bond spectra of physical states (random PEPS have flat spectra).
    """
    base = random_peps(Lx, Ly, D, p, seed)
    out = []
    for row in base:
        new = []
        for a in row:
            a = a.copy()
            for ax in range(4):
                w = np.exp(-0.5 * np.arange(a.shape[ax]))
                sh = [1] * 5
                sh[ax] = a.shape[ax]
                a = a * w.reshape(sh)
            a /= np.linalg.norm(a)
            new.append(a.astype(dtype))
        out.append(new)
    return out


def product_peps(Lx: int, Ly: int, D: int, p: int, seed: int, dtype=np.float64):
    """Product state embedded at bond dimension D: only virtual index 0 is occupied.

    Returns (peps, vectors) where vectors[r][c] is the unit local state v_rc.
    """
    g = _rng(seed, 2)
    peps, vecs = [], []
    for r in range(Lx):
        row, vrow = [], []
        for c in range(Ly):
            v = g.standard_normal(p)
            v /= np.linalg.norm(v)
            a = np.zeros(bond_dims(Lx, Ly, r, c, D) + (p,))
            a[0, 0, 0, 0, :] = v
            row.append(a.astype(dtype))
            vrow.append(v)
        peps.append(row)
        vecs.append(vrow)
    return peps, vecs


def identity_pepo(Lx: int, Ly: int, p: int, dtype=np.float64):
    """w = 1 PEPO that is the identity on every site (the norm <psi|psi>)."""
    w = np.eye(p).reshape(1, 1, 1, 1, p, p).astype(dtype)
    return [[w.copy() for _ in range(Ly)] for _ in range(Lx)]


def _sym(g: np.random.Generator, p: int) -> np.ndarray:
    m = g.standard_normal((p, p))
    return 0.5 * (m + m.T)


def dense_pepo(Lx: int, Ly: int, p: int, w: int, seed: int, dtype=np.float64):
    """PEPO whose every (l,u,r,d) channel block is a random symmetric p x p matrix.

    Open-boundary legs have dimension 1 (channel 0 kept).
    """
    g = _rng(seed, 3)
    out = []
    for r in range(Lx):
        row = []
        for c in range(Ly):
            dl, du, dr, dd = bond_dims(Lx, Ly, r, c, w)
            t = np.zeros((dl, du, dr, dd, p, p))
            for idx in np.ndindex(dl, du, dr, dd):
                t[idx] = _sym(g, p)
            row.append(t.astype(dtype))
        out.append(row)
    return out


# ----------------------------------------------------------------------------
# Finite-state-machine PEPO for H = sum_i h_i + sum_<ij> sum_k t^k_ij X^k_i Y^k_j
# ----------------------------------------------------------------------------

@dataclass
class Hamiltonian:
    """Term list of a nearest-neighbour Hamiltonian on an open Lx x Ly lattice.

    onsite[r][c]      h_rc (p x p)
    X[k], Y[k]        operator pair of hopping channel k (p x p)
    t_h[k][r][c]      coefficient of X^k_(r,c) Y^k_(r,c+1)
    t_v[k][r][c]      coefficient of X^k_(r,c) Y^k_(r+1,c)
    """
    Lx: int
    Ly: int
    p: int
    onsite: list
    X: list
    Y: list
    t_h: np.ndarray = field(default=None)
    t_v: np.ndarray = field(default=None)

    @property
    def K(self) -> int:
        return len(self.X)


def hubbard_operators():
    """Creation/annihilation matrices on the basis |0>,|up>,|dn>,|up dn>.

    Ordering convention |up dn> = c_up^dag c_dn^dag |0>, giving the on-site sign on
    c_dn^dag |up> = -|up dn>. Returns (cu_dag, cu, cd_dag, cd, n_up n_dn).
    """
    cu_dag = np.zeros((4, 4))
    cu_dag[1, 0] = 1.0      # |0>  -> |up>
    cu_dag[3, 2] = 1.0      # |dn> -> |up dn>
    cd_dag = np.zeros((4, 4))
    cd_dag[2, 0] = 1.0      # |0>  -> |dn>
    cd_dag[3, 1] = -1.0     # |up> -> -|up dn>
    nn = np.diag([0.0, 0.0, 0.0, 1.0])
    return cu_dag, cu_dag.T.copy(), cd_dag, cd_dag.T.copy(), nn


def hubbard_hamiltonian(Lx: int, Ly: int, seed: int, K: int = 4) -> Hamiltonian:
    """Hubbard-shaped term list: h_i = U_i n_up n_dn, K hopping channels.

    Channels cycle through (c_up^dag, c_up), (c_up, c_up^dag), (c_dn^dag, c_dn),
    (c_dn, c_dn^dag); U_i and every t^k_ij are N(0,1) from the seed. Bosonic
    sandwich: no inter-site Jordan-Wigner strings.
    """
    g = _rng(seed, 4)
    cu_dag, cu, cd_dag, cd, nn = hubbard_operators()
    pairs = [(cu_dag, cu), (cu, cu_dag), (cd_dag, cd), (cd, cd_dag)]
    X = [pairs[k % 4][0] for k in range(K)]
    Y = [pairs[k % 4][1] for k in range(K)]
    U = g.standard_normal((Lx, Ly))
    onsite = [[U[r, c] * nn for c in range(Ly)] for r in range(Lx)]
    t_h = g.standard_normal((K, Lx, Ly))
    t_v = g.standard_normal((K, Lx, Ly))
    return Hamiltonian(Lx, Ly, HUB_DIM, onsite, X, Y, t_h, t_v)


def random_hamiltonian(Lx: int, Ly: int, p: int, K: int, seed: int) -> Hamiltonian:
    """Random symmetric h_i, X^k, Y^k and N(0,1) couplings."""
    g = _rng(seed, 5)
    onsite = [[_sym(g, p) for _ in range(Ly)] for _ in range(Lx)]
    X = [_sym(g, p) for _ in range(K)]
    Y = [_sym(g, p) for _ in range(K)]
    t_h = g.standard_normal((K, Lx, Ly))
    t_v = g.standard_normal((K, Lx, Ly))
    return Hamiltonian(Lx, Ly, p, onsite, X, Y, t_h, t_v)


def fsm_pepo(ham: Hamiltonian, dtype=np.float64):
    """Finite-state-machine PEPO (bond w = K + 2) that encodes ``ham`` exactly.

    Horizontal bond states: N = 0 (nothing placed yet in this row), D = 1 (the
    one term has been placed), X^k = 2 + k (horizontal term pending).
    Vertical bonds in columns c < Ly-1: I = 0 (pass), X^k = 1 + k (vertical term
    pending); index K + 1 is padding. The last column is a "spine" whose
    vertical bonds use the horizontal encoding {N, D, X^k} and collect the
    single placed term down to the bottom-right corner.
    Boundary legs select N (left), I (top, c < Ly-1), N (top, spine),
    I (bottom, c < Ly-1) and D (bottom-right root).
    """
    Lx, Ly, p, K = ham.Lx, ham.Ly, ham.p, ham.K
    w = K + 2
    N, Dn = 0, 1
    I = 0
    eye = np.eye(p)
    out = []
    for r in range(Lx):
        row = []
        for c in range(Ly):
            full = np.zeros((w, w, w, w, p, p))
            h = ham.onsite[r][c]

            def put(l, u, rr, d, op):
                # op is the operator matrix <p'|op|p>; W[..., p, p'] = op[p', p]
                full[l, u, rr, d] += op.T

            if c < Ly - 1:
                put(N, I, N, I, eye)
                put(Dn, I, Dn, I, eye)
                put(N, I, Dn, I, h)
                for k in range(K):
                    put(N, I, 2 + k, I, ham.X[k])
                    if c > 0:
                        put(2 + k, I, Dn, I, ham.t_h[k, r, c - 1] * ham.Y[k])
                    put(N, I, N, 1 + k, ham.X[k])
                    if r > 0:
                        put(N, 1 + k, Dn, I, ham.t_v[k, r - 1, c] * ham.Y[k])
            else:
                # spine rules (l, u) -> d, r leg is the open boundary (state N)
                put(N, N, N, N, eye)
                put(N, N, N, Dn, h)
                put(Dn, N, N, Dn, eye)
                put(N, Dn, N, Dn, eye)
                for k in range(K):
                    put(N, N, N, 2 + k, ham.X[k])
                    if c > 0:
                        put(2 + k, N, N, Dn, ham.t_h[k, r, c - 1] * ham.Y[k])
                    if r > 0:
                        put(N, 2 + k, N, Dn, ham.t_v[k, r - 1, c] * ham.Y[k])
            # boundary selections
            sl = slice(N, N + 1) if c == 0 else slice(None)
            if r == 0:
                su = slice(N, N + 1) if c == Ly - 1 else slice(I, I + 1)
            else:
                su = slice(None)
            sr = slice(N, N + 1) if c == Ly - 1 else slice(None)
            if r == Lx - 1:
                sd = slice(Dn, Dn + 1) if c == Ly - 1 else slice(I, I + 1)
            else:
                sd = slice(None)
            row.append(np.ascontiguousarray(full[sl, su, sr, sd]).astype(dtype))
        out.append(row)
    return out


def pepo_channels(W: np.ndarray, tol: float = 0.0):
    """Nonzero (l,u,r,d) channel blocks of one PEPO site, in C order (host bookkeeping)."""
    return [idx for idx in np.ndindex(*W.shape[:4]) if np.max(np.abs(W[idx])) > tol]


def random_boundary(bonds, phys, seed: int, dtype=np.float64):
    """Synthetic boundary MPS T_c[t_{c-1}, U_c, t_c] with the given bond profile.

    ``bonds`` has length Ly+1 with bonds[0] = bonds[Ly] = 1; ``phys[c]`` is the
    bundle dimension of site c. Entries N(0,1), each tensor scaled to unit norm.
    """
    g = _rng(seed, 6)
    out = []
    for c in range(len(phys)):
        t = g.standard_normal((bonds[c], phys[c], bonds[c + 1]))
        t /= np.linalg.norm(t)
        out.append(t.astype(dtype))
    return out


def boundary_bond_profile(Ly: int, chi: int, bundle: int):
    """Bond profile min(chi, bundle^(c+1), bundle^(Ly-1-c)) of a boundary of Ly sites."""
    bonds = [1]
    for c in range(Ly - 1):
        left = bundle ** min(c + 1, 8)
        right = bundle ** min(Ly - 1 - c, 8)
        bonds.append(int(min(chi, left, right)))
    bonds.append(1)
    return bonds


def interior_row_inputs(Lx: int, Ly: int, D: int, chi: int, row: int, K: int, seed: int, p: int = 4):
    """Inputs of one interior-row absorption: (peps, pepo, boundary).

    Random PEPS (seed), the Hubbard-shaped FSM PEPO with K hopping channels (p = 4; a
    random Hamiltonian otherwise) and a random boundary MPS with the bond profile of a
    top-to-bottom sweep, bond bundle D (K + 2) D, physical bundles those of ``row``.
    """
    peps = random_peps(Lx, Ly, D, p, seed=seed)
    ham = hubbard_hamiltonian(Lx, Ly, seed=seed, K=K) if p == 4 else random_hamiltonian(Lx, Ly, p, K, seed)
    pepo = fsm_pepo(ham)
    bonds = boundary_bond_profile(Ly, chi, D * (K + 2) * D)
    phys = [peps[row][c].shape[1] * pepo[row][c].shape[1] * peps[row][c].shape[1] for c in range(Ly)]
    bnd = random_boundary(bonds, phys, seed=seed + 1000 * row, dtype=np.float64)
    return peps, pepo, bnd


def pack_lattice(tensors, dtype=np.float64) -> np.ndarray:
    """Concatenate site tensors (row-major site order, each C-contiguous) into one flat buffer."""
    return np.concatenate([np.ascontiguousarray(t, dtype=dtype).ravel() for row in tensors for t in row])


def pack_boundary(tensors, dtype=np.float64) -> np.ndarray:
    return np.concatenate([np.ascontiguousarray(t, dtype=dtype).ravel() for t in tensors])
