"""Seeded synthetic workloads shaped like the paper's Hubbard runs (Sec. V).

The paper's trained PEPS tensors are not available, so every workload is
seeded synthetic data of the paper's sizes: random PEPS (N(0,1), unit-norm
sites), a Hubbard-shaped finite-state-machine PEPO (on-site U n_up n_dn and K
hopping channels, coefficients N(0,1)) and, for single-row timing, a seeded
random boundary MPS with the bond profile min(chi, B^(c+1), B^(Ly-1-c)) that a
top-to-bottom sweep produces at an interior row.

Data only (no method arithmetic): built from ``synth.lattice``.
"""
from __future__ import annotations

import struct
from dataclasses import dataclass

import numpy as np

from synth import lattice as L

MAGIC = 0x3144425350455046


@dataclass
class RowWorkload:
    name: str
    Lx: int
    Ly: int
    D: int
    p: int
    K: int
    chi: int
    row: int
    peps: list
    pepo: list
    boundary: list   # T_c [t, U, t']

    @property
    def w(self):
        return self.K + 2


def hubbard_row(name, Lx, Ly, D, chi, row, K=4, seed=0, p=4) -> RowWorkload:
    peps, pepo, bnd = L.interior_row_inputs(Lx, Ly, D, chi, row, K, seed, p)
    return RowWorkload(name, Lx, Ly, D, p, K, chi, row, peps, pepo, bnd)


C3 = dict(name="6x6 D=6 w=4 chi=256 row 2", Lx=6, Ly=6, D=6, chi=256, row=2, K=2)
C4 = dict(name="8x8 D=6 w=6 chi=500 row 4", Lx=8, Ly=8, D=6, chi=500, row=4, K=4)


def boundary_blob(tensors, next_row: int, layer: int, elem: int, log_scale: float = 0.0) -> bytes:
    """Checkpoint layout of fpeps_export_boundary / fpeps_import_boundary."""
    Ly = len(tensors)
    bonds = [tensors[0].shape[0]] + [t.shape[2] for t in tensors]
    phys = [t.shape[1] for t in tensors]
    head = struct.pack(f"<{5 + Ly + 1 + Ly}q", MAGIC, Ly, next_row, layer, elem, *bonds, *phys)
    head += struct.pack("<d", log_scale)
    dt = np.float64 if elem == 8 else np.float32
    body = b"".join(np.ascontiguousarray(t, dtype=dt).tobytes() for t in tensors)
    return head + body
