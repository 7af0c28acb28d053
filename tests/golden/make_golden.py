"""Write stored oracle values for GPU parity tests (calls only oracle/ and synth/).

Configurations (seeded synthetic inputs, no paper data):
  c2_fsm        4x4, D=4, p=4, FSM PEPO w=4 (K=2, random symmetric h, X, Y), chi=64,
                oversample 10, q=2, n_fit=1: <psi|H|psi> (layer 1) and <psi|psi> (layer 0).
  c2_fsm_decay  the same with the decaying-bond-weight PEPS (exp(-i/2) on every
                virtual index), whose bond spectra are well separated.
  c3_fsm[_decay] 6x6, D=6, p=4, FSM PEPO w=4 (K=2, random symmetric h, X, Y), chi=256,
                oversample 10, q=2, n_fit=1: <psi|H|psi> and <psi|psi> by full sweeps,
                the log-scale of every compressed row and the kept spectra of row 2.
  c3_row2       6x6, D=6, p=4, Hubbard-shaped FSM PEPO w=4 (K=2), chi=256: row 2 absorbed
                into a seeded random boundary MPS (bond profile of a top-down sweep),
                zip-up rSVD (oversample 10, q=2) + one CBE fit pass: the row's log-scale,
                the zip-up and fit spectra of every bond.
Usage: python tests/golden/make_golden.py [--decay] [--c3 | --c3row] [seeds...]
       -> tests/golden/c2_fsm[_decay]_seed{S}.json, c3_fsm[_decay]_seed{S}.json,
          c3_row2_seed{S}.json
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import boundary as B  # noqa: E402
from synth import lattice as L    # noqa: E402


def c2(seed: int, sketch_seed: int = 1, decay: bool = False):
    peps = (L.decaying_peps if decay else L.random_peps)(4, 4, 4, 4, seed=seed)
    ham = L.random_hamiltonian(4, 4, 4, 2, seed=seed)
    pepo = L.fsm_pepo(ham)
    prm = B.RsvdParams(oversample=10, power_iters=2, n_fit=1)
    t0 = time.time()
    sn, ln, rows_n = B.contract(peps, pepo, 64, prm, seed=sketch_seed, layer=1, return_rows=True)
    sd, ld, rows_d = B.contract(peps, L.identity_pepo(4, 4, 4), 64, prm, seed=sketch_seed, layer=0, return_rows=True)
    return {
        "config": "4x4 D=4 p=4 FSM w=4 (K=2) chi=64 oversample=10 q=2 n_fit=1" + (" decaying PEPS" if decay else ""),
        "decay": decay,
        "peps_seed": seed, "ham_seed": seed, "sketch_seed": sketch_seed,
        "num_sign": sn, "num_log": ln, "den_sign": sd, "den_log": ld,
        "zip_spectra_row1_layer1": [list(map(float, s)) for s in rows_n[0].zip_spectra],
        "fit_spectra_row1_layer1": [list(map(float, s)) for s in rows_n[0].fit_spectra],
        "oracle_seconds": time.time() - t0,
    }


def c3(seed: int, sketch_seed: int = 1, decay: bool = False):
    peps = (L.decaying_peps if decay else L.random_peps)(6, 6, 6, 4, seed=seed)
    ham = L.random_hamiltonian(6, 6, 4, 2, seed=seed)
    pepo = L.fsm_pepo(ham)
    prm = B.RsvdParams(oversample=10, power_iters=2, n_fit=1)
    t0 = time.time()
    sn, ln, rows_n = B.contract(peps, pepo, 256, prm, seed=sketch_seed, layer=1, return_rows=True)
    t1 = time.time()
    sd, ld, rows_d = B.contract(peps, L.identity_pepo(6, 6, 4), 256, prm, seed=sketch_seed, layer=0,
                                return_rows=True)
    return {
        "config": "6x6 D=6 p=4 FSM w=4 (K=2) chi=256 oversample=10 q=2 n_fit=1" + (" decaying PEPS" if decay else ""),
        "decay": decay,
        "peps_seed": seed, "ham_seed": seed, "sketch_seed": sketch_seed,
        "num_sign": sn, "num_log": ln, "den_sign": sd, "den_log": ld,
        "row_log_scale_layer1": [float(r.log_scale) for r in rows_n],
        "row_log_scale_layer0": [float(r.log_scale) for r in rows_d],
        "zip_spectra_row2_layer1": [list(map(float, s)) for s in rows_n[1].zip_spectra],
        "fit_spectra_row2_layer1": [list(map(float, s)) for s in rows_n[1].fit_spectra],
        "oracle_seconds_layer1": t1 - t0,
        "oracle_seconds": time.time() - t0,
    }


def c3row(seed: int, sketch_seed: int = 1):
    Lx, Ly, D, chi, row, K = 6, 6, 6, 256, 2, 2
    peps, pepo, bnd = L.interior_row_inputs(Lx, Ly, D, chi, row, K, seed)
    prm = B.RsvdParams(oversample=10, power_iters=2, n_fit=1)
    t0 = time.time()
    res = B.absorb_row(bnd, peps[row], pepo[row], chi, prm, seed=sketch_seed, layer=1, row=row)
    return {
        "config": "6x6 D=6 p=4 Hubbard FSM w=4 (K=2) chi=256, row 2 into a seeded boundary, "
                  "oversample=10 q=2 n_fit=1",
        "Lx": Lx, "Ly": Ly, "D": D, "chi": chi, "row": row, "K": K,
        "input_seed": seed, "sketch_seed": sketch_seed,
        "boundary_bonds": [int(bnd[0].shape[0])] + [int(t.shape[2]) for t in bnd],
        "log_scale": float(res.log_scale),
        "zip_spectra": [list(map(float, s)) for s in res.zip_spectra],
        "fit_spectra": [list(map(float, s)) for s in res.fit_spectra],
        "new_bonds": [int(res.T[0].shape[0])] + [int(t.shape[2]) for t in res.T],
        "oracle_seconds": time.time() - t0,
    }


if __name__ == "__main__":
    here = os.path.dirname(os.path.abspath(__file__))
    args = sys.argv[1:]
    decay = "--decay" in args
    big = "--c3" in args
    one_row = "--c3row" in args
    args = [a for a in args if a not in ("--decay", "--c3", "--c3row")]
    for s in [int(x) for x in (args or ["0"])]:
        if one_row:
            out = c3row(s)
            with open(os.path.join(here, f"c3_row2_seed{s}.json"), "w") as f:
                json.dump(out, f, indent=1)
            print(s, out["log_scale"], out["oracle_seconds"])
            continue
        out = (c3 if big else c2)(s, decay=decay)
        stem = "c3_fsm" if big else "c2_fsm"
        name = f"{stem}_decay_seed{s}.json" if decay else f"{stem}_seed{s}.json"
        with open(os.path.join(here, name), "w") as f:
            json.dump(out, f, indent=1)
        print(s, out["num_log"], out["den_log"], out["oracle_seconds"])
