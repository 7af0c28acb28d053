"""Write stored oracle values for GPU parity tests (calls only oracle/ and synth/).

Configurations (seeded synthetic inputs, no paper data):
  c2_fsm        4x4, D=4, p=4, FSM PEPO w=4 (K=2, random symmetric h, X, Y), chi=64,
                oversample 10, q=2, n_fit=1: <psi|H|psi> (layer 1) and <psi|psi> (layer 0).
  c2_fsm_decay  the same with the decaying-bond-weight PEPS (exp(-i/2) on every
                virtual index), whose bond spectra are well separated.
Usage: python tests/golden/make_golden.py [--decay] [seeds...]
       -> tests/golden/c2_fsm[_decay]_seed{S}.json
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


if __name__ == "__main__":
    here = os.path.dirname(os.path.abspath(__file__))
    args = sys.argv[1:]
    decay = "--decay" in args
    args = [a for a in args if a != "--decay"]
    for s in [int(x) for x in (args or ["0"])]:
        out = c2(s, decay=decay)
        name = f"c2_fsm_decay_seed{s}.json" if decay else f"c2_fsm_seed{s}.json"
        with open(os.path.join(here, name), "w") as f:
            json.dump(out, f, indent=1)
        print(s, out["num_log"], out["den_log"], out["oracle_seconds"])
