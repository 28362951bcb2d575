"""Writes the exact (dense eigendecomposition, unfiltered) occupation and band
energy of the 1,024-water Hamiltonian (N = 23,552) to
tests/golden/exact_1024h2o.json.  Calls only the input generator and oracle/.
Takes ~20 GB of host memory and tens of minutes."""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import synth  # noqa: E402
from oracle import bsr, dense  # noqa: E402


def main():
    w = synth.SIGN_1024
    h = synth.build_hamiltonian(w)
    t0 = time.time()
    n_occ, e_band, ev = dense.band_energy_exact(bsr.Mat.of(h.H), h.mu)
    out = {"workload": w.name, "N": w.n, "n_atoms": h.n_atoms, "mu": h.mu, "trace_p": n_occ, "e_band": e_band,
           "e_band_per_atom": e_band / h.n_atoms, "homo": float(ev[ev < h.mu].max()),
           "lumo": float(ev[ev > h.mu].min()), "e_min": float(ev[0]), "e_max": float(ev[-1]),
           "seconds": time.time() - t0,
           "source": "oracle/dense.py (numpy eigvalsh of the dense H), written by tests/golden/make_golden_exact.py"}
    with open(os.path.join(HERE, "exact_1024h2o.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
