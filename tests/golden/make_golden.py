"""Writes the oracle's results for the 1,024-water sign iteration (N = 23,552,
eps 1e-7, tol 1e-9) to tests/golden/sign_1024h2o.json.

Calls only the input generator and oracle/ (FP64 plain C, no GPU).  The values
are the oracle's own; the GPU test compares its band energy per atom with them.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import bsr, sign  # noqa: E402


def main():
    w = synth.SIGN_1024
    h = synth.build_hamiltonian(w)
    t0 = time.time()
    r = sign.sign_iterate(bsr.Mat.of(h.H), h.mu, w.eps_filter, w.tol)
    out = {"workload": w.name, "n_mol": w.n_mol, "n_atoms": h.n_atoms, "N": w.n, "eps_filter": w.eps_filter,
           "tol": w.tol, "mu": h.mu, "gamma": h.gamma, "alpha": r.alpha, "iterations": r.iterations,
           "converged": r.converged, "stalled": r.stalled, "residuals": r.residuals, "trace_p": r.trace_p,
           "e_band": r.e_band, "e_band_per_atom": r.e_band / h.n_atoms, "flops": r.flops,
           "n_products": r.n_products, "nnzb_history": r.nnzb_history, "oracle_threads": bsr.num_threads(),
           "oracle_seconds": time.time() - t0,
           "source": "oracle/sign.py (FP64 plain C), written by tests/golden/make_golden.py"}
    with open(os.path.join(HERE, "sign_1024h2o.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: out[k] for k in ("iterations", "converged", "trace_p", "e_band", "oracle_seconds")}))


if __name__ == "__main__":
    main()
