"""The five seeded workloads, by what they are and their sizes.

Seeds: workload k (1..5) uses 200303868 + k; system s of the 64-system batch
uses 200303868 * 100 + s.  Block sizes: O = 13, H = 5 (DZVP) or O = 23, H = 7.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import splitmix
from .waterbox import Hamiltonian, gapped_hamiltonian, decay_matrix, overlap_matrix, place_waters, BlockMatrix

BASE_SEED = 200303868


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    n_mol: int
    basis: tuple[int, int]
    seed: int
    eps_filter: float
    tol: float = 1e-9
    switch: float = 0.0          # residual below which the mixed tier switches to FP64

    @property
    def n_atoms(self) -> int:
        return 3 * self.n_mol

    @property
    def n(self) -> int:
        return self.n_mol * (self.basis[0] + 2 * self.basis[1])


# 32 waters, N = 736: one FP64 product C = A.A of the decay matrix, eps 1e-6
DECAY_32 = Workload("decay-32h2o-dzvp-mult", 32, (13, 5), BASE_SEED + 1, 1e-6)
# 1,024 waters, N = 23,552: FP64 sign iteration, eps 1e-7, tol 1e-9
SIGN_1024 = Workload("sign-1024h2o-dzvp-fp64", 1024, (13, 5), BASE_SEED + 2, 1e-7, 1e-9)
# 4,096 waters, O = 23 / H = 7, N = 151,552: mixed sign iteration, switch at 1e-4
SIGN_4096 = Workload("sign-4096h2o-23-7-mixed", 4096, (23, 7), BASE_SEED + 3, 1e-6, 1e-8, 1e-4)
# 20,736 waters, N = 767,232
SIGN_20736 = Workload("sign-20736h2o-23-7-mixed", 20736, (23, 7), BASE_SEED + 5, 1e-6, 1e-8, 1e-4)


# The submatrix method's comparison system: 6,192 waters with a minimal basis (SZV: 4
# functions on O, 1 on H), N = 37,152.
SUBMATRIX_6192 = Workload("submatrix-6192h2o-szv", 6192, (4, 1), BASE_SEED + 6, 1e-6, 1e-9)


def batch_seed(rank: int = 0) -> int:
    """Seed of the uneven-system batch solved by one rank (each rank its own systems)."""
    return BASE_SEED * 100 + 100000 * rank


def batch_systems(n_sys: int = 64, seed: int = BASE_SEED * 100, lo: int = 100, hi: int = 2000):
    """64 uneven systems: n_mol log-uniform in [lo, hi], O in {13, 23}, H in {5, 7}."""
    out = []
    for s in range(n_sys):
        sd = seed + s
        u = splitmix.uniform01(splitmix.substream(sd, 7), np.arange(3, dtype=np.uint64))
        n_mol = int(round(math.exp(math.log(lo) + u[0] * (math.log(hi) - math.log(lo)))))
        b_o = 13 if u[1] < 0.5 else 23
        b_h = 5 if u[2] < 0.5 else 7
        out.append(Workload(f"batch-sys{s}", n_mol, (b_o, b_h), sd, 1e-6, 1e-9))
    return out


def small(n_mol: int, basis=(13, 5), seed: int = BASE_SEED + 11, box: float | None = None,
          eps: float = 1e-7, tol: float = 1e-9) -> Workload:
    return Workload(f"small-{n_mol}h2o", n_mol, basis, seed, eps, tol)


def build_hamiltonian(w: Workload, box: float | None = None) -> Hamiltonian:
    wb = place_waters(w.n_mol, w.seed, box=box)
    return gapped_hamiltonian(wb, w.basis, w.seed)


def build_overlap(w: Workload, box: float | None = None) -> BlockMatrix:
    """The overlap matrix S of the workload's water box (same pattern as its Hamiltonian)."""
    wb = place_waters(w.n_mol, w.seed, box=box)
    return overlap_matrix(wb, w.basis, w.seed)


def build_decay(w: Workload, box: float | None = None) -> BlockMatrix:
    wb = place_waters(w.n_mol, w.seed, box=box)
    return decay_matrix(wb, w.basis, w.seed)[0]
