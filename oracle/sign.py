"""Density matrix by the sign-matrix iteration, FP64 (TEST INFRASTRUCTURE ONLY).

Follows the paper's section "Sign-Method":

* sign(A) = A (A^2)^(-1/2) (Eq. signdef); the density matrix of an orthogonal
  basis (S = 1) is P = (1 - sign(H - mu 1)) / 2;
* the second-order Newton-Schulz iteration X_{k+1} = X_k (3 - X_k^2) / 2, the
  polynomial the paper also prints as the first refinement function
  f_1(Z) = Z (3 - Y) / 2 with Y = Z^2 (section "OT/IR");
* after every matrix product the small blocks are flushed to zero with
  eps_filter.

Readings taken where the paper is silent:

* X_0 = (H - mu 1) / alpha with alpha = max_i sum_j |(H - mu 1)_ij| (the
  Gershgorin bound on the spectral radius), so that the spectrum of X_0 lies in
  [-1, 1] where the iteration converges; sign is invariant under this scaling;
* each step forms X2 = filter(X X), tests r = ||X2 - 1||_F / N on the
  filtered product (the paper flushes small elements after every product, so
  X2 is the square the method holds), stops when r < tol, and otherwise sets
  T = 3 1 - X2 and X <- filter(X T / 2) (product on the right);
* at most ``max_iter`` steps.  Without filtering every eigenvalue moves toward
  +-1 monotonically and the residual ratio r_k / r_{k-1} only falls, so once a
  step has cut the residual by more than half, the next one must too; a step
  that does not (r_k > r_{k-1} / 2 after r_{k-1} < r_{k-2} / 2) means filtering
  has stalled the iteration (reported, not raised);
* Tr(P) = (N - Tr X) / 2 and the band energy is E = Tr(P H), with no spin factor.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

from . import bsr


@dataclasses.dataclass
class SignResult:
    X: bsr.Mat                 # converged sign(H - mu 1)
    P: bsr.Mat                 # density matrix (1 - X) / 2
    iterations: int            # Newton-Schulz steps taken (products X.X formed)
    residuals: list            # r_k = ||X_k^2 - 1||_F / N per step
    converged: bool
    stalled: bool
    alpha: float               # Gershgorin scale
    trace_p: float             # Tr(P)
    e_band: float              # Tr(P H)
    flops: int                 # sum of 2 m k n over every block product
    n_products: int
    seconds: float
    nnzb_history: list         # blocks of X after each step


def gershgorin(H: bsr.Mat, mu: float) -> float:
    """max_i sum_j |(H - mu 1)_ij|."""
    return float(bsr.abs_row_sums(H, mu).max())


def sign_iterate(H: bsr.Mat, mu: float, eps: float, tol: float, max_iter: int = 100,
                 stall_ratio: float = 0.5) -> SignResult:
    t0 = time.perf_counter()
    n = H.n
    alpha = gershgorin(H, mu)
    X = bsr.add_identity(H, 1.0 / alpha, -mu / alpha)          # (H - mu 1) / alpha
    res, flops, nprod, hist = [], 0, 0, []
    converged = stalled = False
    it = 0
    while it < max_iter:
        X2, info = bsr.multiply(1.0, X, X, eps=eps, info=True)
        it += 1
        flops += info.flops
        nprod += info.n_products
        r = float(np.sqrt(info.dev2)) / n
        res.append(r)
        if r < tol:
            converged = True
            break
        if len(res) >= 3 and res[-2] < stall_ratio * res[-3] and r > stall_ratio * res[-2]:
            stalled = True
            break
        T = bsr.add_identity(X2, -1.0, 3.0)                        # 3 1 - X^2
        X, info = bsr.multiply(0.5, X, T, eps=eps, info=True)      # X (3 1 - X^2) / 2
        flops += info.flops
        nprod += info.n_products
        hist.append(X.nnzb)
    P = bsr.add_identity(X, -0.5, 0.5)                             # (1 - X) / 2
    trace_p = bsr.trace(P)
    e_band = bsr.trace_product(P, H)
    return SignResult(X=X, P=P, iterations=it, residuals=res, converged=converged, stalled=stalled,
                      alpha=alpha, trace_p=trace_p, e_band=e_band, flops=flops, n_products=nprod,
                      seconds=time.perf_counter() - t0, nnzb_history=hist)


def band_energy(P: bsr.Mat, H: bsr.Mat) -> float:
    """E_band = Tr(P H)."""
    return bsr.trace_product(P, H)
