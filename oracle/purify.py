"""Canonical density matrices without a known chemical potential, FP64 (TEST INFRASTRUCTURE
ONLY).

Section "Purification methods": purifications map the eigenvalues of K to occupations and
are grand-canonical by construction; canonical ensembles need modified algorithms or
extra iterations to place mu.  CP2K offers the trace-resetting fourth-order method
(TRS4), the trace-conserving second-order method (TC2) and the sign method.  The paper
names them only; the steps below restate the published algorithms (TC2: Niklasson,
Phys. Rev. B 66, 155115 (2002); TRS4: Niklasson, Tymczak and Challacombe,
J. Chem. Phys. 118, 8611 (2003)):

* start: X_0 = (g 1 - H) / (2 g) with g = max_i sum_j |H_ij| (the Gershgorin bound, so
  the spectrum of X_0 lies in [0, 1] and the lowest states of H sit near 1);
* TC2 step: X <- X^2 when Tr(X) > N_occ, else X <- 2 X - X^2 (one product);
* TRS4 step: with X2 = X^2, F = X2 (4 X - 3 X2) and G = X2 (1 - X)^2, the trace-resetting
  parameter gamma = (N_occ - Tr F) / Tr G; gamma in [0, 6]: X <- F + gamma G =
  X2 (gamma + (4 - 2 gamma) X + (gamma - 3) X2); gamma > 6: X <- 2 X - X2;
  gamma < 0: X <- X2 (two products in the first case, one otherwise);
* the sign method with the chemical potential found by bisection: mu halves
  [mu_lo, mu_hi] (default the Gershgorin interval of H) until Tr(P(mu)) is within 1/2 of
  N_occ, each trial a full sign iteration.

Readings where the paper is silent: every product is filtered with eps_filter; the
traces Tr(X^2), Tr(X^3) = Tr(X2 X), Tr(X^4) = Tr(X2 X2) come from the factors without
forming the products; the iteration stops when the idempotency measure
(Tr X - Tr X^2) / N = sum_i x_i (1 - x_i) / N falls below tol, or after max_iter steps.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

from . import bsr, sign


@dataclasses.dataclass
class PurifyResult:
    P: bsr.Mat
    iterations: int
    converged: bool
    idempotency: list          # (Tr X - Tr X^2) / N before each step
    steps: dict                # how often each branch ran
    trace_p: float
    e_band: float
    scale: float               # g
    flops: int
    multiplies: int
    seconds: float


def _start(H: bsr.Mat):
    g = sign.gershgorin(H, 0.0)
    return bsr.add_identity(H, -1.0 / (2 * g), 0.5), g          # (g 1 - H) / (2 g)


def purify(H: bsr.Mat, n_occ: float, eps: float, tol: float, method: str = "tc2",
           max_iter: int = 200) -> PurifyResult:
    """TC2 or TRS4 purification of H to the projector on its n_occ lowest states."""
    if method not in ("tc2", "trs4"):
        raise ValueError(method)
    t0 = time.perf_counter()
    n = H.n
    X, g = _start(H)
    hist, steps = [], {"square": 0, "two_minus": 0, "trs4": 0}
    flops = mults = 0
    converged = False
    it = 0

    def mult(alpha, A, B, beta=0.0, Cin=None):
        nonlocal flops, mults
        C, inf = bsr.multiply(alpha, A, B, beta, Cin, eps=eps, info=True)
        flops += inf.flops
        mults += 1
        return C

    while it < max_iter:
        t1 = bsr.trace(X)
        t2 = bsr.trace_product(X, X)
        e = (t1 - t2) / n
        hist.append(e)
        if abs(e) < tol:
            converged = True
            break
        it += 1
        if method == "tc2":
            if t1 > n_occ:
                X = mult(1.0, X, X)
                steps["square"] += 1
            else:
                X = mult(-1.0, X, X, 2.0, X)                     # 2 X - X^2
                steps["two_minus"] += 1
            continue
        X2 = mult(1.0, X, X)
        s2 = bsr.trace(X2)
        s3 = bsr.trace_product(X2, X)
        s4 = bsr.trace_product(X2, X2)
        tr_f = 4 * s3 - 3 * s4
        tr_g = s2 - 2 * s3 + s4
        gamma = (n_occ - tr_f) / tr_g if tr_g != 0 else (7.0 if n_occ > tr_f else -1.0)
        if gamma > 6:
            X = bsr.add(2.0, X, -1.0, X2)
            steps["two_minus"] += 1
        elif gamma < 0:
            X = X2
            steps["square"] += 1
        else:
            Q = bsr.add(4.0 - 2.0 * gamma, X, gamma - 3.0, X2)   # (4 - 2 gamma) X + (gamma - 3) X2
            Q = bsr.add_identity(Q, 1.0, gamma)                  # + gamma 1
            X = mult(1.0, X2, Q)
            steps["trs4"] += 1
    return PurifyResult(P=X, iterations=it, converged=converged, idempotency=hist, steps=steps,
                        trace_p=bsr.trace(X), e_band=bsr.trace_product(X, H), scale=g, flops=flops,
                        multiplies=mults, seconds=time.perf_counter() - t0)


@dataclasses.dataclass
class MuSearchResult:
    mu: float
    result: sign.SignResult
    evaluations: int
    mus: list
    traces: list


def mu_search(H: bsr.Mat, n_occ: float, eps: float, tol: float, mu_lo: float | None = None,
              mu_hi: float | None = None, max_eval: int = 60, order: int = 2) -> MuSearchResult:
    """Sign method with mu placed by bisection so that Tr(P) = n_occ (within 1/2)."""
    g = sign.gershgorin(H, 0.0)
    lo = -g if mu_lo is None else mu_lo
    hi = g if mu_hi is None else mu_hi
    mus, trs = [], []
    r = None
    for k in range(max_eval):
        mu = 0.5 * (lo + hi)
        r = sign.sign_iterate(H, mu, eps, tol, order=order)
        mus.append(mu)
        trs.append(r.trace_p)
        if abs(r.trace_p - n_occ) < 0.5:
            return MuSearchResult(mu=mu, result=r, evaluations=k + 1, mus=mus, traces=trs)
        if r.trace_p > n_occ:
            hi = mu
        else:
            lo = mu
    return MuSearchResult(mu=mus[-1], result=r, evaluations=max_eval, mus=mus, traces=trs)
