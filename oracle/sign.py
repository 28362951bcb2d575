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

Higher orders (section "Sign-Method": third- and fifth-order steps from Pade
approximants, up to seventh order; the fifth-order step is printed as
X_{k+1} = X_k (35 X^8 - 180 X^6 + 378 X^4 - 420 X^2 + 315) / 128 and taken with four
products per iteration):

* the step of order n + 1 is X <- X p_n(X^2) with p_n(y) = sum_{j<=n} c_j (1 - y)^j and
  c_j = binom(2j, j) / 4^j, the series of (1 - z)^(-1/2) cut after j = n (sign(x) =
  x (x^2)^(-1/2) = x (1 - (1 - x^2))^(-1/2)).  n = 1, 2, 3 give the refinement functions
  f_1, f_2, f_3 printed in section "OT/IR", n = 4 the printed fifth-order step;
* the paper names neither the four products nor where the filter sits between them.
  The reading taken, with Y = filter(X X) (the residual test as above), Z = 1 - Y
  (no product), Z2 = filter(Z Z) and the pairs q_i = c_2i + c_2i+1 Z:
  p_n = q_0 + Z2 R with R = sum_{i>=1} Z2^(i-1) q_i (plus c_n Z2^(n/2 - 1) when n is even),
  R summed innermost first, R <- filter(Z2 R + q_i); then V = filter(Z2 R),
  U = q_0 + V (an unfiltered sum) and X <- filter(X U).  For n = 2, R = c_2 and
  U = q_0 + c_2 Z2 directly.  For n = 4 that is exactly four products: X X, Z Z, Z2 R,
  X U.  Orders 3, 4, 6, 7 take 3, 4, 5, 5.  Two choices here decide how far the
  filtered iteration gets:
  - powers of Z rather than of Y (the printed form): the c_j are positive and at most
    1, so no intermediate is a cancelling sum of large terms;
  - near convergence U - 1 is c_1 Z, a matrix of residual-sized blocks.  Filtering it
    on its own (as the output of a product such as Z2 R + q_0) drops the corrections of
    blocks just above eps, which then are never made: at eps 1e-7 the seventh order
    stalled near r = 1e-8 that way, where Newton-Schulz reaches 4e-12.  Every filtered
    product here holds either a Z2 factor or X, as Newton-Schulz's X (3 - Y) / 2 does;
* the stall test above is kept for every order: per eigenvalue the step maps
  e = 1 - x^2 to e' with e'/e increasing in e, the premise of that test.

Non-orthogonal basis (section "Sign-Method": P = (1 - sign(S^-1 K - mu 1)) S^-1 / 2,
with inverse square roots from the sign of the block matrix [[0, A], [1, 0]], which is
[[0, A^(1/2)], [A^(-1/2), 0]]):

* inverse_sqrt runs the sign iteration of the chosen order on that block matrix, in the
  coupled form its block structure gives (Y, Z below), on A = S / g with g the largest
  absolute row sum of S, from Y_0 = A, Z_0 = 1, testing ||Z Y - 1||_F / N;
* density_matrix_nonorth takes the reading P = S^(-1/2) P' S^(-1/2), where P' is the
  density matrix of K' = S^(-1/2) K S^(-1/2) (the sign of S^-1 K - mu 1 is the sign of
  K' - mu 1 under the similarity by S^(1/2)); every product is filtered.
"""
from __future__ import annotations

import dataclasses
import math
import time
from fractions import Fraction

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
    multiplies: int = 0        # matrix products formed
    order: int = 2


def gershgorin(H: bsr.Mat, mu: float) -> float:
    """max_i sum_j |(H - mu 1)_ij|."""
    return float(bsr.abs_row_sums(H, mu).max())


def series_coefficients(order: int) -> list:
    """Exact c_0..c_n (n = order - 1), c_j = binom(2j, j) / 4^j: p_n(y) = sum_j c_j (1 - y)^j."""
    return [Fraction(math.comb(2 * j, j), 4 ** j) for j in range(order)]


def pade_coefficients(order: int) -> list:
    """Exact coefficients a_0..a_n of the same p_n in powers of y, p_n(y) = sum_i a_i y^i
    (the form the paper prints)."""
    c = series_coefficients(order)
    a = [Fraction(0)] * len(c)
    for j, cj in enumerate(c):
        for i in range(j + 1):                                   # (1 - y)^j, binomially
            a[i] += cj * math.comb(j, i) * (-1) ** i
    return a


def _step_polynomial(Y: bsr.Mat, order: int, eps: float, mult) -> bsr.Mat:
    """U = p_n(Y) for the step of the given order, by the scheme of the module header
    (Y = filter(X X), or Z Y in the square-root iteration); mult(alpha, A, B, beta, Cin)
    forms one filtered product.  Order 2: U = (3 - Y) / 2, no product."""
    n = order - 1
    c = [float(v) for v in series_coefficients(order)]
    if n == 1:
        return bsr.add_identity(Y, -c[1], c[0] + c[1])             # 1 + (1 - Y)/2

    Z = bsr.add_identity(Y, -1.0, 1.0)                           # 1 - Y

    def pair(i):                                                 # c_2i+1 Z + c_2i 1
        return bsr.add_identity(Z, c[2 * i + 1], c[2 * i])

    Z2 = mult(1.0, Z, Z)
    m = n // 2
    if n % 2 == 0:
        R = bsr.add(1.0, pair(m - 1), c[n], Z2)
        i = m - 2
    else:
        R = pair(m)
        i = m - 1
    if n == 2:
        return R                                                 # q_0 + c_2 Z2
    while i >= 1:
        R = mult(1.0, Z2, R, 1.0, pair(i))
        i -= 1
    return bsr.add(1.0, pair(0), 1.0, mult(1.0, Z2, R))


class _Work:
    """Counts the filtered products of an iteration."""

    def __init__(self, eps: float, prescreen: bool = False):
        self.eps, self.flops, self.n_products, self.multiplies = eps, 0, 0, 0
        self.prescreen = prescreen

    def __call__(self, alpha, A, B, beta=0.0, Cin=None, info=False):
        C, inf = bsr.multiply(alpha, A, B, beta, Cin, eps=self.eps, info=True, prescreen=self.prescreen)
        self.flops += inf.flops
        self.n_products += inf.n_products
        self.multiplies += 1
        return (C, inf) if info else C


def _higher_order_update(X: bsr.Mat, Y: bsr.Mat, order: int, eps: float, prescreen: bool = False):
    """X p_n(Y) for Y = filter(X X), by the four-product scheme of the module header.
    Returns the new X and the (flops, block products, matrix products) it took."""
    w = _Work(eps, prescreen)
    U = _step_polynomial(Y, order, eps, w)
    Xn = w(1.0, X, U)
    return Xn, (w.flops, w.n_products, w.multiplies)


def sign_iterate(H: bsr.Mat, mu: float, eps: float, tol: float, max_iter: int = 100,
                 stall_ratio: float = 0.5, order: int = 2, prescreen: bool = False) -> SignResult:
    """prescreen: every product forms only the blocks whose norm bound reaches eps
    (bsr.multiply); the iteration is the same bit for bit, with fewer block products."""
    t0 = time.perf_counter()
    n = H.n
    alpha = gershgorin(H, mu)
    X = bsr.add_identity(H, 1.0 / alpha, -mu / alpha)          # (H - mu 1) / alpha
    if not 2 <= order <= 7:
        raise ValueError("order must be 2 to 7")
    res, flops, nprod, hist = [], 0, 0, []
    mults = 0
    converged = stalled = False
    it = 0
    while it < max_iter:
        X2, info = bsr.multiply(1.0, X, X, eps=eps, info=True, prescreen=prescreen)
        mults += 1
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
        if order == 2:
            T = bsr.add_identity(X2, -1.0, 3.0)                    # 3 1 - X^2
            X, info = bsr.multiply(0.5, X, T, eps=eps, info=True, prescreen=prescreen)  # X (3 1 - X^2) / 2
            flops += info.flops
            nprod += info.n_products
            mults += 1
        else:
            X, (f, npr, nm) = _higher_order_update(X, X2, order, eps, prescreen)
            flops += f
            nprod += npr
            mults += nm
        hist.append(X.nnzb)
    P = bsr.add_identity(X, -0.5, 0.5)                             # (1 - X) / 2
    trace_p = bsr.trace(P)
    e_band = bsr.trace_product(P, H)
    return SignResult(X=X, P=P, iterations=it, residuals=res, converged=converged, stalled=stalled,
                      alpha=alpha, trace_p=trace_p, e_band=e_band, flops=flops, n_products=nprod,
                      seconds=time.perf_counter() - t0, nnzb_history=hist, multiplies=mults, order=order)


def band_energy(P: bsr.Mat, H: bsr.Mat) -> float:
    """E_band = Tr(P H)."""
    return bsr.trace_product(P, H)


# ------------------------------------------------------------------ non-orthogonal basis
@dataclasses.dataclass
class SqrtResult:
    Sinvsqrt: bsr.Mat          # S^(-1/2)
    Ssqrt: bsr.Mat             # S^(1/2)
    iterations: int
    residuals: list            # ||Z Y - 1||_F / N per step
    converged: bool
    stalled: bool
    scale: float               # g: the iteration runs on S / g
    flops: int
    n_products: int
    multiplies: int


def identity_like(M: bsr.Mat) -> bsr.Mat:
    """The identity with M's block sizes (diagonal blocks only)."""
    nb = M.nblk
    data = np.concatenate([np.eye(int(b)).ravel() for b in M.bs]) if nb else np.zeros(0)
    return bsr.Mat(M.bs, np.arange(nb + 1, dtype=np.int64), np.arange(nb, dtype=np.int32), data)


def inverse_sqrt(S: bsr.Mat, eps: float, tol: float, max_iter: int = 100, stall_ratio: float = 0.5,
                 order: int = 2) -> SqrtResult:
    """S^(-1/2) and S^(1/2) of a symmetric positive definite S by the sign iteration on the
    block matrix [[0, A], [1, 0]] (section "Sign-Method": its sign is [[0, A^(1/2)],
    [A^(-1/2), 0]]), A = S / g with g = max_i sum_j |S_ij| so that the spectrum of A lies in
    (0, 1].  The iterate keeps the form [[0, Y], [Z, 0]]; its square is diag(Y Z, Z Y), and
    with Y, Z functions of A (so Y Z = Z Y) the step X <- X p(X^2) reads
        W = filter(Z Y);  r = ||W - 1||_F / N;  stop when r < tol;
        U = p(W);  Y <- filter(Y U);  Z <- filter(U Z)
    from Y_0 = A, Z_0 = 1 (U as in the sign iteration of the same order).  Then
    S^(1/2) = sqrt(g) Y and S^(-1/2) = Z / sqrt(g).  The stall test is the sign iteration's."""
    if not 2 <= order <= 7:
        raise ValueError("order must be 2 to 7")
    n = S.n
    g = gershgorin(S, 0.0)
    Y = bsr.add_identity(S, 1.0 / g, 0.0)
    Zm = identity_like(S)
    w = _Work(eps)
    res = []
    converged = stalled = False
    it = 0
    while it < max_iter:
        W, inf = w(1.0, Zm, Y, info=True)
        it += 1
        r = float(np.sqrt(inf.dev2)) / n
        res.append(r)
        if r < tol:
            converged = True
            break
        if len(res) >= 3 and res[-2] < stall_ratio * res[-3] and r > stall_ratio * res[-2]:
            stalled = True
            break
        U = _step_polynomial(W, order, eps, w)
        Y = w(1.0, Y, U)
        Zm = w(1.0, U, Zm)
    rg = float(np.sqrt(g))
    return SqrtResult(Sinvsqrt=bsr.add_identity(Zm, 1.0 / rg, 0.0), Ssqrt=bsr.add_identity(Y, rg, 0.0),
                      iterations=it, residuals=res, converged=converged, stalled=stalled, scale=g,
                      flops=w.flops, n_products=w.n_products, multiplies=w.multiplies)


@dataclasses.dataclass
class NonorthResult:
    P: bsr.Mat                 # density matrix in the non-orthogonal basis
    sign: SignResult           # the sign iteration on S^(-1/2) K S^(-1/2)
    sqrt: SqrtResult
    trace_ps: float            # Tr(P S), the electron count (states)
    e_band: float              # Tr(P K)
    flops: int                 # every block product: square root, transforms, sign


def density_matrix_nonorth(K: bsr.Mat, S: bsr.Mat, mu: float, eps: float, tol: float, max_iter: int = 100,
                           order: int = 2, sqrt_tol: float | None = None) -> NonorthResult:
    """P = (1 - sign(S^-1 K - mu 1)) S^-1 / 2 (section "Sign-Method").

    Reading: sign(S^-1 K - mu 1) = S^(-1/2) sign(S^(-1/2) K S^(-1/2) - mu 1) S^(1/2) (a
    similarity), so P = S^(-1/2) P' S^(-1/2) with P' the orthogonal-basis density matrix of
    K' = S^(-1/2) K S^(-1/2); S^(-1/2) comes from inverse_sqrt.  Every product is filtered.
    Tr(P S) = Tr(P') and Tr(P K) = Tr(P' K')."""
    sq = inverse_sqrt(S, eps, sqrt_tol if sqrt_tol is not None else tol, max_iter, order=order)
    w = _Work(eps)
    Zs = sq.Sinvsqrt
    Kp = w(1.0, w(1.0, Zs, K), Zs)
    r = sign_iterate(Kp, mu, eps, tol, max_iter, order=order)
    P = w(1.0, w(1.0, Zs, r.P), Zs)
    return NonorthResult(P=P, sign=r, sqrt=sq, trace_ps=bsr.trace_product(P, S), e_band=bsr.trace_product(P, K),
                         flops=sq.flops + w.flops + r.flops)


# ------------------------------------------------------------------ Hotelling inverse
@dataclasses.dataclass
class InverseResult:
    Ainv: bsr.Mat
    iterations: int
    residuals: list            # ||A X - 1||_F / N per step
    converged: bool
    stalled: bool
    scale: float               # X_0 = 1 / g
    flops: int
    multiplies: int


def hotelling_inverse(A: bsr.Mat, eps: float, tol: float, max_iter: int = 100,
                      stall_ratio: float = 0.5) -> InverseResult:
    """A^-1 of a symmetric positive definite A by Hotelling's iteration (section
    "Preconditioners": X <- X (2 1 - A X), with aggressive filtering of the iterates).

    Readings: X_0 = 1 / g with g = max_i sum_j |A_ij| (so the spectrum of A X_0 lies in
    (0, 1] and the residual 1 - A X contracts); each step forms T = filter(A X), tests
    r = ||T - 1||_F / N, stops when r < tol, and otherwise sets X <- filter(2 X - X T).
    Since 1 - A X (2 - A X) = (1 - A X)^2, the residual squares at every unfiltered step.
    The stall test is the sign iteration's."""
    n = A.n
    g = gershgorin(A, 0.0)
    X = bsr.add_identity(identity_like(A), 1.0 / g, 0.0)
    w = _Work(eps)
    res = []
    converged = stalled = False
    it = 0
    while it < max_iter:
        T, inf = w(1.0, A, X, info=True)
        it += 1
        r = float(np.sqrt(inf.dev2)) / n
        res.append(r)
        if r < tol:
            converged = True
            break
        if len(res) >= 3 and res[-2] < stall_ratio * res[-3] and r > stall_ratio * res[-2]:
            stalled = True
            break
        X = w(-1.0, X, T, 2.0, X)                                # 2 X - X T
    return InverseResult(Ainv=X, iterations=it, residuals=res, converged=converged, stalled=stalled, scale=g,
                         flops=w.flops, multiplies=w.multiplies)
