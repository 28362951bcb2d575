"""Mistakes planted in the oracle (on the CPU) must fail its pins: the pins of the
higher-order steps, the coupled square root and the non-orthogonal density matrix are
evaluated with a dropped term, a flipped sign, a wrong factor and swapped roots."""
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sl

import synth
from oracle import bsr, sign

HERE = os.path.dirname(os.path.abspath(__file__))


def _printed(order):
    with open(os.path.join(HERE, "golden", "sign_orders.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                v = [int(t) for t in line.split()]
                if v[0] == order:
                    return v[1], v[2:]


@pytest.fixture(scope="module")
def system():
    w = synth.small(6, seed=606)
    h = synth.build_hamiltonian(w)
    return h, bsr.Mat.of(h.H), bsr.Mat.of(synth.build_overlap(w))


def _eigen_map_error(H, order):
    """The pin of one unfiltered step against the printed polynomial's eigenvalue map."""
    r = sign.sign_iterate(H, 0.0, eps=0.0, tol=1e-300, max_iter=1, order=order)
    x, Q = np.linalg.eigh(bsr.to_dense(H) / r.alpha)
    den, coef = _printed(order)
    X1 = Q @ np.diag(x * np.polyval(np.array(coef[::-1], float), x * x) / den) @ Q.T
    return np.linalg.norm(bsr.to_dense(r.X) - X1) / np.linalg.norm(X1)


@pytest.mark.parametrize("plant", ["drop_last_term", "flip_first_order_sign"])
@pytest.mark.parametrize("order", [3, 5])
def test_step_polynomial_mistakes_fail_the_eigen_map_pin(system, monkeypatch, plant, order):
    _, H, _ = system
    assert _eigen_map_error(H, order) < 1e-13
    good = sign.series_coefficients

    def bad(o):
        c = list(good(o))
        if plant == "drop_last_term":
            c[-1] = Fraction(0)
        else:
            c[1] = -c[1]
        return c

    monkeypatch.setattr(sign, "series_coefficients", bad)
    assert _eigen_map_error(H, order) > 1e-4


def _coupled_step_error(S, order):
    """The pin of one coupled square-root step against one dense step on [[0, A], [1, 0]]."""
    Sd = bsr.to_dense(S)
    n = Sd.shape[0]
    r = sign.inverse_sqrt(S, eps=0.0, tol=1e-300, max_iter=1, order=order)
    X0 = np.block([[np.zeros((n, n)), Sd / r.scale], [np.eye(n), np.zeros((n, n))]])
    den, coef = _printed(order)
    X2 = X0 @ X0
    X1 = X0 @ (sum(c * np.linalg.matrix_power(X2, i) for i, c in enumerate(coef)) / den)
    Y1 = bsr.to_dense(r.Ssqrt) / np.sqrt(r.scale)
    return np.linalg.norm(Y1 - X1[:n, n:]) / np.linalg.norm(X1[:n, n:])


def test_a_wrong_factor_in_the_coupled_step_fails_its_pin(system, monkeypatch):
    _, _, S = system
    assert _coupled_step_error(S, 2) < 1e-13
    # plant: U = W (the square) instead of p(W)
    monkeypatch.setattr(sign, "_step_polynomial", lambda W, order, eps, mult: W)
    assert _coupled_step_error(S, 2) > 1e-3


def _nonorth_error(h, K, S):
    """The pin of P against the generalized eigenproblem K c = S c e."""
    e, C = sl.eigh(bsr.to_dense(K), bsr.to_dense(S))
    Pe = C[:, e < 0] @ C[:, e < 0].T
    r = sign.density_matrix_nonorth(K, S, 0.0, eps=0.0, tol=1e-13)
    return np.linalg.norm(bsr.to_dense(r.P) - Pe) / np.linalg.norm(Pe)


def test_swapped_square_roots_fail_the_generalized_eigenproblem_pin(system, monkeypatch):
    h, K, S = system
    assert _nonorth_error(h, K, S) < 1e-10
    good = sign.inverse_sqrt

    def swapped(*a, **k):
        r = good(*a, **k)
        r.Sinvsqrt, r.Ssqrt = r.Ssqrt, r.Sinvsqrt
        return r

    monkeypatch.setattr(sign, "inverse_sqrt", swapped)
    assert _nonorth_error(h, K, S) > 1e-2


class _FlippedTrace:
    """bsr with Tr(X) reflected about n_occ, so that every trace comparison turns around."""

    def __init__(self, n_occ):
        from oracle import bsr as real
        self._real, self._n = real, n_occ

    def __getattr__(self, name):
        return getattr(self._real, name)

    def trace(self, M):
        return 2 * self._n - self._real.trace(M)


def _projector_error(h, H, method):
    from oracle import purify
    w, Q = np.linalg.eigh(bsr.to_dense(H))
    Pe = Q[:, :h.n_occ] @ Q[:, :h.n_occ].T
    r = purify.purify(H, h.n_occ, eps=0.0, tol=1e-13, method=method, max_iter=60)
    return np.linalg.norm(bsr.to_dense(r.P) - Pe) / np.linalg.norm(Pe)


def test_an_inverted_tc2_branch_fails_the_projector_pin(system, monkeypatch):
    from oracle import purify
    h, H, _ = system
    assert _projector_error(h, H, "tc2") < 1e-10
    monkeypatch.setattr(purify, "bsr", _FlippedTrace(h.n_occ))
    assert _projector_error(h, H, "tc2") > 1e-2


def test_a_reversed_bisection_fails_the_gap_pin(system, monkeypatch):
    from oracle import purify
    h, H, _ = system
    Hs = bsr.add_identity(H, 1.0, 1.0)                      # the gap away from the interval's middle
    w = np.linalg.eigvalsh(bsr.to_dense(Hs))
    in_gap = lambda mu: w[h.n_occ - 1] < mu < w[h.n_occ]   # noqa: E731
    assert in_gap(purify.mu_search(Hs, h.n_occ, 0.0, 1e-12).mu)
    real = sign.sign_iterate

    def reflected(*a, **k):
        r = real(*a, **k)
        r.trace_p = 2 * h.n_occ - r.trace_p
        return r

    monkeypatch.setattr(purify.sign, "sign_iterate", reflected)
    assert not in_gap(purify.mu_search(Hs, h.n_occ, 0.0, 1e-12, max_eval=12).mu)
