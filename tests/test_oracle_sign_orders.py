"""Pins of the oracle's higher-order sign iterations and of its block-sparse add (no GPU):
the step polynomials the paper prints, the order of convergence and the limit of the
series behind them, the exact eigenvalue map of one step, the four products per
fifth-order iteration, and the add against dense arithmetic."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle import bsr, sign

HERE = os.path.dirname(os.path.abspath(__file__))


def _printed():
    """{order: (denominator, [coefficients])} from tests/golden/sign_orders.txt."""
    out = {}
    with open(os.path.join(HERE, "golden", "sign_orders.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                v = [int(t) for t in line.split()]
                out[v[0]] = (v[1], v[2:])
    return out


def test_coefficients_equal_the_printed_polynomials():
    printed = _printed()
    assert sorted(printed) == [2, 3, 4, 5]
    for order, (den, coef) in printed.items():
        got = sign.pade_coefficients(order)
        assert got == [Fraction(c, den) for c in coef], order


@pytest.mark.parametrize("order", range(2, 8))
def test_step_has_the_stated_order(order):
    # x p(x^2) with e = 1 - x^2: exactly, 1 - (x p(x^2))^2 = 2 c_o e^o + O(e^(o+1)), where
    # c_o = binom(2o, o) / 4^o is the first dropped term of (1 - e)^(-1/2).  A wrong
    # coefficient anywhere leaves a lower power of e.
    a = sign.pade_coefficients(order)
    c_next = Fraction(math.comb(2 * order, order), 4 ** order)
    for e in (Fraction(1, 10 ** 4), Fraction(1, 10 ** 6)):
        y = 1 - e
        p = sum(ai * y ** i for i, ai in enumerate(a))
        e_new = 1 - y * p * p
        assert abs(e_new / e ** order / (2 * c_next) - 1) < 20 * e * order


@pytest.mark.parametrize("order", range(2, 8))
def test_polynomial_stays_below_the_inverse_square_root(order):
    # the dropped terms of (1 - z)^(-1/2) are all positive: 0 < y^(-1/2) - p(y) on (0, 1),
    # and more terms come closer
    a = [float(v) for v in sign.pade_coefficients(order)]
    b = [float(v) for v in sign.pade_coefficients(order + 1)] if order < 7 else None
    y = np.linspace(0.01, 0.99, 99)
    p = np.polyval(a[::-1], y)
    assert np.all(p < y ** -0.5)
    if b is not None:
        assert np.all(np.polyval(b[::-1], y) > p)


@pytest.mark.parametrize("order", range(2, 8))
def test_residual_ratio_grows_with_the_residual(order):
    # premise of the stall test for every order: per eigenvalue e'/e is increasing in e
    # (exact rational arithmetic: near e = 0 the ratio is far below double rounding)
    a = sign.pade_coefficients(order)
    g = []
    for k in range(1, 400):
        e = Fraction(k, 400)
        y = 1 - e
        p = sum(ai * y ** i for i, ai in enumerate(a))
        g.append((1 - y * p * p) / e)
    assert all(g1 > g0 for g0, g1 in zip(g, g[1:]))


@pytest.fixture(scope="module")
def small_h():
    return synth.build_hamiltonian(synth.small(10, seed=5150))


@pytest.mark.parametrize("order", range(2, 8))
def test_one_step_is_the_eigenvalue_map(small_h, order):
    # eps = 0: X_1 = Q diag(x p(x^2)) Q^T for X_0 = Q diag(x) Q^T; orders 2-5 evaluate p
    # from the printed polynomials, 6 and 7 from the pinned coefficients
    H = bsr.Mat.of(small_h.H)
    r = sign.sign_iterate(H, 0.0, eps=0.0, tol=1e-300, max_iter=1, order=order)
    X0 = bsr.to_dense(H) / r.alpha
    x, Q = np.linalg.eigh(X0)
    printed = _printed()
    if order in printed:
        den, coef = printed[order]
        p = np.polyval(np.array(coef[::-1], dtype=float), x * x) / den
    else:
        p = np.polyval(np.array([float(v) for v in sign.pade_coefficients(order)])[::-1], x * x)
    X1 = Q @ np.diag(x * p) @ Q.T
    assert np.linalg.norm(bsr.to_dense(r.X) - X1) / np.linalg.norm(X1) < 1e-13


@pytest.mark.parametrize("order", range(2, 8))
def test_every_order_converges_to_the_dense_sign(small_h, order):
    H = bsr.Mat.of(small_h.H)
    r = sign.sign_iterate(H, 0.0, eps=0.0, tol=1e-13, order=order)
    assert r.converged and not r.stalled
    D = bsr.to_dense(H)
    w, Q = np.linalg.eigh(D)
    S = Q @ np.diag(np.sign(w)) @ Q.T
    assert np.linalg.norm(bsr.to_dense(r.X) - S) / np.linalg.norm(S) < 1e-12
    P = bsr.to_dense(r.P)
    assert np.linalg.norm(P @ P - P) < 1e-10
    assert r.trace_p == pytest.approx(small_h.n_occ, abs=1e-9)


def test_higher_orders_take_fewer_iterations_and_the_stated_products(small_h):
    H = bsr.Mat.of(small_h.H)
    per_iter = {2: 2, 3: 3, 4: 4, 5: 4, 6: 5, 7: 5}
    its = {}
    for order, k in per_iter.items():
        r = sign.sign_iterate(H, 0.0, eps=1e-7, tol=1e-9, order=order)
        assert r.converged
        # every iteration but the last (which only forms X X and stops) takes k products;
        # the fifth order takes the paper's four
        assert r.multiplies == k * (r.iterations - 1) + 1
        its[order] = r.iterations
    assert its[2] > its[3] >= its[5] >= its[7]


def test_filtered_higher_order_energy_agrees_with_newton_schulz(small_h):
    H = bsr.Mat.of(small_h.H)
    e2 = sign.sign_iterate(H, 0.0, eps=1e-7, tol=1e-9).e_band
    for order in (3, 5, 7):
        e = sign.sign_iterate(H, 0.0, eps=1e-7, tol=1e-9, order=order).e_band
        assert abs(e - e2) / small_h.n_atoms < 1e-7


def test_bad_order_is_refused(small_h):
    with pytest.raises(ValueError):
        sign.sign_iterate(bsr.Mat.of(small_h.H), 0.0, 0.0, 1e-9, order=8)


def _rand_mat(bs, density, seed):
    return bsr.Mat.of(synth.random_block_matrix(bs, density, seed))


@pytest.mark.parametrize("alpha,beta", [(1.0, 1.0), (0.75, -1.40625), (-2.5, 0.3)])
def test_add_equals_dense_sum_on_the_union(alpha, beta):
    bs = [13, 5, 5, 23, 7, 7] * 3
    A = _rand_mat(bs, 0.3, 1)
    B = _rand_mat(bs, 0.4, 2)
    C = bsr.add(alpha, A, beta, B)
    # same elementwise arithmetic as alpha*a + beta*b on the dense arrays (a missing
    # block is zero there, and alpha*a + 0 = alpha*a)
    assert np.array_equal(bsr.to_dense(C), alpha * bsr.to_dense(A) + beta * bsr.to_dense(B))
    pa = set(zip(A.rows.tolist(), A.col.tolist()))
    pb = set(zip(B.rows.tolist(), B.col.tolist()))
    assert set(zip(C.rows.tolist(), C.col.tolist())) == pa | pb
    assert all(np.all(np.diff(C.col[C.rp[i]:C.rp[i + 1]]) > 0) for i in range(C.nblk))


def test_add_edge_cases():
    bs = [13, 5, 5] * 4
    A = _rand_mat(bs, 0.5, 3)
    empty = bsr.Mat(np.array(bs), np.zeros(len(bs) + 1, dtype=np.int64), np.zeros(0, dtype=np.int32), np.zeros(0))
    assert np.array_equal(bsr.add(2.0, A, 3.0, empty).data, 2.0 * A.data)
    assert np.array_equal(bsr.add(2.0, empty, 3.0, A).data, 3.0 * A.data)
    assert bsr.add(1.0, empty, 1.0, empty).nnzb == 0
    same = bsr.add(0.5, A, 0.25, A)
    assert np.array_equal(same.col, A.col) and np.array_equal(same.data, 0.5 * A.data + 0.25 * A.data)
    with pytest.raises(ValueError):
        bsr.add(1.0, A, 1.0, _rand_mat([13, 5] * 6, 0.5, 4))
