"""Pins of the oracle's non-orthogonal path (no GPU): the inverse square root from the
sign of the block matrix [[0, A], [1, 0]] (section "Sign-Method"), checked against the
sign of that matrix and against the eigendecomposition, and the density matrix
P = (1 - sign(S^-1 K - mu 1)) S^-1 / 2 against the paper's formula evaluated densely and
against the generalized eigenproblem K c = S c e."""
import os

import numpy as np
import pytest
import scipy.linalg as sl

import synth
from oracle import bsr, sign

HERE = os.path.dirname(os.path.abspath(__file__))


def _printed_poly(order):
    with open(os.path.join(HERE, "golden", "sign_orders.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                v = [int(t) for t in line.split()]
                if v[0] == order:
                    return v[1], v[2:]
    raise KeyError(order)


@pytest.fixture(scope="module")
def system():
    w = synth.small(8, seed=6060)
    h = synth.build_hamiltonian(w)
    S = bsr.Mat.of(synth.build_overlap(w))
    return h, bsr.Mat.of(h.H), S


def test_overlap_is_symmetric_positive_definite_and_keeps_the_gap(system):
    h, K, S = system
    Sd = bsr.to_dense(S)
    assert np.array_equal(Sd, Sd.T)
    ev = np.linalg.eigvalsh(Sd)
    assert 0.1 <= ev[0] and ev[-1] <= 1.9                 # the generator's Gershgorin bound
    e = sl.eigh(bsr.to_dense(K), Sd, eigvals_only=True)
    assert int((e < 0).sum()) == h.n_occ                  # Sylvester: same occupied count at mu = 0
    assert e[e < 0].max() < -0.13 and e[e > 0].min() > 0.13


def test_block_sign_identity_and_converged_roots(system):
    _, _, S = system
    Sd = bsr.to_dense(S)
    n = Sd.shape[0]
    M = np.block([[np.zeros((n, n)), Sd], [np.eye(n), np.zeros((n, n))]])
    sgn = sl.signm(M)
    w, Q = np.linalg.eigh(Sd)
    root = Q @ np.diag(np.sqrt(w)) @ Q.T
    iroot = Q @ np.diag(1 / np.sqrt(w)) @ Q.T
    # the relation the paper states
    assert np.allclose(sgn[:n, n:], root, atol=1e-9) and np.allclose(sgn[n:, :n], iroot, atol=1e-9)
    assert np.allclose(sgn[:n, :n], 0, atol=1e-9) and np.allclose(sgn[n:, n:], 0, atol=1e-9)
    for order in (2, 3, 5, 7):
        r = sign.inverse_sqrt(S, eps=0.0, tol=1e-13, order=order)
        assert r.converged
        Z, Y = bsr.to_dense(r.Sinvsqrt), bsr.to_dense(r.Ssqrt)
        assert np.linalg.norm(Z - iroot) / np.linalg.norm(iroot) < 1e-12
        assert np.linalg.norm(Y - root) / np.linalg.norm(root) < 1e-12
        assert np.linalg.norm(Z @ Sd @ Z - np.eye(n)) < 1e-11
        assert np.linalg.norm(Y @ Z - np.eye(n)) < 1e-11


@pytest.mark.parametrize("order", [2, 3, 4, 5])
def test_one_coupled_step_is_one_sign_step_on_the_block_matrix(system, order):
    # X_1 = X_0 p(X_0^2) for X_0 = [[0, S/g], [1, 0]], p the printed step polynomial
    _, _, S = system
    Sd = bsr.to_dense(S)
    n = Sd.shape[0]
    r = sign.inverse_sqrt(S, eps=0.0, tol=1e-300, max_iter=1, order=order)
    g = r.scale
    X0 = np.block([[np.zeros((n, n)), Sd / g], [np.eye(n), np.zeros((n, n))]])
    den, coef = _printed_poly(order)
    X2 = X0 @ X0
    P = sum(c * np.linalg.matrix_power(X2, i) for i, c in enumerate(coef)) / den
    X1 = X0 @ P
    assert np.allclose(X1[:n, :n], 0) and np.allclose(X1[n:, n:], 0)
    Y1 = bsr.to_dense(r.Ssqrt) / np.sqrt(g)
    Z1 = bsr.to_dense(r.Sinvsqrt) * np.sqrt(g)
    assert np.linalg.norm(Y1 - X1[:n, n:]) / np.linalg.norm(X1[:n, n:]) < 1e-13
    assert np.linalg.norm(Z1 - X1[n:, :n]) / np.linalg.norm(X1[n:, :n]) < 1e-13


def test_density_matrix_equals_the_paper_formula_and_the_generalized_eigenproblem(system):
    h, K, S = system
    Kd, Sd = bsr.to_dense(K), bsr.to_dense(S)
    n = Kd.shape[0]
    r = sign.density_matrix_nonorth(K, S, 0.0, eps=0.0, tol=1e-13)
    assert r.sign.converged and r.sqrt.converged
    P = bsr.to_dense(r.P)
    # the printed formula, with a dense sign of the non-symmetric S^-1 K
    Si = np.linalg.inv(Sd)
    Pf = 0.5 * (np.eye(n) - sl.signm(Si @ Kd)) @ Si
    assert np.linalg.norm(P - Pf) / np.linalg.norm(Pf) < 1e-10
    # occupied generalized eigenvectors (C^T S C = 1): P = C_occ C_occ^T
    e, C = sl.eigh(Kd, Sd)
    occ = e < 0
    Pe = C[:, occ] @ C[:, occ].T
    assert np.linalg.norm(P - Pe) / np.linalg.norm(Pe) < 1e-10
    assert np.linalg.norm(P @ Sd @ P - P) < 1e-10
    assert r.trace_ps == pytest.approx(h.n_occ, abs=1e-9)
    assert r.e_band == pytest.approx(e[occ].sum(), abs=1e-9)


def test_identity_overlap_reduces_to_the_orthogonal_iteration(system):
    h, K, S = system
    I = sign.identity_like(S)
    r = sign.density_matrix_nonorth(K, I, 0.0, eps=1e-7, tol=1e-9)
    o = sign.sign_iterate(K, 0.0, eps=1e-7, tol=1e-9)
    assert r.sqrt.iterations == 1                           # Z Y = 1 at once
    assert np.linalg.norm(bsr.to_dense(r.P) - bsr.to_dense(o.P)) < 1e-12
    assert r.e_band == pytest.approx(o.e_band, abs=1e-12)


@pytest.mark.parametrize("order", [2, 5])
def test_filtered_density_matrix_energy(system, order):
    h, K, S = system
    e, C = sl.eigh(bsr.to_dense(K), bsr.to_dense(S))
    r = sign.density_matrix_nonorth(K, S, 0.0, eps=1e-7, tol=1e-9, order=order)
    assert r.sign.converged or r.sign.stalled
    assert abs(r.e_band - e[e < 0].sum()) / h.n_atoms < 1e-6
    assert r.trace_ps == pytest.approx(h.n_occ, abs=1e-5)


def test_hotelling_inverse(system):
    _, _, S = system
    Sd = bsr.to_dense(S)
    n = Sd.shape[0]
    r = sign.hotelling_inverse(S, eps=0.0, tol=1e-13)
    assert r.converged
    assert np.linalg.norm(bsr.to_dense(r.Ainv) - np.linalg.inv(Sd)) / np.linalg.norm(np.linalg.inv(Sd)) < 1e-12
    # the residual squares exactly: 1 - S X_1 = (1 - S X_0)^2 with X_0 = 1 / g
    one = sign.hotelling_inverse(S, eps=0.0, tol=1e-300, max_iter=2)
    R0 = np.eye(n) - Sd / one.scale
    assert one.residuals[0] == pytest.approx(np.linalg.norm(R0) / n, rel=1e-12)
    assert one.residuals[1] == pytest.approx(np.linalg.norm(R0 @ R0) / n, rel=1e-10)
    # two products per step, the last step forms S X only
    assert r.multiplies == 2 * r.iterations - 1
    # and S^-1 = (S^-1/2)^2
    q = sign.inverse_sqrt(S, eps=0.0, tol=1e-13)
    Z = bsr.to_dense(q.Sinvsqrt)
    assert np.linalg.norm(Z @ Z - bsr.to_dense(r.Ainv)) / np.linalg.norm(Z @ Z) < 1e-11
