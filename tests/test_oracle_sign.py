"""Pins of the oracle's sign iteration: dense eigendecomposition, the scalar
Newton-Schulz recurrence on the eigenvalues, closed forms and invariants (no GPU)."""
import numpy as np
import pytest

import synth
from oracle import bsr, sign


def _eigh_sign(D, mu=0.0):
    w, Q = np.linalg.eigh(D - mu * np.eye(D.shape[0]))
    return Q @ np.diag(np.sign(w)) @ Q.T, w


@pytest.fixture(scope="module")
def small_h():
    w = synth.small(12, seed=9001)
    return synth.build_hamiltonian(w)


def test_sign_matches_dense_eigh(small_h):
    H = bsr.Mat.of(small_h.H)
    r = sign.sign_iterate(H, 0.0, eps=0.0, tol=1e-13)
    assert r.converged
    S, _ = _eigh_sign(bsr.to_dense(H))
    X = bsr.to_dense(r.X)
    assert np.linalg.norm(X - S) / np.linalg.norm(S) < 1e-12
    # band energy against the dense definition Tr(P H)
    P = 0.5 * (np.eye(H.n) - S)
    assert r.e_band == pytest.approx(np.trace(P @ bsr.to_dense(H)), abs=1e-10)


def test_residuals_follow_scalar_recurrence(small_h):
    # with eps = 0, X_k = Q f^k(Lambda / alpha) Q^T with f(x) = x (3 - x^2) / 2, so
    # r_k = ||X_k^2 - 1||_F / N is fixed by the eigenvalues alone
    H = bsr.Mat.of(small_h.H)
    r = sign.sign_iterate(H, 0.0, eps=0.0, tol=1e-14)
    D = bsr.to_dense(H)
    alpha = np.abs(D).sum(axis=1).max()
    assert r.alpha == pytest.approx(alpha, rel=1e-14)
    x = np.linalg.eigvalsh(D) / alpha
    for k, rk in enumerate(r.residuals):
        expect = np.sqrt(np.sum((x * x - 1.0) ** 2)) / H.n
        assert rk == pytest.approx(expect, rel=1e-9, abs=1e-14), k
        x = 0.5 * x * (3.0 - x * x)


def test_invariants_of_converged_density_matrix(small_h):
    H = bsr.Mat.of(small_h.H)
    r = sign.sign_iterate(H, 0.0, eps=1e-9, tol=1e-10)
    assert r.converged and not r.stalled
    X, P, Hd = bsr.to_dense(r.X), bsr.to_dense(r.P), bsr.to_dense(H)
    n = H.n
    assert np.linalg.norm(X @ X - np.eye(n)) < 1e-6
    assert np.linalg.norm(P @ P - P) < 1e-6
    assert np.linalg.norm(P @ Hd - Hd @ P) < 1e-6
    assert r.trace_p == pytest.approx(small_h.n_occ, abs=1e-6)     # 4 per molecule


def test_band_energy_invariant_for_mu_in_gap(small_h):
    H = bsr.Mat.of(small_h.H)
    es = [sign.sign_iterate(H, mu, eps=0.0, tol=1e-12).e_band for mu in (-0.2, 0.0, 0.15)]
    assert max(es) - min(es) < 1e-9


def test_diagonal_matrix_gives_elementwise_sign():
    d = np.array([0.9, -0.3, 1.7, -1.1, 0.4, -0.8])
    H = bsr.from_dense(np.diag(d), [2, 1, 3])
    r = sign.sign_iterate(H, 0.0, eps=0.0, tol=1e-14)
    np.testing.assert_allclose(bsr.to_dense(r.X), np.diag(np.sign(d)), atol=1e-13)


def test_two_by_two_closed_form():
    # symmetric [[a, b], [b, d]] with eigenvalues of both signs:
    # sign = (2A - tr(A) 1) / sqrt((a - d)^2 + 4 b^2)
    a, b, d = 0.3, 0.8, -0.5
    A = np.array([[a, b], [b, d]])
    expect = (2 * A - (a + d) * np.eye(2)) / np.sqrt((a - d) ** 2 + 4 * b * b)
    for bs in ([2], [1, 1]):
        r = sign.sign_iterate(bsr.from_dense(A, bs), 0.0, eps=0.0, tol=1e-14)
        np.testing.assert_allclose(bsr.to_dense(r.X), expect, atol=1e-13)


def test_scale_and_negation_symmetry(small_h):
    H = bsr.Mat.of(small_h.H)
    X1 = bsr.to_dense(sign.sign_iterate(H, 0.0, 0.0, 1e-13).X)
    H3 = H.copy()
    H3.data *= 3.0
    X3 = bsr.to_dense(sign.sign_iterate(H3, 0.0, 0.0, 1e-13).X)
    Hn = H.copy()
    Hn.data *= -1.0
    Xn = bsr.to_dense(sign.sign_iterate(Hn, 0.0, 0.0, 1e-13).X)
    assert np.abs(X1 - X3).max() < 1e-11
    assert np.abs(X1 + Xn).max() < 1e-11


def test_block_diagonal_is_independent():
    # molecules in a box so large that no inter-molecular pair is within 8 A:
    # the sign is the direct sum of the per-molecule signs
    w = synth.small(3, seed=31)
    h = synth.build_hamiltonian(w, box=60.0)
    H = bsr.Mat.of(h.H)
    assert H.nnzb == 27
    X = bsr.to_dense(sign.sign_iterate(H, 0.0, 0.0, 1e-13).X)
    D = bsr.to_dense(H)
    for m in range(3):
        s = slice(23 * m, 23 * (m + 1))
        S, _ = _eigh_sign(D[s, s])
        np.testing.assert_allclose(X[s, s], S, atol=1e-12)
    off = X.copy()
    for m in range(3):
        off[23 * m:23 * (m + 1), 23 * m:23 * (m + 1)] = 0
    assert np.abs(off).max() == 0.0


def test_filtering_error_is_small(small_h):
    H = bsr.Mat.of(small_h.H)
    exact = sign.sign_iterate(H, 0.0, 0.0, 1e-12)
    # the filtered fixed point keeps ||X^2 - 1||_F ~ 1e-6 here (N = 276), so r floors near 5e-9
    filt = sign.sign_iterate(H, 0.0, 1e-7, 2e-8)
    assert filt.converged
    assert abs(exact.e_band - filt.e_band) / (3 * 12) < 1e-6
    assert sum(filt.nnzb_history) <= sum(exact.nnzb_history)


def test_stall_is_reported():
    # eps so large that the filter destroys the iteration: it must stop, not loop forever
    w = synth.small(12, seed=9001)
    H = bsr.Mat.of(synth.build_hamiltonian(w).H)
    r = sign.sign_iterate(H, 0.0, eps=0.05, tol=1e-14, max_iter=60)
    assert not r.converged
    assert r.stalled or r.iterations == 60


@pytest.mark.parametrize("order", [2, 3])
def test_prescreened_iteration_is_the_same_bit_for_bit(order):
    # the prescreen leaves every filtered product unchanged, so the whole iteration too, with
    # fewer block products
    h = synth.build_hamiltonian(synth.small(32, basis=(23, 7), seed=8601, eps=1e-4, tol=1e-7))
    H = bsr.Mat.of(h.H)
    a = sign.sign_iterate(H, h.mu, 1e-4, 1e-7, order=order)
    b = sign.sign_iterate(H, h.mu, 1e-4, 1e-7, order=order, prescreen=True)
    assert a.residuals == b.residuals and a.iterations == b.iterations
    assert np.array_equal(a.P.col, b.P.col) and np.array_equal(a.P.data, b.P.data)
    assert a.e_band == b.e_band
    assert b.n_products < a.n_products and b.flops < a.flops
