"""Pins of the oracle's canonical purifications (TC2, TRS4) and of the sign method with a
bisected chemical potential (no GPU): the canonical projector from the eigendecomposition,
a diagonal H by brute force, TRS4's trace reset, invariance under a shift of H, and mu
inside the gap."""
import numpy as np
import pytest

import synth
from oracle import bsr, purify, sign


@pytest.fixture(scope="module")
def gapped():
    h = synth.build_hamiltonian(synth.small(10, seed=8080))
    return h, bsr.Mat.of(h.H)


def _projector(Hd, n_occ):
    w, Q = np.linalg.eigh(Hd)
    return Q[:, :n_occ] @ Q[:, :n_occ].T, w


@pytest.mark.parametrize("method", ["tc2", "trs4"])
def test_purification_gives_the_canonical_projector(gapped, method):
    h, H = gapped
    r = purify.purify(H, h.n_occ, eps=0.0, tol=1e-14, method=method)
    assert r.converged
    Pd, _ = _projector(bsr.to_dense(H), h.n_occ)
    P = bsr.to_dense(r.P)
    assert np.linalg.norm(P - Pd) / np.linalg.norm(Pd) < 1e-10
    assert np.linalg.norm(P @ P - P) < 1e-10
    assert r.trace_p == pytest.approx(h.n_occ, abs=1e-9)


@pytest.mark.parametrize("method", ["tc2", "trs4"])
def test_diagonal_h_by_brute_force(method):
    # 1x1 blocks: every step acts on each diagonal entry; the canonical projector occupies
    # the n_occ smallest entries
    rng = np.random.default_rng(3)
    d = np.concatenate([rng.uniform(-2.0, -0.3, 7), rng.uniform(0.4, 2.0, 9)])
    rng.shuffle(d)
    D = np.diag(d)
    H = bsr.from_dense(D, [1] * d.shape[0])
    r = purify.purify(H, 7, eps=0.0, tol=1e-14, method=method)
    occ = np.zeros_like(d)
    occ[np.argsort(d)[:7]] = 1.0
    assert np.allclose(np.diag(bsr.to_dense(r.P)), occ, atol=1e-10)


def test_trs4_steps_reset_the_trace(gapped):
    # gamma is chosen so that Tr(F + gamma G) = N_occ: after every such step the trace is exact
    h, H = gapped
    prev = None
    seen = 0
    for k in range(1, 12):
        r = purify.purify(H, h.n_occ, eps=0.0, tol=1e-300, method="trs4", max_iter=k)
        if prev is not None and r.steps["trs4"] > prev:
            assert r.trace_p == pytest.approx(h.n_occ, abs=1e-9)
            seen += 1
        prev = r.steps["trs4"]
    assert seen >= 3


@pytest.mark.parametrize("method", ["tc2", "trs4"])
def test_a_shift_of_h_leaves_the_canonical_projector(gapped, method):
    h, H = gapped
    a = purify.purify(H, h.n_occ, eps=0.0, tol=1e-13, method=method)
    b = purify.purify(bsr.add_identity(H, 1.0, 0.37), h.n_occ, eps=0.0, tol=1e-13, method=method)
    assert np.linalg.norm(bsr.to_dense(a.P) - bsr.to_dense(b.P)) < 1e-9


@pytest.mark.parametrize("method", ["tc2", "trs4"])
def test_filtered_purification_agrees_with_the_sign_method(gapped, method):
    h, H = gapped
    s = sign.sign_iterate(H, 0.0, 1e-7, 1e-9)
    r = purify.purify(H, h.n_occ, eps=1e-7, tol=1e-9, method=method)
    assert r.converged
    assert abs(r.e_band - s.e_band) / h.n_atoms < 1e-7
    assert r.trace_p == pytest.approx(h.n_occ, abs=1e-5)


def test_tc2_takes_one_product_per_step_and_trs4_at_most_two(gapped):
    h, H = gapped
    a = purify.purify(H, h.n_occ, eps=1e-7, tol=1e-9, method="tc2")
    assert a.multiplies == a.iterations
    b = purify.purify(H, h.n_occ, eps=1e-7, tol=1e-9, method="trs4")
    assert b.multiplies == b.iterations + b.steps["trs4"]


def test_mu_search_lands_in_the_gap(gapped):
    h, H = gapped
    for shift in (0.0, 1.0, -1.1):
        Hs = bsr.add_identity(H, 1.0, shift)
        m = purify.mu_search(Hs, h.n_occ, 0.0, 1e-12)
        _, w = _projector(bsr.to_dense(Hs), h.n_occ)
        assert w[h.n_occ - 1] < m.mu < w[h.n_occ]
        assert m.result.trace_p == pytest.approx(h.n_occ, abs=1e-8)
        g = sign.gershgorin(Hs, 0.0)
        assert m.evaluations <= int(np.ceil(np.log2(2 * g / (w[h.n_occ] - w[h.n_occ - 1])))) + 1
        # the bisection's trials: below the gap too few states, above too many
        for mu, t in zip(m.mus[:-1], m.traces[:-1]):
            assert (t < h.n_occ) == (mu < w[h.n_occ - 1])
