"""GPU parity of the canonical purifications (dbcsr_purify: TC2, TRS4) and of the sign
method with a bisected chemical potential (dbcsr_sign_mu_search) against the FP64 oracle."""
import numpy as np
import pytest

import synth
from oracle import bsr, purify, sign

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2003_03868_gb300 as m
    m.lib()
    return m


def _mat(M):
    rp, col, data = M.export()
    return bsr.Mat(M.blk_size, rp, col, data)


def _gpu(gb, M):
    return gb.Matrix.of(synth.BlockMatrix(M.bs, M.rp, M.col, M.data))


@pytest.mark.parametrize("method", ["tc2", "trs4"])
@pytest.mark.parametrize("n_mol,basis,eps,tol", [(8, (13, 5), 0.0, 1e-12), (24, (13, 5), 1e-7, 1e-9),
                                                 (16, (23, 7), 1e-6, 1e-8)])
def test_purification_matches_oracle(gb, method, n_mol, basis, eps, tol):
    h = synth.build_hamiltonian(synth.small(n_mol, basis=basis, seed=4040 + n_mol))
    o = purify.purify(bsr.Mat.of(h.H), h.n_occ, eps, tol, method=method)
    assert o.converged
    H = gb.Matrix.of(h.H)
    f = gb.purify(H, h.n_occ, eps, tol, method=method, full_products=True)
    assert f.converged
    assert f.report.alpha == pytest.approx(o.scale, rel=1e-15)
    # Near the end TRS4's gamma = (N - Tr F) / Tr G divides rounding noise by Tr G -> 0, so
    # the last step may take another (equally valid) branch and one more step; the two runs
    # agree step for step while the idempotency measure is well above rounding
    assert abs(f.report.iterations - o.iterations) <= (1 if method == "trs4" else 0)
    hist = [f.report.residual_history[i] for i in range(f.report.iterations + 1)]
    big = [i for i, e in enumerate(o.idempotency) if abs(e) > 1e-9 and i < len(hist)]
    np.testing.assert_allclose([hist[i] for i in big], [o.idempotency[i] for i in big], rtol=1e-6)
    assert abs(f.report.e_band - o.e_band) / h.n_atoms < 1e-10
    assert f.report.trace_p == pytest.approx(o.trace_p, abs=1e-8)
    P = _mat(f.P)
    if np.array_equal(P.col, o.P.col):
        assert np.linalg.norm(P.data - o.P.data) / np.linalg.norm(o.P.data) < max(1e-9, 10 * eps)
    # default: mirrored products
    g = gb.purify(H, h.n_occ, eps, tol, method=method)
    assert g.converged
    assert abs(g.report.iterations - o.iterations) <= 1
    assert abs(g.report.e_band - o.e_band) / h.n_atoms < max(1e-10, 0.1 * eps)
    D = bsr.to_dense(_mat(g.P))
    assert np.array_equal(D, D.T)


@pytest.mark.parametrize("method", ["tc2", "trs4"])
def test_purification_against_eigh(gb, method):
    h = synth.build_hamiltonian(synth.small(10, seed=123))
    Hd = bsr.to_dense(bsr.Mat.of(h.H))
    w, Q = np.linalg.eigh(Hd)
    Pd = Q[:, :h.n_occ] @ Q[:, :h.n_occ].T
    g = gb.purify(gb.Matrix.of(h.H), h.n_occ, 0.0, 1e-13, method=method)
    P = bsr.to_dense(_mat(g.P))
    assert np.linalg.norm(P - Pd) / np.linalg.norm(Pd) < 1e-10


@pytest.mark.parametrize("shift", [0.0, 1.0, -1.1])
def test_mu_search_matches_oracle(gb, shift):
    h = synth.build_hamiltonian(synth.small(12, seed=5050))
    Ho = bsr.add_identity(bsr.Mat.of(h.H), 1.0, shift)
    o = purify.mu_search(Ho, h.n_occ, 1e-7, 1e-9)
    g = gb.sign_mu_search(_gpu(gb, Ho), h.n_occ, 1e-7, 1e-9)
    assert g.evaluations == o.evaluations
    assert g.mu == pytest.approx(o.mu, rel=1e-12, abs=1e-14)
    assert g.report.trace_p == pytest.approx(h.n_occ, abs=1e-5)
    assert abs(g.report.e_band - o.result.e_band) / h.n_atoms < 1e-8
    w = np.linalg.eigvalsh(bsr.to_dense(Ho))
    assert w[h.n_occ - 1] < g.mu < w[h.n_occ]


def test_purify_arguments_are_checked(gb):
    h = synth.build_hamiltonian(synth.small(6, seed=7))
    H = gb.Matrix.of(h.H)
    P = gb.Matrix(H.blk_size, H.stream)
    o = gb.SignOpts(0.0, 1e-9, 10, gb.DBCSR_FP64, 0.0, 0.0, 0, 0, 0, 0)
    import ctypes as C
    assert gb.lib().dbcsr_purify(H.handle, h.n_occ, 3, C.byref(o), P.handle, None) == gb._ffi.DBCSR_EINVAL
    assert gb.lib().dbcsr_purify(H.handle, -1.0, 1, C.byref(o), P.handle, None) == gb._ffi.DBCSR_EINVAL
    o.prec = gb.DBCSR_MIXED
    assert gb.lib().dbcsr_purify(H.handle, h.n_occ, 1, C.byref(o), P.handle, None) == gb._ffi.DBCSR_EINVAL
    assert gb.lib().dbcsr_purify(H.handle, h.n_occ, 1, None, H.handle, None) == gb._ffi.DBCSR_EINVAL
