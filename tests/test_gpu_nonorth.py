"""GPU parity of the non-orthogonal path against the FP64 oracle, through the C ABI: the
inverse square root from the sign of [[0, S], [1, 0]] (dbcsr_inverse_sqrt) and the density
matrix P = (1 - sign(S^-1 K - mu 1)) S^-1 / 2 (dbcsr_sign_iterate_nonorth)."""
import numpy as np
import pytest
import scipy.linalg as sl

import synth
from oracle import bsr, sign

pytestmark = pytest.mark.gpu

DE_ATOM = 1e-6


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


def _system(n_mol, basis, seed):
    w = synth.small(n_mol, basis=basis, seed=seed)
    return synth.build_hamiltonian(w), synth.build_overlap(w)


CASES = [(8, (13, 5), 0.0, 1e-12), (24, (13, 5), 1e-7, 1e-9), (16, (23, 7), 1e-6, 1e-8)]


@pytest.mark.parametrize("order", [2, 3, 5])
@pytest.mark.parametrize("n_mol,basis,eps,tol", CASES)
def test_inverse_sqrt_matches_oracle(gb, order, n_mol, basis, eps, tol):
    h, s = _system(n_mol, basis, 2024 + n_mol)
    So = bsr.Mat.of(s)
    o = sign.inverse_sqrt(So, eps, tol, order=order)
    S = gb.Matrix.of(s)
    # both triangles of every product: the oracle's iteration to rounding
    f = gb.inverse_sqrt(S, eps, tol, order=order, full_products=True)
    assert f.report.alpha == pytest.approx(o.scale, rel=1e-15)
    assert bool(f.report.converged) == o.converged and bool(f.report.stalled) == o.stalled
    assert f.report.iterations == o.iterations
    np.testing.assert_allclose(f.residuals, o.residuals, rtol=1e-6, atol=1e-10)
    for got, ref in ((_mat(f.Sinvsqrt), o.Sinvsqrt), (_mat(f.Ssqrt), o.Ssqrt)):
        if np.array_equal(got.col, ref.col):
            assert np.linalg.norm(got.data - ref.data) / np.linalg.norm(ref.data) < 1e-9
        else:   # a block whose norm sits at eps within rounding: compare densely
            assert np.linalg.norm(bsr.to_dense(got) - bsr.to_dense(ref)) / np.linalg.norm(ref.data) < 1e-9
    # default: mirrored products
    g = gb.inverse_sqrt(S, eps, tol, order=order)
    assert g.converged or g.report.stalled
    assert abs(g.report.iterations - o.iterations) <= 1
    Z, Sd = bsr.to_dense(_mat(g.Sinvsqrt)), bsr.to_dense(So)
    assert np.array_equal(Z, Z.T)
    assert np.linalg.norm(Z @ Sd @ Z - np.eye(Sd.shape[0])) / np.sqrt(Sd.shape[0]) < max(1e-11, 10 * eps)


@pytest.mark.parametrize("order", [2, 5])
@pytest.mark.parametrize("n_mol,basis,eps,tol", CASES)
def test_nonorth_density_matrix_matches_oracle(gb, order, n_mol, basis, eps, tol):
    h, s = _system(n_mol, basis, 3030 + n_mol)
    o = sign.density_matrix_nonorth(bsr.Mat.of(h.H), bsr.Mat.of(s), 0.0, eps, tol, order=order)
    K, S = gb.Matrix.of(h.H), gb.Matrix.of(s)
    f = gb.sign_iterate_nonorth(K, S, 0.0, eps, tol, order=order, full_products=True)
    assert f.report.iterations == o.sign.iterations
    assert f.report_sqrt.iterations == o.sqrt.iterations
    assert abs(f.report.e_band - o.e_band) / h.n_atoms < 1e-10
    assert f.report.trace_p == pytest.approx(o.trace_ps, abs=1e-8)
    assert f.report.trace_p == pytest.approx(h.n_occ, abs=1e-5)
    g = gb.sign_iterate_nonorth(K, S, 0.0, eps, tol, order=order)
    assert abs(g.report.e_band - o.e_band) / h.n_atoms < max(1e-10, 0.1 * eps)
    assert g.report.trace_p == pytest.approx(h.n_occ, abs=1e-5)
    P = bsr.to_dense(_mat(g.P))
    assert np.array_equal(P, P.T)


def test_nonorth_against_generalized_eigenproblem(gb):
    h, s = _system(10, (13, 5), 77)
    Kd, Sd = bsr.to_dense(bsr.Mat.of(h.H)), bsr.to_dense(bsr.Mat.of(s))
    e, C = sl.eigh(Kd, Sd)
    Pe = C[:, e < 0] @ C[:, e < 0].T
    g = gb.sign_iterate_nonorth(gb.Matrix.of(h.H), gb.Matrix.of(s), 0.0, 0.0, 1e-13)
    P = bsr.to_dense(_mat(g.P))
    assert np.linalg.norm(P - Pe) / np.linalg.norm(Pe) < 1e-10
    assert np.linalg.norm(P @ Sd @ P - P) < 1e-10
    assert g.report.e_band == pytest.approx(e[e < 0].sum(), abs=1e-9)


def test_identity_overlap_gives_the_orthogonal_result_bit_for_bit(gb):
    h, s = _system(12, (13, 5), 91)
    Io = sign.identity_like(bsr.Mat.of(s))
    I = gb.Matrix.of(synth.BlockMatrix(Io.bs, Io.rp, Io.col, Io.data))
    K = gb.Matrix.of(h.H)
    # unfiltered, the congruences by S^-1/2 = 1 are exact (with eps > 0 they would drop H's
    # blocks under eps, which the orthogonal iteration keeps in X_0)
    g = gb.sign_iterate_nonorth(K, I, 0.0, 0.0, 1e-11)
    d = gb.sign_iterate(K, 0.0, 0.0, 1e-11)
    assert g.report_sqrt.iterations == 1 and g.report_sqrt.converged
    assert g.report.iterations == d.report.iterations
    for a, b in zip(g.P.export(), d.P.export()):
        assert np.array_equal(a, b)


def test_nonorth_mixed_matches_fp64_oracle(gb):
    h, s = _system(24, (13, 5), 5151)
    o = sign.density_matrix_nonorth(bsr.Mat.of(h.H), bsr.Mat.of(s), 0.0, 1e-7, 1e-8)
    g = gb.sign_iterate_nonorth(gb.Matrix.of(h.H), gb.Matrix.of(s), 0.0, 1e-7, 1e-8, prec=gb.DBCSR_MIXED)
    assert g.report.fp64_from > 1 and g.report_sqrt.fp64_from > 1
    assert abs(g.report.e_band - o.e_band) / h.n_atoms < DE_ATOM
    # the square root ends on the true S (re-anchored in FP64), so Tr(P S) keeps the FP64 accuracy
    assert g.report.trace_p == pytest.approx(h.n_occ, abs=1e-6)


@pytest.mark.parametrize("order", [2, 5])
def test_mixed_inverse_sqrt_ends_on_the_true_matrix(gb, order):
    h, s = _system(24, (13, 5), 6161)
    S = gb.Matrix.of(s)
    g = gb.inverse_sqrt(S, 1e-7, 1e-9, prec=gb.DBCSR_MIXED, order=order)
    f = gb.inverse_sqrt(S, 1e-7, 1e-9, order=order)
    assert g.report.fp64_from > 1 and (g.converged or g.report.stalled)
    Sd = bsr.to_dense(bsr.Mat.of(s))
    n = Sd.shape[0]
    for r in (g, f):
        Z = bsr.to_dense(_mat(r.Sinvsqrt))
        assert np.linalg.norm(Z @ Sd @ Z - np.eye(n)) / np.sqrt(n) < 1e-6


def test_nonorth_arguments_are_checked(gb):
    h, s = _system(6, (13, 5), 5)
    K, S = gb.Matrix.of(h.H), gb.Matrix.of(s)
    # an output aliasing S
    assert gb.lib().dbcsr_inverse_sqrt(S.handle, None, S.handle, None, None) == gb._ffi.DBCSR_EINVAL
    with pytest.raises(gb.DbcsrError) as e:
        gb.sign_iterate_nonorth(K, S, 0.0, 0.0, 1e-9, P=K)
    assert e.value.status == gb._ffi.DBCSR_EINVAL
    with pytest.raises(gb.DbcsrError) as e:
        gb.inverse_sqrt(S, 0.0, 1e-9, order=9)
    assert e.value.status == gb._ffi.DBCSR_EINVAL


@pytest.mark.parametrize("n_mol,basis,eps,tol", CASES)
def test_hotelling_inverse_matches_oracle(gb, n_mol, basis, eps, tol):
    h, s = _system(n_mol, basis, 7070 + n_mol)
    So = bsr.Mat.of(s)
    o = sign.hotelling_inverse(So, eps, tol)
    S = gb.Matrix.of(s)
    f = gb.inverse_hotelling(S, eps, tol, full_products=True)
    assert bool(f.report.converged) == o.converged and f.report.iterations == o.iterations
    np.testing.assert_allclose(f.residuals, o.residuals, rtol=1e-6, atol=1e-12)
    got = _mat(f.P)
    assert np.linalg.norm(bsr.to_dense(got) - bsr.to_dense(o.Ainv)) / np.linalg.norm(o.Ainv.data) < 1e-9
    g = gb.inverse_hotelling(S, eps, tol)                      # mirrored products
    X, Sd = bsr.to_dense(_mat(g.P)), bsr.to_dense(So)
    assert np.array_equal(X, X.T)
    assert np.linalg.norm(Sd @ X - np.eye(Sd.shape[0])) / np.sqrt(Sd.shape[0]) < max(1e-11, 10 * eps)
