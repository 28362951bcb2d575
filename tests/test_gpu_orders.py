"""GPU parity of the block-sparse add (dbcsr_add) and of the higher-order sign
iterations (orders 3 to 7) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

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


def _same(G, O):
    assert np.array_equal(G.rp, O.rp)
    assert np.array_equal(G.col, O.col)
    assert np.array_equal(G.data, O.data)


# ------------------------------------------------------------------ add
@pytest.mark.parametrize("bs,da,db", [([13, 5, 5] * 40, 0.2, 0.35),           # 120 rows, ~30-40 blocks a row
                                      ([23, 7, 7, 13, 5, 5] * 30, 0.05, 0.6),  # one side much denser
                                      ([5] * 700, 0.08, 0.08)])                # rows of 56 blocks: two ballot chunks
@pytest.mark.parametrize("alpha,beta", [(1.0, 1.0), (0.75, -1.40625), (-2.5, 0.3)])
def test_add_matches_oracle_bit_for_bit(gb, bs, da, db, alpha, beta):
    a = synth.random_block_matrix(bs, da, 11, empty_rows=(3, 17))
    b = synth.random_block_matrix(bs, db, 12, empty_rows=(17, 40))
    A, B = gb.Matrix.of(a), gb.Matrix.of(b)
    gb.add(alpha, A, beta, B)
    _same(_mat(A), bsr.add(alpha, bsr.Mat.of(a), beta, bsr.Mat.of(b)))
    _same(_mat(B), bsr.Mat.of(b))                    # B unchanged


def test_add_edge_cases(gb):
    bs = [13, 5, 5] * 8
    a = synth.random_block_matrix(bs, 0.4, 21)
    Ao = bsr.Mat.of(a)
    empty = synth.random_block_matrix(bs, 0.0, 22, diag=False)
    # B empty, A empty, both empty
    A = gb.Matrix.of(a)
    gb.add(2.0, A, 3.0, gb.Matrix.of(empty))
    _same(_mat(A), bsr.add(2.0, Ao, 3.0, bsr.Mat.of(empty)))
    E = gb.Matrix.of(empty)
    gb.add(2.0, E, 3.0, gb.Matrix.of(a))
    _same(_mat(E), bsr.add(2.0, bsr.Mat.of(empty), 3.0, Ao))
    E2 = gb.Matrix.of(empty)
    gb.add(1.0, E2, 1.0, gb.Matrix.of(empty))
    assert _mat(E2).nnzb == 0
    # B the same handle as A
    A = gb.Matrix.of(a)
    gb.add(0.5, A, 0.25, A)
    _same(_mat(A), bsr.add(0.5, Ao, 0.25, Ao))
    # errors: block sizes differ, unfinalized operand
    with pytest.raises(gb.DbcsrError) as e:
        gb.add(1.0, gb.Matrix.of(a), 1.0, gb.Matrix.of(synth.random_block_matrix([13, 5] * 12, 0.4, 23)))
    assert e.value.status == gb._ffi.DBCSR_EINVAL
    with pytest.raises(gb.DbcsrError) as e:
        gb.add(1.0, gb.Matrix.of(a), 1.0, gb.Matrix(bs, None))
    assert e.value.status == gb._ffi.DBCSR_ESTATE


# ------------------------------------------------------------------ higher orders
@pytest.mark.parametrize("order", [3, 4, 5, 6, 7])
@pytest.mark.parametrize("n_mol,basis,eps,tol", [(8, (13, 5), 0.0, 1e-12), (24, (13, 5), 1e-7, 1e-8),
                                                 (16, (23, 7), 1e-6, 1e-8)])
def test_higher_order_sign_matches_oracle(gb, order, n_mol, basis, eps, tol):
    h = synth.build_hamiltonian(synth.small(n_mol, basis=basis, seed=777 + n_mol))
    H = gb.Matrix.of(h.H)
    o = sign.sign_iterate(bsr.Mat.of(h.H), 0.0, eps, tol, order=order)
    assert o.converged
    # both triangles of every product formed: the oracle's iteration to rounding
    f = gb.sign_iterate(H, 0.0, eps, tol, full_products=True, order=order)
    assert bool(f.report.converged) == o.converged
    assert f.report.iterations == o.iterations
    np.testing.assert_allclose(f.residuals, o.residuals, rtol=1e-6, atol=1e-10)
    assert abs(f.report.e_band - o.e_band) / h.n_atoms < 1e-10
    assert f.report.trace_p == pytest.approx(h.n_occ, abs=1e-5)
    assert f.report.flops <= o.flops * (1 + 1e-12)             # the prescreen only skips filtered blocks
    rp, col, data = f.P.export()
    if np.array_equal(col, o.P.col):
        assert np.linalg.norm(data - o.P.data) / np.linalg.norm(o.P.data) < 1e-9
    # default: mirrored symmetric products, to the filter's accuracy
    g = gb.sign_iterate(H, 0.0, eps, tol, order=order)
    assert g.converged
    assert abs(g.report.iterations - o.iterations) <= 1
    assert abs(g.report.e_band - o.e_band) / h.n_atoms < max(1e-10, 0.1 * eps)


@pytest.mark.parametrize("order", [3, 5, 7])
def test_higher_order_against_dense_eigh(gb, order):
    h = synth.build_hamiltonian(synth.small(10, seed=4321))
    Hd = bsr.to_dense(bsr.Mat.of(h.H))
    w, Q = np.linalg.eigh(Hd)
    Pd = 0.5 * (np.eye(Hd.shape[0]) - Q @ np.diag(np.sign(w)) @ Q.T)
    g = gb.sign_iterate(gb.Matrix.of(h.H), 0.0, 0.0, 1e-13, order=order)
    P = bsr.to_dense(_mat(g.P))
    assert np.linalg.norm(P - Pd) / np.linalg.norm(Pd) < 1e-11


@pytest.mark.parametrize("order", [3, 5])
def test_higher_order_mixed_matches_fp64_oracle(gb, order):
    h = synth.build_hamiltonian(synth.small(24, seed=990 + 24))
    g = gb.sign_iterate(gb.Matrix.of(h.H), 0.0, 1e-7, 1e-8, prec=gb.DBCSR_MIXED, switch_tol=1e-4, order=order)
    o = sign.sign_iterate(bsr.Mat.of(h.H), 0.0, 1e-7, 1e-8, order=order)
    assert g.report.fp64_from > 1
    assert g.converged
    assert abs(g.report.e_band - o.e_band) / h.n_atoms < DE_ATOM
    assert g.report.trace_p == pytest.approx(h.n_occ, abs=1e-4)


def test_higher_order_batch_equals_single_runs(gb):
    rng = np.random.default_rng(5)
    hs = [synth.build_hamiltonian(synth.small(int(rng.integers(6, 30)), basis=b, seed=4400 + i))
          for i, b in enumerate([(13, 5), (23, 7), (13, 7), (23, 5)])]
    Hs = [gb.Matrix.of(h.H) for h in hs]
    mus = [0.0, 0.2, -0.22, 0.1]
    Ps, reps, st = gb.sign_iterate_batched(Hs, mus, 1e-7, 1e-9, order=5)
    for h, H, P, r, mu in zip(hs, Hs, Ps, reps, mus):
        g = gb.sign_iterate(H, mu, 1e-7, 1e-9, order=5)
        assert r.iterations == g.report.iterations
        for a, b in zip(P.export(), g.P.export()):
            assert np.array_equal(a, b)


def test_order_arguments_are_checked(gb):
    h = synth.build_hamiltonian(synth.small(6, seed=3))
    H = gb.Matrix.of(h.H)
    for bad in (1, 8, -2):
        with pytest.raises(gb.DbcsrError) as e:
            gb.sign_iterate(H, 0.0, 0.0, 1e-9, order=bad, raise_on_notconv=True)
        assert e.value.status == gb._ffi.DBCSR_EINVAL
    with pytest.raises(gb.DbcsrError) as e:
        gb.sign_iterate(H, 0.0, 0.0, 1e-9, prec=gb.DBCSR_MIXED, order=5, low_correction=True)
    assert e.value.status == gb._ffi.DBCSR_EINVAL
    # order 0 is the default, Newton-Schulz
    a = gb.sign_iterate(H, 0.0, 0.0, 1e-11, order=0)
    b = gb.sign_iterate(H, 0.0, 0.0, 1e-11)
    assert a.report.iterations == b.report.iterations
    for x, y in zip(a.P.export(), b.P.export()):
        assert np.array_equal(x, y)
