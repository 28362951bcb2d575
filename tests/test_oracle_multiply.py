"""Pins of the oracle's block-sparse product, filter and traces against dense
linear algebra and brute force (no GPU)."""
import itertools

import numpy as np
import pytest

import synth
from oracle import bsr


def _mat(bs, density, seed, **kw):
    return bsr.Mat.of(synth.random_block_matrix(bs, density, seed, **kw))


SIZES = [
    [13, 5, 5, 13, 5, 5, 13, 5, 5],
    [1, 2, 3, 4, 5, 6, 7],
    [23, 7, 7, 23, 7, 7],
    [4],
]


@pytest.mark.parametrize("bs", SIZES)
@pytest.mark.parametrize("density", [0.0, 0.3, 1.0])
def test_product_equals_dense_gemm(bs, density):
    A = _mat(bs, density, 1)
    B = _mat(bs, density, 2)
    C = bsr.multiply(1.0, A, B)
    ref = bsr.to_dense(A) @ bsr.to_dense(B)
    np.testing.assert_allclose(bsr.to_dense(C), ref, rtol=0, atol=1e-14 * max(1, np.abs(ref).max()))


@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (-0.5, 1.5), (2.0, -1.0), (0.0, 1.0)])
def test_alpha_beta_update(alpha, beta):
    bs = SIZES[0]
    A, B, Cin = _mat(bs, 0.4, 3), _mat(bs, 0.4, 4), _mat(bs, 0.3, 5)
    C = bsr.multiply(alpha, A, B, beta, Cin)
    ref = alpha * (bsr.to_dense(A) @ bsr.to_dense(B)) + beta * bsr.to_dense(Cin)
    np.testing.assert_allclose(bsr.to_dense(C), ref, rtol=0, atol=1e-14)
    # the pattern of the result is the union of A*B's and C_in's (beta != 0)
    rp, col = bsr.product_pattern(A, B, Cin if beta != 0 else None)
    assert np.array_equal(C.col, col) and np.array_equal(C.rp, rp)


def test_pattern_and_product_count_brute_force():
    bs = SIZES[1]
    A, B = _mat(bs, 0.35, 6), _mat(bs, 0.35, 7)
    _, info = bsr.multiply(1.0, A, B, info=True)
    nb = len(bs)
    pa = {(int(i), int(j)) for i, j in zip(A.rows, A.col)}
    pb = {(int(i), int(j)) for i, j in zip(B.rows, B.col)}
    prods = [(i, k, j) for i, k, j in itertools.product(range(nb), repeat=3) if (i, k) in pa and (k, j) in pb]
    assert info.n_products == len(prods)
    assert info.flops == sum(2 * bs[i] * bs[k] * bs[j] for i, k, j in prods)
    cands = sorted({(i, j) for i, _, j in prods})
    got = sorted(zip(info.unfiltered.rows.tolist(), info.unfiltered.col.tolist()))
    assert got == cands


def test_non_commuting_operands_not_transposed():
    # A*B != B*A and != A^T*B for random non-symmetric data: a swapped or transposed
    # operand in the oracle would fail here
    bs = SIZES[0]
    A, B = _mat(bs, 0.5, 8), _mat(bs, 0.5, 9)
    C = bsr.to_dense(bsr.multiply(1.0, A, B))
    Ad, Bd = bsr.to_dense(A), bsr.to_dense(B)
    assert np.abs(C - Ad @ Bd).max() < 1e-13
    assert np.abs(C - Bd @ Ad).max() > 1e-2
    assert np.abs(C - Ad.T @ Bd).max() > 1e-2


@pytest.mark.parametrize("eps", [1e-3, 0.3, 2.0])
def test_filter_is_dense_gemm_then_block_mask(eps):
    bs = SIZES[0]
    A, B = _mat(bs, 0.5, 10, scale=0.3), _mat(bs, 0.5, 11, scale=0.3)
    C, info = bsr.multiply(1.0, A, B, eps=eps, info=True)
    ref = bsr.to_dense(A) @ bsr.to_dense(B)
    roff = np.concatenate([[0], np.cumsum(bs)])
    mask = np.zeros_like(ref)
    cands = set(zip(info.unfiltered.rows.tolist(), info.unfiltered.col.tolist()))
    for I, J in itertools.product(range(len(bs)), repeat=2):
        blk = ref[roff[I]:roff[I + 1], roff[J]:roff[J + 1]]
        if (I, J) in cands and (np.linalg.norm(blk) >= eps or I == J):
            mask[roff[I]:roff[I + 1], roff[J]:roff[J + 1]] = 1
    np.testing.assert_allclose(bsr.to_dense(C), ref * mask, rtol=0, atol=1e-14)
    # diagonal blocks survive any threshold
    for I in range(len(bs)):
        if (I, I) in cands:
            assert C.block(I, I) is not None


def test_norm_bound_prescreen_is_exact():
    # ||C_IJ||_F <= sum_K ||A_IK||_F ||B_KJ||_F (triangle inequality + submultiplicativity):
    # a candidate whose bound is below eps is always filtered
    bs = SIZES[2]
    A, B = _mat(bs, 0.6, 12), _mat(bs, 0.6, 13)
    _, info = bsr.multiply(1.0, A, B, info=True)
    nA, _ = bsr.block_norms(A)
    nB, _ = bsr.block_norms(B)
    for b in range(info.unfiltered.nnzb):
        I, J = int(info.unfiltered.rows[b]), int(info.unfiltered.col[b])
        bound = 0.0
        for p in range(A.rp[I], A.rp[I + 1]):
            K = int(A.col[p])
            lo, hi = int(B.rp[K]), int(B.rp[K + 1])
            k = lo + int(np.searchsorted(B.col[lo:hi], J))
            if k < hi and B.col[k] == J:
                bound += nA[p] * nB[k]
        assert info.norms[b] <= bound * (1 + 1e-14)


def test_block_norms_and_identity_deviation():
    bs = SIZES[1]
    M = _mat(bs, 0.5, 14)
    norms, dev2 = bsr.block_norms(M)
    D = bsr.to_dense(M)
    roff = np.concatenate([[0], np.cumsum(bs)])
    for b in range(M.nnzb):
        I, J = int(M.rows[b]), int(M.col[b])
        blk = D[roff[I]:roff[I + 1], roff[J]:roff[J + 1]]
        assert norms[b] == pytest.approx(np.linalg.norm(blk), rel=1e-15)
    full = bsr.lib().oracle_sum_dev2(M.nblk, bsr._p(M.bs), bsr._p(M.rp), bsr._p(M.col), bsr._p(dev2))
    assert full == pytest.approx(np.linalg.norm(D - np.eye(D.shape[0])) ** 2, rel=1e-13)


def test_empty_rows_and_empty_matrix():
    bs = SIZES[0]
    A = _mat(bs, 0.5, 15, empty_rows=(2, 4))
    B = _mat(bs, 0.5, 16)
    C = bsr.multiply(1.0, A, B)
    for r in (2, 4):
        assert C.rp[r + 1] == C.rp[r]
    np.testing.assert_allclose(bsr.to_dense(C), bsr.to_dense(A) @ bsr.to_dense(B), atol=1e-14)
    Z = _mat(bs, 0.0, 17, diag=False)
    assert Z.nnzb == 0
    assert bsr.multiply(1.0, Z, B).nnzb == 0


def test_traces():
    bs = SIZES[0]
    A, B = _mat(bs, 0.5, 18), _mat(bs, 0.5, 19)
    Ad, Bd = bsr.to_dense(A), bsr.to_dense(B)
    assert bsr.trace(A) == pytest.approx(np.trace(Ad), rel=1e-14)
    assert bsr.trace_product(A, B) == pytest.approx(np.trace(Ad @ Bd), rel=1e-13)
    assert bsr.trace_product(A, B) != pytest.approx(np.sum(Ad * Bd), rel=1e-6)   # not <A, B>


def test_gershgorin_row_sums():
    bs = SIZES[1]
    A = _mat(bs, 0.5, 20)
    D = bsr.to_dense(A)
    for mu in (0.0, 0.7):
        ref = np.abs(D - mu * np.eye(D.shape[0])).sum(axis=1)
        np.testing.assert_allclose(bsr.abs_row_sums(A, mu), ref, rtol=1e-14)


def test_decay_matrix_square_matches_dense():
    A = bsr.Mat.of(synth.build_decay(synth.DECAY_32))
    C, info = bsr.multiply(1.0, A, A, eps=1e-6, info=True)
    D = bsr.to_dense(A)
    ref = D @ D
    np.testing.assert_allclose(bsr.to_dense(info.unfiltered), ref, rtol=0, atol=1e-13 * np.abs(ref).max())
    # the product of a 99.96%-dense 96-block matrix with itself is block-dense
    assert info.unfiltered.nnzb == 96 * 96


def test_thread_count_does_not_change_results(monkeypatch):
    import subprocess, sys, os
    code = ("import numpy as np, synth; from oracle import bsr;"
            "A=bsr.Mat.of(synth.build_decay(synth.DECAY_32));"
            "C=bsr.multiply(1.0,A,A,eps=1e-6); import hashlib;"
            "print(hashlib.sha256(C.data.tobytes()).hexdigest())")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    outs = []
    for t in ("1", "3"):
        env = dict(os.environ, OMP_NUM_THREADS=t)
        outs.append(subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True,
                                   text=True, check=True).stdout.strip())
    assert outs[0] == outs[1]


def test_set_num_threads_gives_the_same_product():
    A = bsr.Mat.of(synth.build_decay(synth.DECAY_32))
    n0 = bsr.num_threads()
    try:
        bsr.set_num_threads(1)
        assert bsr.num_threads() == 1
        C1 = bsr.multiply(1.0, A, A, eps=1e-6)
        bsr.set_num_threads(max(2, n0))
        C2 = bsr.multiply(1.0, A, A, eps=1e-6)
    finally:
        bsr.set_num_threads(n0)
    assert np.array_equal(C1.col, C2.col) and np.array_equal(C1.data, C2.data)


def _dense_block(D, roff, I, J):
    return D[roff[I]:roff[I + 1], roff[J]:roff[J + 1]]


@pytest.mark.parametrize("bs", [SIZES[0], SIZES[1], SIZES[2], [32, 1, 17, 32, 2]])
@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (-0.5, 1.5), (2.0, -1.0)])
def test_product_block_matches_dense_and_full_product(bs, alpha, beta):
    # product_block checks sampled outputs of products too large for the oracle's full
    # multiply; every block of small ragged products (including blocks outside the
    # product's pattern, empty rows and a C input) must equal the dense definition
    # alpha*A*B + beta*C_in and the same block of the full oracle product
    A = _mat(bs, 0.45, 21, empty_rows=(1,))
    B = _mat(bs, 0.45, 22, empty_rows=(len(bs) - 1,))
    Cin = _mat(bs, 0.3, 23)
    Ad, Bd, Cd = bsr.to_dense(A), bsr.to_dense(B), bsr.to_dense(Cin)
    ref = alpha * (Ad @ Bd) + beta * Cd
    full = bsr.to_dense(bsr.multiply(alpha, A, B, beta, Cin if beta != 0.0 else None))
    roff = np.concatenate([[0], np.cumsum(bs)])
    scale = max(1.0, np.abs(ref).max())
    n_absent = 0
    for I, J in itertools.product(range(len(bs)), repeat=2):
        got = bsr.product_block(I, J, alpha, A, B, beta, Cin)
        assert got.shape == (bs[I], bs[J])
        want = _dense_block(ref, roff, I, J)
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-15 * scale * 8)
        # same loop order as the full product: equal to rounding of the last bit
        np.testing.assert_allclose(got, _dense_block(full, roff, I, J), rtol=0, atol=1e-15 * scale)
        if np.all(want == 0.0):
            n_absent += 1
            assert np.all(got == 0.0)
    # the empty row of A gives whole zero block rows (beta C_in aside)
    assert n_absent >= 1 or beta != 0.0


def test_product_block_wrong_b_block_fails_the_pin():
    # planted mistake: the block of B found for (K, J) is its neighbour in storage (an
    # off-by-one of the search), emulated by shifting B's block offsets by one block
    bs = SIZES[0]
    A, B = _mat(bs, 0.5, 24), _mat(bs, 0.5, 25)
    ref = bsr.to_dense(A) @ bsr.to_dense(B)
    roff = np.concatenate([[0], np.cumsum(bs)])
    good_err = max(np.abs(bsr.product_block(I, J, 1.0, A, B) - _dense_block(ref, roff, I, J)).max()
                   for I, J in itertools.product(range(len(bs)), repeat=2))
    assert good_err < 1e-13
    Bbad = B.copy()
    Bbad.boff = np.concatenate([B.boff[1:], [B.boff[-1]]]).astype(np.int64)
    Bbad.data = np.concatenate([B.data, np.zeros(32 * 32)])    # reads stay inside the buffer
    bad_err = max(np.abs(bsr.product_block(I, J, 1.0, A, Bbad) - _dense_block(ref, roff, I, J)).max()
                  for I, J in itertools.product(range(len(bs)), repeat=2))
    assert bad_err > 1e-2


def _dense_pattern(M, weights=None):
    D = np.zeros((M.nblk, M.nblk))
    D[M.rows, M.col] = 1.0 if weights is None else weights
    return D


@pytest.mark.parametrize("eps", [1e-2, 1e-1, 1.0])          # the 32-water box screens from about 1e-2
@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (-0.5, 1.5)])
def test_prescreen_leaves_the_filtered_product_unchanged(eps, alpha, beta):
    A = bsr.Mat.of(synth.build_decay(synth.DECAY_32))
    Cin = _mat(A.bs, 0.2, 31)
    full, fi = bsr.multiply(alpha, A, A, beta, Cin, eps=eps, info=True)
    pre, pi = bsr.multiply(alpha, A, A, beta, Cin, eps=eps, info=True, prescreen=True)
    assert np.array_equal(full.rp, pre.rp) and np.array_equal(full.col, pre.col)
    assert np.array_equal(full.data, pre.data)                 # the same loops on the kept blocks
    assert pi.dev2 == fi.dev2
    assert pi.unfiltered.nnzb < fi.unfiltered.nnzb and pi.n_products < fi.n_products
    # without a threshold nothing is screened
    _, zi = bsr.multiply(alpha, A, A, beta, Cin, eps=0.0, info=True, prescreen=True)
    assert zi.n_products == bsr.multiply(alpha, A, A, beta, Cin, info=True)[1].n_products


def test_prescreen_forms_the_blocks_whose_bound_reaches_eps():
    # brute force on dense block-norm matrices: formed <=> diagonal or |alpha| (NA NB)_IJ >= eps
    # (candidates within 1e-9 of eps, where the summation order could decide, are left out);
    # product and flop counts over the formed blocks
    A = bsr.Mat.of(synth.build_decay(synth.DECAY_32))
    eps, alpha = 0.1, -0.75
    _, fi = bsr.multiply(alpha, A, A, info=True)
    _, pi = bsr.multiply(alpha, A, A, eps=eps, info=True, prescreen=True)
    na, _ = bsr.block_norms(A)
    bound = abs(alpha) * (_dense_pattern(A, na) @ _dense_pattern(A, na))
    cand = _dense_pattern(fi.unfiltered) > 0
    formed = _dense_pattern(pi.unfiltered) > 0
    assert not np.any(formed & ~cand)
    want = cand & ((bound >= eps) | np.eye(A.nblk, dtype=bool))
    clear = np.abs(bound / eps - 1.0) > 1e-9
    assert np.array_equal(formed[clear], want[clear])
    assert 0 < formed.sum() < cand.sum()
    PA = _dense_pattern(A)
    assert pi.n_products == int((PA @ PA)[formed].sum())
    m = A.bs.astype(np.float64)
    flops = 2.0 * m[:, None] * ((PA * m[None, :]) @ PA) * m[None, :]
    assert pi.flops == int(round(flops[formed].sum()))
