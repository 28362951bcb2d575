"""GPU parity of the block-sparse product, filter, traces and Gershgorin bound
against the FP64 oracle (through the C ABI)."""
import numpy as np
import pytest

import synth
from oracle import bsr

pytestmark = pytest.mark.gpu

REL_FP64 = 1e-12       # relative Frobenius error allowed per FP64 product on a shared pattern


@pytest.fixture(scope="module")
def gb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2003_03868_gb300 as m
    m.lib()
    return m


def _pair(gb, bm):
    return gb.Matrix.of(bm), bsr.Mat.of(bm)


def _assert_same(gm, om: bsr.Mat, rel=REL_FP64):
    rp, col, data = gm.export()
    assert np.array_equal(rp, om.rp), "row pointers differ"
    assert np.array_equal(col, om.col), "block columns differ"
    if om.data.size == 0:
        assert data.size == 0
        return
    den = max(np.linalg.norm(om.data), 1e-300)
    err = np.linalg.norm(data - om.data) / den
    assert err <= rel, f"relative Frobenius error {err:.2e}"
    # element by element as well
    np.testing.assert_allclose(data, om.data, rtol=0, atol=rel * max(1.0, np.abs(om.data).max()) * 10)


SIZES = [
    [13, 5, 5] * 6,
    [1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 18, 19, 20, 21, 22, 23, 24, 25, 26, 27, 28, 29, 30, 31, 32],
    [23, 7, 7] * 5,
    [4] * 70,            # more block columns than one bitmap word and than one warp
]


@pytest.mark.parametrize("si", range(len(SIZES)))
@pytest.mark.parametrize("density", [0.05, 0.4, 1.0])
def test_product_matches_oracle_eps0(gb, si, density):
    bs = SIZES[si]
    a = synth.random_block_matrix(bs, density, 100 + si)
    b = synth.random_block_matrix(bs, density, 200 + si)
    (A, Ao), (B, Bo) = _pair(gb, a), _pair(gb, b)
    C = gb.Matrix(A.blk_size, A.stream)
    st = gb.multiply(1.0, A, B, 0.0, C, 0.0)
    Co, info = bsr.multiply(1.0, Ao, Bo, info=True)
    _assert_same(C, Co)
    assert st.n_products == info.n_products
    assert st.flops == info.flops
    assert st.n_candidates == info.unfiltered.nnzb == st.n_formed


@pytest.mark.parametrize("alpha,beta", [(1.0, 1.0), (-0.5, 1.5), (2.0, -1.0), (0.0, 1.0)])
def test_alpha_beta_matches_oracle(gb, alpha, beta):
    bs = SIZES[0]
    a, b, c = (synth.random_block_matrix(bs, 0.3, s) for s in (31, 32, 33))
    (A, Ao), (B, Bo), (Cm, Co) = _pair(gb, a), _pair(gb, b), _pair(gb, c)
    gb.multiply(alpha, A, B, beta, Cm, 0.0)
    ref = bsr.multiply(alpha, Ao, Bo, beta, Co)
    _assert_same(Cm, ref)


def test_in_place_update_aliasing(gb):
    # X <- 1.5 X - 0.5 X.Y with C aliasing A, as in the sign iteration
    bs = SIZES[2]
    x = synth.random_block_matrix(bs, 0.4, 41, symmetric=True)
    y = synth.random_block_matrix(bs, 0.4, 42, symmetric=True)
    (X, Xo), (Y, Yo) = _pair(gb, x), _pair(gb, y)
    gb.multiply(-0.5, X, Y, 1.5, X, 0.0)
    _assert_same(X, bsr.multiply(-0.5, Xo, Yo, 1.5, Xo))
    # and A = B = C
    Z, Zo = _pair(gb, x)
    gb.multiply(1.0, Z, Z, 0.0, Z, 0.0)
    _assert_same(Z, bsr.multiply(1.0, Zo, Zo))


@pytest.mark.parametrize("eps", [1e-3, 0.05, 0.5])
def test_filtered_product_matches_oracle(gb, eps):
    bs = SIZES[0]
    a = synth.random_block_matrix(bs, 0.5, 51, scale=0.2)
    b = synth.random_block_matrix(bs, 0.5, 52, scale=0.2)
    (A, Ao), (B, Bo) = _pair(gb, a), _pair(gb, b)
    C = gb.Matrix(A.blk_size, A.stream)
    st = gb.multiply(1.0, A, B, 0.0, C, eps)
    Co, info = bsr.multiply(1.0, Ao, Bo, eps=eps, info=True)
    # no block norm sits within rounding of eps in this data (else the masks could differ)
    assert np.min(np.abs(info.norms - eps)) > 1e-9 * eps
    _assert_same(C, Co)
    assert st.n_kept == Co.nnzb
    assert st.n_candidates == info.unfiltered.nnzb
    assert st.n_formed <= st.n_candidates


def test_decay_32_waters(gb):
    # C = A.A of the 32-water decay matrix, eps 1e-6 (N = 736)
    a = synth.build_decay(synth.DECAY_32)
    A, Ao = _pair(gb, a)
    C = gb.Matrix(A.blk_size, A.stream)
    st = gb.multiply(1.0, A, A, 0.0, C, 1e-6)
    Co, info = bsr.multiply(1.0, Ao, Ao, eps=1e-6, info=True)
    _assert_same(C, Co)
    assert st.n_candidates == 96 * 96


def test_empty_and_ragged(gb):
    bs = SIZES[0]
    a = synth.random_block_matrix(bs, 0.5, 61, empty_rows=(0, 7, 17))
    b = synth.random_block_matrix(bs, 0.5, 62, empty_rows=(3,))
    (A, Ao), (B, Bo) = _pair(gb, a), _pair(gb, b)
    C = gb.Matrix(A.blk_size, A.stream)
    gb.multiply(1.0, A, B, 0.0, C, 0.0)
    _assert_same(C, bsr.multiply(1.0, Ao, Bo))
    z = synth.random_block_matrix(bs, 0.0, 63, diag=False)
    Z, Zo = _pair(gb, z)
    C2 = gb.Matrix(A.blk_size, A.stream)
    st = gb.multiply(1.0, Z, B, 0.0, C2, 0.0)
    assert st.n_products == 0 and C2.nnzb == 0


def test_single_block_matrix(gb):
    a = synth.random_block_matrix([7], 1.0, 71)
    A, Ao = _pair(gb, a)
    C = gb.Matrix(A.blk_size, A.stream)
    gb.multiply(1.0, A, A, 0.0, C, 0.0)
    _assert_same(C, bsr.multiply(1.0, Ao, Ao))


def test_traces_and_gershgorin(gb):
    bs = SIZES[1]
    a = synth.random_block_matrix(bs, 0.4, 81)
    b = synth.random_block_matrix(bs, 0.4, 82)
    (A, Ao), (B, Bo) = _pair(gb, a), _pair(gb, b)
    assert gb.trace(A) == pytest.approx(bsr.trace(Ao), rel=1e-13, abs=1e-13)
    assert gb.trace_product(A, B) == pytest.approx(bsr.trace_product(Ao, Bo), rel=1e-12, abs=1e-12)
    for mu in (0.0, 0.3):
        assert gb.gershgorin(A, mu) == pytest.approx(bsr.abs_row_sums(Ao, mu).max(), rel=1e-14)


def test_standalone_filter(gb):
    bs = SIZES[0]
    a = synth.random_block_matrix(bs, 0.6, 91, scale=0.3)
    A, Ao = _pair(gb, a)
    A.filter(0.9)
    _assert_same(A, bsr.filter_blocks(Ao, 0.9))


def test_put_block_order_and_duplicates(gb):
    bs = [5, 13, 5]
    m = gb.Matrix(bs)
    blocks = {(2, 0): np.arange(25.).reshape(5, 5), (0, 1): np.ones((5, 13)), (1, 1): np.eye(13)}
    for (i, j), v in blocks.items():
        m.put_block(i, j, v)
    m.finalize()
    for (i, j), v in blocks.items():
        np.testing.assert_array_equal(m.get_block(i, j), v)
    assert m.get_block(0, 0) is None
    d = gb.Matrix(bs)
    d.put_block(0, 0, np.zeros((5, 5)))
    d.put_block(0, 0, np.zeros((5, 5)))
    with pytest.raises(gb.DbcsrError):
        d.finalize()


def test_bitwise_reproducible(gb):
    a = synth.build_decay(synth.DECAY_32)
    outs = []
    for _ in range(2):
        A = gb.Matrix.of(a)
        C = gb.Matrix(A.blk_size, A.stream)
        gb.multiply(1.0, A, A, 0.0, C, 1e-6)
        outs.append(C.export()[2].tobytes())
    assert outs[0] == outs[1]


def test_pool_trim_keeps_live_matrices(gb):
    # the library's caching pool hands its free memory back; live matrices are untouched
    import torch
    a = synth.random_block_matrix(SIZES[0], 0.5, 77)
    A, Ao = gb.Matrix.of(a), bsr.Mat.of(a)
    C_ = gb.Matrix(A.blk_size, A.stream)
    gb.multiply(1.0, A, A, 0.0, C_, 0.0)
    before = C_.export()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    gb.pool_trim(0)
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0
    for x, y in zip(before, C_.export()):
        assert np.array_equal(x, y)
    gb.multiply(1.0, A, A, 0.0, C_, 0.0)         # the pool grows again on demand
    _assert_same(C_, bsr.multiply(1.0, Ao, Ao))


def _one_dense_row(nb, seed):
    """Blocks of edge 1-3; row 0 holds every block, the other rows their diagonal and
    three random blocks, so row 0 of A*A has ~nb candidates and nb products per block."""
    from synth.waterbox import BlockMatrix
    rng = np.random.default_rng(seed)
    bs = rng.integers(1, 4, nb).astype(np.int32)
    rows = [np.arange(nb)]
    for i in range(1, nb):
        rows.append(np.unique(np.concatenate([[i], rng.choice(nb, 3, replace=False)])))
    rp = np.zeros(nb + 1, dtype=np.int64)
    np.cumsum([len(r) for r in rows], out=rp[1:])
    col = np.concatenate(rows).astype(np.int32)
    rr = np.repeat(np.arange(nb), np.diff(rp))
    vals = rng.uniform(-1, 1, int((bs[rr].astype(np.int64) * bs[col]).sum()))
    return BlockMatrix(bs, rp, col, vals)


@pytest.mark.parametrize("eps", [0.0, 0.5])
def test_wide_rows_take_the_global_and_ordered_paths(gb, eps):
    # row 0 has 9,000 A blocks (at least 4,096 selects the ordered FP64 bound) and about
    # 9,000 candidates (too many for the shared-memory accumulators and stack cursors, which
    # fit about 6,000 and 8,000)
    a = _one_dense_row(9000, 8)
    (A, Ao) = _pair(gb, a)
    C = gb.Matrix(A.blk_size, A.stream)
    st = gb.multiply(1.0, A, A, 0.0, C, eps)
    Co, info = bsr.multiply(1.0, Ao, Ao, 0.0, None, eps, info=True)
    _assert_same(C, Co)
    assert st.n_candidates == info.unfiltered.nnzb
    if eps == 0.0:
        assert st.flops == info.flops


def _one_row_of(c, nb):
    """1x1 blocks; row 0 holds blocks 0..c-1, every other row its diagonal: row 0 of A*A has
    exactly c candidates."""
    from synth.waterbox import BlockMatrix
    rng = np.random.default_rng(c)
    rows = [np.arange(c)] + [np.array([i]) for i in range(1, nb)]
    rp = np.zeros(nb + 1, dtype=np.int64)
    np.cumsum([len(r) for r in rows], out=rp[1:])
    col = np.concatenate(rows).astype(np.int32)
    return BlockMatrix(np.ones(nb, dtype=np.int32), rp, col, rng.uniform(-1, 1, col.shape[0]))


def test_row_lengths_at_the_default_shared_memory_limit(gb):
    # The stack builder keeps a row's candidates in dynamic shared memory (20 bytes each in
    # the bound pass, 12 in the fill pass, after a bitmap).  Rows whose dynamic size falls
    # just under 48 KB need the opt-in too, as the kernels' static arrays count against the
    # same limit; sweep every row length whose dynamic size lies in the top 1 KB below it.
    def sm_rank(nb):
        nwords = (nb + 31) // 32
        return 2 * ((nwords + 1) & ~1) * 4

    cases = set()
    for per in (20, 12):
        for c in range(2000, 4200):
            dyn = sm_rank(c + 64) + per * c
            if 48 * 1024 - 1024 < dyn <= 48 * 1024:
                cases.add(c)
    assert len(cases) > 100
    for c in sorted(cases):
        a = _one_row_of(c, c + 64)
        (A, Ao) = _pair(gb, a)
        C = gb.Matrix(A.blk_size, A.stream)
        gb.multiply(1.0, A, A, 0.0, C, 0.0)
        _assert_same(C, bsr.multiply(1.0, Ao, Ao))
