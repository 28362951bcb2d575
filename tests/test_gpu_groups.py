"""The block groups of the tensor-core tier (dbcsr_matrix_groups) against a plain restatement of
their definition: every block row proposes its 12 strongest off-diagonal couplings (largest
block norm, ties to the lower column); the proposals are taken in decreasing norm (ties: lower
row, then lower column) and merge two groups by single linkage unless the merged group would
exceed 112 rows or 16 blocks; groups are numbered in the order of their first block.  Integer
output: compared exactly, on the norms the library ranked."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

KTOP, WIDTH, MEMBERS = 12, 112, 16


@pytest.fixture(scope="module")
def gb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2003_03868_gb300 as m
    m.lib()
    return m


def groups_by_definition(bs, rp, col, norms):
    nb = len(bs)
    rows = np.repeat(np.arange(nb, dtype=np.int64), np.diff(rp))
    off = rows != col
    r, c, w = rows[off], col[off].astype(np.int64), norms[off]
    o = np.lexsort((c, -w, r))                         # per row: norm descending, column ascending
    r, c, w = r[o], c[o], w[o]
    rank = np.arange(r.size) - np.searchsorted(r, r, side="left")
    keep = rank < KTOP
    a, b, w = np.minimum(r, c)[keep], np.maximum(r, c)[keep], w[keep]
    parent = list(range(nb))
    width = [int(x) for x in bs]
    count = [1] * nb

    def find(x):
        while parent[x] != x:
            x = parent[x]
        return x

    for k in np.lexsort((b, a, -w)):
        x, y = find(int(a[k])), find(int(b[k]))
        if x == y or width[x] + width[y] > WIDTH or count[x] + count[y] > MEMBERS:
            continue
        x, y = min(x, y), max(x, y)
        parent[y] = x
        width[x] += width[y]
        count[x] += count[y]
    gid, g_of = {}, np.empty(nb, dtype=np.int32)
    for i in range(nb):
        g_of[i] = gid.setdefault(find(i), len(gid))
    return g_of, len(gid)


def _check(gb, M, bs):
    rp, col, _ = M.export()
    g_of, norms, ng = M.groups()
    ref, ng_ref = groups_by_definition(np.asarray(bs), rp, col, norms)
    assert ng == ng_ref
    assert np.array_equal(g_of, ref)
    # the caps hold
    w = np.bincount(g_of, weights=np.asarray(bs, dtype=np.float64))
    assert w.max() <= WIDTH and np.bincount(g_of).max() <= MEMBERS
    return g_of


def test_water_hamiltonian_groups(gb):
    h = synth.build_hamiltonian(synth.small(64, basis=(23, 7), seed=8401))
    M = gb.Matrix.of(h.H)
    g_of = _check(gb, M, h.H.blk_size)
    assert g_of.max() + 1 < len(h.H.blk_size)         # something merged


def test_tied_norms_break_to_the_lower_column(gb):
    # all entries 1: a block's norm depends only on its shape, so most couplings tie
    a = synth.random_block_matrix([7, 23, 7] * 12, 0.6, 8402, symmetric=True)
    a.data[:] = 1.0
    _check(gb, gb.Matrix.of(a), a.blk_size)


@pytest.mark.parametrize("bs", [[32] * 20, [1] * 40, [5, 13, 32, 1, 17] * 8])
def test_width_and_member_caps(gb, bs):
    a = synth.random_block_matrix(bs, 0.7, 8403, symmetric=True)
    _check(gb, gb.Matrix.of(a), bs)


def test_sparse_rows_and_a_diagonal_matrix(gb):
    bs = [13, 5, 5] * 10
    a = synth.random_block_matrix(bs, 0.05, 8404, empty_rows=(3, 17))
    _check(gb, gb.Matrix.of(a), bs)
    d = synth.random_block_matrix(bs, 0.0, 8405)
    g_of = _check(gb, gb.Matrix.of(d), bs)
    assert np.array_equal(g_of, np.arange(len(bs)))    # no coupling: every block alone


def test_groups_need_a_finalized_matrix(gb):
    M = gb.Matrix(np.array([5, 5], dtype=np.int32))
    with pytest.raises(gb.DbcsrError) as e:
        M.groups()
    assert e.value.status == gb._ffi.DBCSR_ESTATE
