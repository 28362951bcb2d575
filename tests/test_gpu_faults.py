"""Failure detection without a GPU fault: a bounded device-side wait that runs out returns
DBCSR_ETIMEOUT and leaves the context usable; non-finite input stops the sign iteration with a
status instead of a result.  Nothing here traps, faults or hangs the GPU: the wait self-test
waits on a barrier that nothing arrives on, for a short cycle limit, with no copy in flight."""
import ctypes as C

import numpy as np
import pytest

import synth
from oracle import bsr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2003_03868_gb300 as m
    m.lib()
    return m


def test_bounded_wait_runs_out_and_the_context_stays_usable(gb):
    lib = gb.lib()
    waited = C.c_int64(0)
    limit = 2_000_000                                   # about a millisecond of SM cycles
    st = lib.dbcsr_wait_selftest(limit, 0, C.byref(waited))
    assert st == gb._ffi.DBCSR_ETIMEOUT
    assert waited.value >= limit
    assert b"ran out" in lib.dbcsr_last_error()
    # a wait whose barrier completes returns at once
    st = lib.dbcsr_wait_selftest(limit, 1, C.byref(waited))
    assert st == gb._ffi.DBCSR_OK and waited.value < limit
    # the context still computes: a product against the oracle
    a = synth.random_block_matrix([13, 5, 5] * 4, 0.5, 8101)
    A = gb.Matrix.of(a)
    Cm = gb.Matrix(A.blk_size, A.stream)
    gb.multiply(1.0, A, A, 0.0, Cm, 0.0)
    ref = bsr.multiply(1.0, bsr.Mat.of(a), bsr.Mat.of(a))
    rp, col, data = Cm.export()
    assert np.array_equal(col, ref.col)
    np.testing.assert_allclose(data, ref.data, rtol=0, atol=1e-12 * np.abs(ref.data).max())


def test_negative_wait_limit_is_rejected(gb):
    st = gb.lib().dbcsr_wait_selftest(-1, 0, None)
    assert st == gb._ffi.DBCSR_EINVAL


@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_non_finite_hamiltonian_stops_the_sign_iteration(gb, bad):
    # one non-finite element of an off-diagonal block: the Gershgorin bound is not finite, so
    # the iteration refuses to start (DBCSR_EINVAL) instead of returning a meaningless P
    h = synth.build_hamiltonian(synth.small(8, seed=8102))
    H0 = h.H
    data = H0.data.copy()
    q = int(np.nonzero(H0.rows() != H0.col)[0][0])         # first off-diagonal block
    data[int(H0.blk_off()[q])] = bad
    H = gb.Matrix.from_blocks(H0.blk_size, H0.row_ptr, H0.col, data)
    with pytest.raises(gb.DbcsrError) as e:
        gb.sign_iterate(H, 0.0, 1e-7, 1e-9)
    assert e.value.status in (gb._ffi.DBCSR_EINVAL, gb._ffi.DBCSR_ENAN)
    assert "not finite" in str(e.value)

