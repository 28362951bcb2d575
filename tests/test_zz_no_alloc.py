"""The allocation-free trace entry point, for callers that may not allocate
device memory during a call (their own arena owns the GPU memory, or they record
a CUDA graph that must not contain allocations).

It must return what dbcsr_trace_product returns, call after call, although
every call reuses the same fixed scratch array inside the library.  This file
sorts last so that a stop-at-first-failure run has already run everything else.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2003_03868_gb300 as m
    m.lib()
    return m


def _noalloc(gb, A, B):
    import torch
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    gb.trace_product_noalloc(A, B, out.data_ptr())
    torch.cuda.synchronize()
    return float(out.item())


def test_matches_trace_product_twice_in_a_row(gb):
    # two different products one after the other: the second call must not see the first's scratch
    bs = [13, 5, 5] * 20
    a = synth.random_block_matrix(bs, 0.5, 7001)
    b = synth.random_block_matrix(bs, 0.5, 7002)
    A, B = gb.Matrix.of(a), gb.Matrix.of(b)
    d = gb.Matrix.of(synth.build_decay(synth.DECAY_32))
    ref_ab = gb.trace_product(A, B)
    ref_dd = gb.trace_product(d, d)
    for _ in range(2):
        got_ab = _noalloc(gb, A, B)
        got_dd = _noalloc(gb, d, d)
        assert got_ab == pytest.approx(ref_ab, rel=1e-12, abs=1e-12)
        assert got_dd == pytest.approx(ref_dd, rel=1e-12, abs=1e-12)


def test_empty_matrix_gives_zero(gb):
    bs = [5, 13, 5]
    Z = gb.Matrix.of(synth.random_block_matrix(bs, 0.0, 7003, diag=False))
    A = gb.Matrix.of(synth.random_block_matrix(bs, 1.0, 7004))
    assert _noalloc(gb, Z, A) == 0.0


def test_rejects_more_blocks_than_the_scratch_holds(gb):
    # 1,100 x 1,100 blocks of edge 1 (1.21M blocks) exceed the 1,048,576-block limit
    n = 1100
    bm = synth.random_block_matrix([1] * n, 1.0, 7005)
    A = gb.Matrix.of(bm)
    import torch
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(gb.DbcsrError) as e:
        gb.trace_product_noalloc(A, A, out.data_ptr())
    assert e.value.status == 3                     # DBCSR_ECAPACITY
    assert "1048576" in str(e.value)
    assert out.item() == 0.0                       # nothing was launched


def test_allocates_nothing_and_replays_in_a_cuda_graph(gb):
    # the stated purpose: no pool allocation during a call (the high-water mark of the
    # library's pool stays at its use before the call), and a call recorded in a CUDA graph
    # replays with the values A holds at replay time
    import torch
    s = torch.cuda.Stream()
    bs = [13, 5, 5] * 12
    a = synth.random_block_matrix(bs, 0.5, 7011)
    b = synth.random_block_matrix(bs, 0.5, 7012)
    A = gb.Matrix.of(a, stream=s.cuda_stream)
    B = gb.Matrix.of(b, stream=s.cuda_stream)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    gb.trace_product_noalloc(A, B, out.data_ptr())          # warm-up (module load)
    s.synchronize()
    now0, _ = gb.pool_usage(reset_high=True)
    gb.trace_product_noalloc(A, B, out.data_ptr())
    s.synchronize()
    now1, high1 = gb.pool_usage()
    assert now1 == now0 and high1 == now0
    assert float(out.item()) == pytest.approx(gb.trace_product(A, B), rel=1e-12, abs=1e-12)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        gb.trace_product_noalloc(A, B, out.data_ptr())
    rng = np.random.default_rng(7013)
    for _ in range(2):
        vals = rng.uniform(-1.0, 1.0, a.data.shape[0])
        A.put_values(vals)
        s.synchronize()
        out.fill_(float("nan"))
        torch.cuda.synchronize()
        now_r, _ = gb.pool_usage(reset_high=True)
        g.replay()
        s.synchronize()
        torch.cuda.synchronize()
        now_a, high = gb.pool_usage()
        assert now_a == now_r and high == now_r            # the replay allocated nothing
        assert float(out.item()) == pytest.approx(gb.trace_product(A, B), rel=1e-12, abs=1e-12)
