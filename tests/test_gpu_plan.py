"""Planned products on fixed patterns (dbcsr_multiply_plan / dbcsr_multiply_execute, a
CUDA graph of the numeric phase) against the one-off product and the oracle."""
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


def _mat(M):
    rp, col, data = M.export()
    return bsr.Mat(M.blk_size, rp, col, data)


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_plan_equals_one_off_product(gb, prec):
    p = gb.DBCSR_FP64 if prec == "fp64" else gb.DBCSR_BF16X3
    a = synth.build_decay(synth.DECAY_32)
    eps = synth.DECAY_32.eps_filter
    A = gb.Matrix.of(a)
    C1 = gb.Matrix(A.blk_size, A.stream)
    gb.multiply(1.0, A, A, 0.0, C1, eps, prec=p)
    ref = _mat(C1)
    C2 = gb.Matrix(A.blk_size, A.stream)
    plan = gb.Plan(1.0, A, A, C2, eps, prec=p)
    for _ in range(3):              # the planned pattern holds every formed block, under-eps ones zeroed
        got = _mat(C2)
        kept = {(int(r), int(c)) for r, c in zip(ref.rows, ref.col)}
        for b in range(got.nnzb):
            I, J = int(got.rows[b]), int(got.col[b])
            blk = got.block(I, J)
            if (I, J) in kept:
                assert np.array_equal(blk, ref.block(I, J))
            else:
                assert I != J and not blk.any()
        assert kept <= {(int(r), int(c)) for r, c in zip(got.rows, got.col)}
        plan.execute()
    assert plan.stats.n_formed == got.nnzb
    plan.close()


def test_plan_with_new_values_matches_oracle(gb):
    a = synth.build_decay(synth.DECAY_32)
    eps = synth.DECAY_32.eps_filter
    A = gb.Matrix.of(a)
    B = gb.Matrix.of(a)
    C_ = gb.Matrix(A.blk_size, A.stream)
    plan = gb.Plan(-0.5, A, B, C_, eps)
    rng = np.random.default_rng(7)
    for step in range(3):
        # new values on the same patterns
        av = a.data * (0.8 + 0.4 * rng.random(a.data.shape))
        bv = a.data * (0.8 + 0.4 * rng.random(a.data.shape))
        A.put_values(av)
        B.put_values(bv)
        plan.execute()
        Ao = bsr.Mat(a.blk_size, a.row_ptr, a.col, av)
        Bo = bsr.Mat(a.blk_size, a.row_ptr, a.col, bv)
        got = _mat(C_)
        for b in range(got.nnzb):
            I, J = int(got.rows[b]), int(got.col[b])
            r = bsr.product_block(I, J, -0.5, Ao, Bo)
            nr = np.linalg.norm(r)
            if I != J and nr < eps * (1 - 1e-12):
                assert not got.block(I, J).any()
            elif I == J or nr > eps * (1 + 1e-12):
                assert np.linalg.norm(got.block(I, J) - r) <= 1e-12 * nr
    plan.close()


def test_plan_pins_its_matrices(gb):
    a = synth.random_block_matrix([13, 5, 5] * 4, 0.5, 11)
    A = gb.Matrix.of(a)
    C_ = gb.Matrix(A.blk_size, A.stream)
    plan = gb.Plan(1.0, A, A, C_, 0.0)
    with pytest.raises(gb.DbcsrError) as e:
        gb.multiply(1.0, A, A, 0.0, C_, 0.0)
    assert e.value.status == gb._ffi.DBCSR_ESTATE
    with pytest.raises(gb.DbcsrError):
        C_.filter(1.0)
    with pytest.raises(gb.DbcsrError):
        A.close()
    with pytest.raises(gb.DbcsrError):          # C may not alias an operand
        gb.Plan(1.0, A, A, A, 0.0)
    plan.close()
    gb.multiply(1.0, A, A, 0.0, C_, 0.0)         # free again once the plan is gone
    A.close()
