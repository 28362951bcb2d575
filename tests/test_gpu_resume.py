"""Checkpoint and resume of the sign iteration: a run stopped after k steps with its X returned
(DBCSR_SIGN_RETURN_X), written to a matrix file and read back, continued by
dbcsr_sign_iterate_resume, must give the uninterrupted run's P -- bit for bit in FP64 and after
the mixed ladder's switch to FP64 (the same products on the same operands), to rounding when
resumed inside the split-BF16 tier (the tensor-core tier regroups the blocks of X)."""
import numpy as np
import pytest

import synth
from oracle import bsr, sign

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2003_03868_gb300 as m
    m.lib()
    return m


@pytest.fixture(scope="module")
def system():
    return synth.build_hamiltonian(synth.small(48, basis=(23, 7), seed=8301))


def _history(rep):
    n = rep.iterations
    return [rep.residual_history[i] for i in range(n)], [rep.nnzb_history[i] for i in range(n)]


def _checkpoint(gb, H, k, tmp_path, **kw):
    first = gb.sign_iterate(H, 0.0, 1e-7, 1e-9, max_iter=k, return_x=True, **kw)
    assert first.report.iterations == k and not first.report.converged
    assert np.isnan(first.report.e_band)
    path = str(tmp_path / f"x_{k}.dbcsr")
    first.P.save(path)
    return gb.Matrix.load(path, stream=H.stream), first.report


@pytest.mark.parametrize("k", [1, 3, 5])
def test_fp64_resume_is_bit_identical(gb, system, tmp_path, k):
    H = gb.Matrix.of(system.H)
    full = gb.sign_iterate(H, 0.0, 1e-7, 1e-9)
    assert full.report.iterations > k
    X, prev = _checkpoint(gb, H, k, tmp_path)
    res = gb.sign_iterate_resume(H, X, prev, 1e-7, 1e-9)
    assert res.report.iterations == full.report.iterations
    assert bool(res.report.converged) == bool(full.report.converged)
    assert _history(res.report) == _history(full.report)
    for a, b in zip(res.P.export(), full.P.export()):
        assert np.array_equal(a, b)
    assert res.report.e_band == full.report.e_band
    assert res.report.flops == full.report.flops              # prev's totals carried on
    # X itself was not touched by the resumed run
    X2, _ = _checkpoint(gb, H, k, tmp_path)
    for a, b in zip(X.export(), X2.export()):
        assert np.array_equal(a, b)


def test_mixed_resume_after_the_switch_is_bit_identical(gb, system, tmp_path):
    H = gb.Matrix.of(system.H)
    kw = dict(prec=gb.DBCSR_MIXED, switch_tol=1e-4)
    full = gb.sign_iterate(H, 0.0, 1e-7, 1e-9, **kw)
    f = full.report.fp64_from
    assert 2 <= f < full.report.iterations
    for k in (f - 1, f):                  # the next X*X is an FP64 product in both
        X, prev = _checkpoint(gb, H, k, tmp_path, **kw)
        assert prev.fp64_from == (f if k >= f - 1 else 0)
        res = gb.sign_iterate_resume(H, X, prev, 1e-7, 1e-9, **kw)
        assert res.report.fp64_from == f
        assert res.report.iterations == full.report.iterations
        assert _history(res.report) == _history(full.report)
        for a, b in zip(res.P.export(), full.P.export()):
            assert np.array_equal(a, b)


def test_mixed_resume_inside_the_low_tier_agrees_with_the_oracle(gb, system, tmp_path):
    H = gb.Matrix.of(system.H)
    kw = dict(prec=gb.DBCSR_MIXED, switch_tol=1e-4)
    X, prev = _checkpoint(gb, H, 2, tmp_path, **kw)
    assert prev.fp64_from == 0
    res = gb.sign_iterate_resume(H, X, prev, 1e-7, 1e-9, **kw)
    assert res.report.converged or res.report.stalled
    o = sign.sign_iterate(bsr.Mat.of(system.H), 0.0, 1e-7, 1e-9)
    assert abs(res.report.e_band - o.e_band) / system.n_atoms < 1e-6
    assert res.report.trace_p == pytest.approx(system.n_occ, abs=1e-5)


def test_resume_checks_its_arguments(gb, system, tmp_path):
    H = gb.Matrix.of(system.H)
    X, prev = _checkpoint(gb, H, 1, tmp_path)
    other = gb.Matrix.of(synth.random_block_matrix([5, 13] * 3, 0.5, 8302))
    with pytest.raises(gb.DbcsrError) as e:
        gb.sign_iterate_resume(H, other, prev, 1e-7, 1e-9)
    assert e.value.status == gb._ffi.DBCSR_EINVAL
    bad = gb._ffi.SignReport()
    bad.iterations = -1
    with pytest.raises(gb.DbcsrError) as e:
        gb.sign_iterate_resume(H, X, bad, 1e-7, 1e-9)
    assert e.value.status == gb._ffi.DBCSR_EINVAL
