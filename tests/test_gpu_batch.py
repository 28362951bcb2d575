"""Batched sign iteration (many uneven systems in one block-diagonal batch) against
the FP64 oracle per system and against the single-system GPU path."""
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


def _systems(n, seed):
    out = []
    rng = np.random.default_rng(seed)
    bases = [(13, 5), (23, 7), (13, 7), (23, 5)]
    for s in range(n):
        w = synth.small(int(rng.integers(6, 40)), basis=bases[s % 4], seed=seed * 100 + s)
        out.append(synth.build_hamiltonian(w))
    return out


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_matches_oracle_per_system(gb, prec):
    hs = _systems(6, 17)
    Hs = [gb.Matrix.of(h.H) for h in hs]
    p = gb.DBCSR_FP64 if prec == "fp64" else gb.DBCSR_MIXED
    Ps, reps, st = gb.sign_iterate_batched(Hs, [0.0] * len(hs), 1e-7, 1e-8, prec=p)
    for h, P, r in zip(hs, Ps, reps):
        o = sign.sign_iterate(bsr.Mat.of(h.H), 0.0, 1e-7, 1e-8)
        assert r.alpha == pytest.approx(o.alpha, rel=1e-15)
        assert r.converged or r.stalled
        assert abs(r.e_band - o.e_band) / h.n_atoms < (1e-7 if prec == "fp64" else DE_ATOM)
        assert r.trace_p == pytest.approx(h.n_occ, abs=1e-5)
        if prec == "fp64":
            assert r.iterations == o.iterations
            # above the rounding floor (~1e-11 here) the residuals agree to 1e-6
            np.testing.assert_allclose([r.residual_history[i] for i in range(r.iterations)], o.residuals,
                                       rtol=1e-6, atol=1e-10)
        rp, col, data = P.export()
        assert rp.shape[0] == h.H.nblk + 1


def test_batch_equals_single_system_runs(gb):
    # the systems finish at different steps and leave the batch one after another; every
    # block product of a system is the same sum in the same order as in its own run, so
    # the FP64 density matrices agree bit for bit
    hs = _systems(5, 23)
    Hs = [gb.Matrix.of(h.H) for h in hs]
    # mu near a band edge (the gap is [-0.25, 0.25]) slows a system down
    mus = [0.0, 0.2, 0.0, -0.22, 0.1]
    Ps, reps, st = gb.sign_iterate_batched(Hs, mus, 1e-7, 1e-9)
    its = set()
    for h, H, P, r, mu in zip(hs, Hs, Ps, reps, mus):
        g = gb.sign_iterate(H, mu, 1e-7, 1e-9)
        assert abs(r.e_band - g.report.e_band) / h.n_atoms < 1e-9
        assert r.iterations == g.report.iterations
        its.add(r.iterations)
        for a, b in zip(P.export(), g.P.export()):
            assert np.array_equal(a, b)
    assert len(its) > 1


def test_batch_stopped_by_max_iter(gb):
    hs = _systems(3, 31)
    Hs = [gb.Matrix.of(h.H) for h in hs]
    Ps, reps, st = gb.sign_iterate_batched(Hs, [0.0] * len(hs), 1e-7, 1e-12, max_iter=3)
    assert st == gb._ffi.DBCSR_ENOTCONV
    for h, H, P, r in zip(hs, Hs, Ps, reps):
        assert r.iterations == 3 and not r.converged and not r.stalled
        g = gb.sign_iterate(H, 0.0, 1e-7, 1e-12, max_iter=3)
        for a, b in zip(P.export(), g.P.export()):
            assert np.array_equal(a, b)


def test_batch_of_one_and_different_mu(gb):
    h = _systems(1, 29)[0]
    H = gb.Matrix.of(h.H)
    Ps, reps, st = gb.sign_iterate_batched([H, H], [0.0, 0.1], 0.0, 1e-11)
    # mu anywhere in the gap gives the same projector
    assert abs(reps[0].e_band - reps[1].e_band) < 1e-8
    assert reps[0].alpha != reps[1].alpha


@pytest.fixture
def queue_schedule(gb):
    gb.set_fp64_schedule(gb.DBCSR_SCHEDULE_QUEUE)
    yield
    gb.set_fp64_schedule(gb.DBCSR_SCHEDULE_PER_SHAPE)


def test_one_launch_schedule_sums_like_the_per_shape_launches(gb):
    # every C element is the same sum in the same order: only the norms of warp-pair classes
    # (per-shape schedule) may round differently
    a = synth.random_block_matrix([13, 5, 5, 23, 7, 7, 1, 32] * 3, 0.6, 41)
    b = synth.random_block_matrix([13, 5, 5, 23, 7, 7, 1, 32] * 3, 0.6, 42)
    A, B = gb.Matrix.of(a), gb.Matrix.of(b)
    out = {}
    for mode in (gb.DBCSR_SCHEDULE_PER_SHAPE, gb.DBCSR_SCHEDULE_QUEUE):
        gb.set_fp64_schedule(mode)
        C = gb.Matrix(A.blk_size, A.stream)
        st = gb.multiply(1.0, A, B, 0.0, C, 0.0)
        out[mode] = (C.export(), st.n_launches)
    gb.set_fp64_schedule(gb.DBCSR_SCHEDULE_PER_SHAPE)
    (rp0, c0, d0), n0 = out[gb.DBCSR_SCHEDULE_PER_SHAPE]
    (rp1, c1, d1), n1 = out[gb.DBCSR_SCHEDULE_QUEUE]
    assert np.array_equal(rp0, rp1) and np.array_equal(c0, c1) and np.array_equal(d0, d1)
    # the small shapes share one launch; the shapes with more than 9 slots per lane keep theirs
    big = sum(1 for m in (13, 5, 23, 7, 1, 32) for n in (13, 5, 23, 7, 1, 32) if (m * n + 31) // 32 > 9)
    assert n1 == 1 + big and n0 > n1
    ref = bsr.multiply(1.0, bsr.Mat.of(a), bsr.Mat.of(b))
    np.testing.assert_allclose(d1, ref.data, rtol=0, atol=1e-12 * np.abs(ref.data).max())


def test_batch_equals_single_runs_with_the_one_launch_schedule(gb, queue_schedule):
    hs = _systems(5, 23)
    Hs = [gb.Matrix.of(h.H) for h in hs]
    mus = [0.0, 0.2, 0.0, -0.22, 0.1]
    Ps, reps, st = gb.sign_iterate_batched(Hs, mus, 1e-7, 1e-9)
    for h, H, P, r, mu in zip(hs, Hs, Ps, reps, mus):
        g = gb.sign_iterate(H, mu, 1e-7, 1e-9)
        o = sign.sign_iterate(bsr.Mat.of(h.H), mu, 1e-7, 1e-9)
        assert abs(r.e_band - o.e_band) / h.n_atoms < 1e-7
        assert r.iterations == g.report.iterations
        for a, b in zip(P.export(), g.P.export()):
            assert np.array_equal(a, b)
