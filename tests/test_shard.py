"""The sign iteration sharded over ranks by domains of block rows (host logic, CPU): the
domain partition and halo lists against brute force, and two gloo ranks running the sharded
driver with the oracle's arithmetic against the single-rank oracle iteration."""
import os
import socket

import numpy as np
import pytest

import synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _system(n_mol=40, box=24.0, seed=777):
    """A dilute water box: its block graph is sparse, so domains and halos are meaningful."""
    return synth.build_hamiltonian(synth.small(n_mol, seed=seed), box=box)


@pytest.fixture(scope="module")
def shard():
    from paper_2003_03868_gb300 import build
    build.build()
    from paper_2003_03868_gb300 import shard as m
    return m


@pytest.mark.parametrize("world", [1, 2, 3, 4])
def test_partition_covers_every_row_with_balanced_domains(shard, world):
    H = _system().H
    owner = shard.partition_rows(H.row_ptr, H.col, world)
    assert owner.shape == (H.blk_size.shape[0],) and owner.min() >= 0 and owner.max() < world
    load = np.bincount(owner, weights=np.diff(H.row_ptr) + 1.0, minlength=world)
    assert load.min() > 0 and load.max() / load.mean() < 1.5
    assert np.array_equal(owner, shard.partition_rows(H.row_ptr, H.col, world))   # deterministic


@pytest.mark.parametrize("world", [2, 4])
def test_domains_have_smaller_halos_than_index_ranges(shard, world):
    # atoms are numbered in random molecule order, so index ranges are scattered in space;
    # the graph domains exchange fewer rows per product
    H = _system(96, 40.0, 31).H
    nb = H.blk_size.shape[0]
    owner = shard.partition_rows(H.row_ptr, H.col, world)
    ranges = (np.arange(nb) * world // nb).astype(np.int32)
    halo = sum(len(shard.halo_rows(H.row_ptr, H.col, owner, r)) for r in range(world))
    halo_ranges = sum(len(shard.halo_rows(H.row_ptr, H.col, ranges, r)) for r in range(world))
    assert halo < 0.8 * halo_ranges, (halo, halo_ranges)


def test_halo_lists_are_the_foreign_columns_of_the_own_rows(shard):
    H = _system().H
    owner = shard.partition_rows(H.row_ptr, H.col, 3)
    for r in range(3):
        want = sorted({int(c) for i in np.nonzero(owner == r)[0]
                       for c in H.col[H.row_ptr[i]:H.row_ptr[i + 1]] if owner[c] != r})
        assert shard.halo_rows(H.row_ptr, H.col, owner, r).tolist() == want


def test_partition_rejects_bad_arguments(shard):
    H = _system().H
    with pytest.raises(RuntimeError):
        shard.partition_rows(H.row_ptr, H.col, 0)
    bad = H.col.copy()
    bad[0] = H.blk_size.shape[0]
    with pytest.raises(RuntimeError):
        shard.partition_rows(H.row_ptr, bad, 2)


class OracleBackend:
    """The oracle's FP64 arithmetic on a rank's rows (test infrastructure)."""

    def _mat(self, R):
        from oracle import bsr
        rp, col, data = R.full()
        return bsr.Mat(R.bs, rp, col, data)

    def gershgorin(self, R, mu):
        from oracle import bsr
        sums = bsr.abs_row_sums(self._mat(R), mu)
        roff = np.concatenate([[0], np.cumsum(R.bs)])
        return float(max(sums[roff[I]:roff[I + 1]].max() for I in R.rows))

    def add_identity(self, R, scale, shift):
        from paper_2003_03868_gb300.shard import Rows
        M = self._mat(R)
        M.data = M.data * scale
        for I in R.rows:
            M.block(int(I), int(I))[np.diag_indices(int(R.bs[I]))] += shift
        return Rows.select(R.bs, M.rp, M.col, M.data, R.rows)

    def multiply(self, alpha, A, B, eps):
        from oracle import bsr
        from paper_2003_03868_gb300.shard import Rows
        Cm, info = bsr.multiply(alpha, self._mat(A), self._mat(B), eps=eps, info=True)
        _, d2 = bsr.block_norms(Cm)
        return Rows.select(A.bs, Cm.rp, Cm.col, Cm.data, A.rows), float(d2.sum()), float(info.flops)


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2003_03868_gb300 import shard
        H = _system().H
        sh = shard.Shard(H.row_ptr, H.col, rank, world)
        Hr = shard.Rows.select(H.blk_size, H.row_ptr, H.col, H.data, sh.own)
        res = shard.sign_iterate(Hr, sh, 0.0, 1e-7, 1e-9, OracleBackend(), dist)
        rp, col, data = res.P.full()
        out.put((rank, rp, col, data, res.iterations, res.residuals, res.alpha, res.trace_p, res.e_band,
                 res.halo_rows, len(sh.own)))
    finally:
        dist.barrier()
        dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_single_rank_oracle_iteration():
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    from oracle import bsr, sign
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted((out.get(timeout=300) for _ in range(2)), key=lambda x: x[0])
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    h = _system()
    ref = sign.sign_iterate(bsr.Mat.of(h.H), 0.0, 1e-7, 1e-9)
    P = sum(bsr.to_dense(bsr.Mat(h.H.blk_size, g[1], g[2], g[3])) for g in got)
    assert all(g[4] == ref.iterations for g in got)
    np.testing.assert_allclose(got[0][5], ref.residuals, rtol=1e-10)
    assert got[0][6] == ref.alpha
    assert np.abs(P - bsr.to_dense(ref.P)).max() < 1e-12
    assert got[0][7] == pytest.approx(ref.trace_p, abs=1e-10)
    assert got[0][8] == pytest.approx(ref.e_band, abs=1e-10)
    # each rank held only its rows of P, and rows did travel between the ranks
    rows = [set(np.nonzero(np.diff(g[1]))[0].tolist()) for g in got]
    assert rows[0] and rows[1] and not rows[0] & rows[1]
    assert all(0 < g[9] < h.H.blk_size.shape[0] - g[10] + 1 for g in got)
