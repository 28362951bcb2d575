"""Runs on several GPUs, host side: the whole-job timing reduction over ranks (gloo, two
processes on the CPU) and the per-rank system sets of the batched solve."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2003_03868_gb300 import ranks
    ms, fl = ranks.job_timing(10.0 + 3.0 * rank, 100.0 * (rank + 1), dist, "cpu")
    out.put((rank, ms, fl))
    dist.barrier()
    dist.destroy_process_group()


def test_job_timing_is_max_time_and_total_work_over_two_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(out.get(timeout=10) for _ in range(2))
    assert got == [(0, 13.0, 300.0), (1, 13.0, 300.0)]


def test_job_timing_without_a_process_group():
    from paper_2003_03868_gb300 import ranks
    assert ranks.job_timing(5.0, 7.0) == (5.0, 7.0)


def test_each_rank_solves_its_own_systems():
    import synth
    a = synth.batch_systems(seed=synth.batch_seed(0))
    b = synth.batch_systems(seed=synth.batch_seed(1))
    assert [w.seed for w in a] == [w.seed for w in synth.batch_systems(seed=synth.batch_seed(0))]
    assert not set(w.seed for w in a) & set(w.seed for w in b)
    assert [(w.n_mol, w.basis) for w in a] != [(w.n_mol, w.basis) for w in b]
    assert all(100 <= w.n_mol <= 2000 for w in a + b)
    # rank 0 keeps the single-GPU batch
    assert [w.seed for w in a] == [w.seed for w in synth.batch_systems()]
