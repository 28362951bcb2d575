"""The sharded sign iteration with the library's arithmetic on the GPU: two ranks (processes
sharing the one GPU, each multiplying only its own rows; the halo rows travel between them
through gloo on the host) against the single-rank FP64 oracle.  The ranks' kernels never wait
on one another: all exchange happens on the host between products."""
import os
import socket

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _system():
    return synth.build_hamiltonian(synth.small(40, seed=777), box=24.0)


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2003_03868_gb300 import shard
        H = _system().H
        sh = shard.Shard(H.row_ptr, H.col, rank, world)
        Hr = shard.Rows.select(H.blk_size, H.row_ptr, H.col, H.data, sh.own)
        res = shard.sign_iterate(Hr, sh, 0.0, 1e-7, 1e-9, shard.LibraryBackend(), dist)
        rp, col, data = res.P.full()
        out.put((rank, rp, col, data, res.iterations, res.residuals, res.trace_p, res.e_band))
    finally:
        dist.barrier()
        dist.destroy_process_group()


def test_two_ranks_on_the_gpu_match_the_oracle():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import torch.multiprocessing as mp
    from oracle import bsr, sign
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted((out.get(timeout=600) for _ in range(2)), key=lambda x: x[0])
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    h = _system()
    ref = sign.sign_iterate(bsr.Mat.of(h.H), 0.0, 1e-7, 1e-9)
    P = sum(bsr.to_dense(bsr.Mat(h.H.blk_size, g[1], g[2], g[3])) for g in got)
    assert all(g[4] == ref.iterations for g in got)
    np.testing.assert_allclose(got[0][5], ref.residuals, rtol=1e-8)
    rel = np.linalg.norm(P - bsr.to_dense(ref.P)) / np.linalg.norm(bsr.to_dense(ref.P))
    assert rel < 1e-11
    assert abs(got[0][7] - ref.e_band) / h.n_atoms < 1e-10
    assert got[0][6] == pytest.approx(h.n_occ, abs=1e-6)
