"""The multi-rank path of the benchmark on CPU ranks (gloo, world size 2).

Under torchrun each rank steps its own replica of the workload (groups and
problems shard with no exchange), so the only collective is the max-reduction
of the timed region; the job rate is all ranks' units over the slowest rank's
time. The reference arm runs on rank 0 only; the other ranks exit without work.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = 10.0 + 5.0 * rank          # rank 1 is the slow one
    ms = bench.max_over_ranks(ms_local, world, "cpu")
    rate = bench.job_rate(1000, world, ms)
    # reference arm: rank 0 alone works; the others return 0 at once
    args = type("A", (), {"warmup": 3, "steps": 1})()
    rc_ref = bench.run_reference(args, None, "x") if rank != 0 else 0
    out.put((rank, ms, rate, rc_ref))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_share_only_the_timing_reduction():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rate, rc_ref in res:
        assert ms == 15.0                      # the slowest rank's time on every rank
        assert rate == pytest.approx(2 * 1000 / 15e-3)
        assert rc_ref == 0
