"""Host logic of the benchmark's multi-rank mode, on two gloo ranks (CPU)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r pretends its timed region took (1 + r) s and its e2e loop (3 - r) s
    t_max, e2e_max = bench.max_over_ranks([1.0 + rank, 3.0 - rank], world)
    out[rank] = (t_max, e2e_max, bench.job_throughput(world, 10, 100, t_max))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_and_job_rate(repo_root):
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    os.environ.setdefault("PYTHONPATH", repo_root)
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        t_max, e2e_max, rate = out[r]
        assert t_max == 2.0 and e2e_max == 3.0
        assert rate == pytest.approx(2 * 10 * 100 / 2.0)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks([0.5, 0.25], 1) == [0.5, 0.25]
    assert bench.job_throughput(1, 1000, 819250, 0.0141) == pytest.approx(1000 * 819250 / 0.0141)
