"""Host logic of the multi-rank benchmark path on CPU ranks (gloo, world 2):
each rank runs its own product (weak scaling); the job's time is the slowest
rank's, reduced with a MAX all-reduce."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = [0.5, 0.8][rank]                  # seconds each rank took for its steps
    t_max = bench.max_over_ranks(local, world, device="cpu")
    value = bench.whole_job_value(world, 10, 2.0 * 4096 ** 3, t_max)
    q.put((rank, t_max, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_time_and_weak_scaling_value():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t_max, value in out:
        assert t_max == 0.8
        assert abs(value - 2 * 10 * 2.0 * 4096 ** 3 / 0.8 / 1e9) < 1e-6 * value


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(1.25, 1) == 1.25
    assert bench.whole_job_value(1, 4, 1e9, 2.0) == 2.0
