"""The N > 1 timing of bench.py on CPU: world size 2 over gloo; the job time
is the slowest rank's, and the ranks together count one graph per step."""
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


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 + 50.0 * rank            # rank 1 is the slow one
    total = bench.slowest_rank_ms(local_ms, world, "cpu")
    out[rank] = (total, bench.job_value(1_000_000, total / 5))
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0][0] == out[1][0] == 150.0
    # one graph of 1e6 edges every 30 ms
    assert abs(out[0][1] - 1_000_000 / 0.030) < 1e-6


def test_single_rank_is_unchanged():
    import bench
    assert bench.slowest_rank_ms(42.0, 1, "cpu") == 42.0
    assert bench.job_value(10, 1.0) == 10_000.0
