"""The exchange step of a census split over ranks (the 128-bit sums as
carried 32-bit limbs), on CPU: world size 2 and 3 over gloo, with values
chosen so that every limb carries and the totals wrap modulo 2^128."""
import os
import random
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1610_09411_gb300 import shard  # noqa: E402

M128 = 1 << 128

VALUES = {
    0: [2**64 - 1, M128 - 1, 2**96 + 2**32 - 1, 0, 2**127, 12345678901234567890123456789],
    1: [1, 1, 2**32 + 1, M128 - 1, 2**127, 98765432109876543210987654321],
    2: [2**32 - 1, 2**64, 2**95, 7, 1, 2**126 + 5],
}


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
    out[rank] = shard.allreduce_u128(VALUES[rank], device="cpu")
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_allreduce_u128_with_carries(world):
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    want = [sum(VALUES[r][i] for r in range(world)) % M128 for i in range(len(VALUES[0]))]
    for r in range(world):
        assert out[r] == want


def test_limbs_round_trip_and_sum_locally():
    rng = random.Random(7)
    parts = [[rng.getrandbits(128) for _ in range(40)] for _ in range(50)]
    limb_sum = [sum(col) for col in zip(*(shard.to_limbs(p) for p in parts))]
    assert max(limb_sum) < 2**63
    assert shard.from_limbs(limb_sum) == [sum(col) % M128 for col in zip(*parts)]
    v = [0, 1, M128 - 1, 2**64, 3 * 2**96 + 17]
    assert shard.from_limbs(shard.to_limbs(v)) == v
