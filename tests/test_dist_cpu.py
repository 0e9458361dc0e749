"""The N > 1 path on CPU: gloo process groups of world size 2 (and 3) run the
register partition, the per-register gather and the max-over-ranks timing
that the batched multi-GPU runs use; no GPU and no data-path collective."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1912_10877_gb300 import dist as D


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_partition_is_a_balanced_cover():
    rs = np.random.default_rng(0)
    nq = rs.integers(10, 19, 1024)
    for world in (1, 2, 3, 4, 8):
        parts = D.partition_registers(nq, world)
        flat = sorted(r for p in parts for r in p)
        assert flat == list(range(len(nq)))
        costs = [D.shard_cost(nq, p) for p in parts]
        # LPT bound: the heaviest shard exceeds the mean by at most the largest item
        assert max(costs) <= sum(costs) / world + (1 << int(nq.max()))
    assert D.partition_registers([5, 3], 4)[2:] == [[], []]


def _worker(rank, world, port, nq, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        parts = D.partition_registers(nq, world)
        mine = parts[rank]
        # each rank "computes" a per-register value from the register index alone
        vals = [np.sin(r) * nq[r] for r in mine]
        full = D.gather_per_register(vals, mine, len(nq))
        t = D.max_over_ranks(0.5 + rank)
        s = D.sum_over_ranks(D.shard_cost(nq, mine))
        np.save(os.path.join(out_dir, f"r{rank}.npy"), np.concatenate([full, [t, s]]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_gather_every_register(tmp_path, world):
    rs = np.random.default_rng(world)
    nq = [int(x) for x in rs.integers(10, 19, 37)]
    mp.start_processes(_worker, args=(world, free_port(), nq, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    want = np.array([np.sin(r) * nq[r] for r in range(len(nq))])
    for rank in range(world):
        got = np.load(tmp_path / f"r{rank}.npy")
        assert np.allclose(got[:-2], want, rtol=0, atol=0)
        assert got[-2] == 0.5 + (world - 1)
        assert got[-1] == sum(1 << q for q in nq)


def test_single_process_fallbacks():
    assert not dist.is_initialized()
    out = D.gather_per_register([1.0, 2.0], [2, 0], 3)
    assert out[0] == 2.0 and out[2] == 1.0 and np.isnan(out[1])
    assert D.max_over_ranks(1.5) == 1.5
