"""Multi-process helpers for the batched path (one process per GPU).

Registers of a batch are independent problems (Sec. "Batched Quantum
Registers"), so N processes split them with no data-path collective: each
rank runs the registers it owns, and only the per-register results are
gathered at the end.  The partition balances the work, which is proportional
to the amplitude count 2^n of a register, with the longest-processing-time
rule: registers in decreasing cost order, each to the currently lightest rank
(ties: lowest rank, then lowest register index), so every rank computes the
same partition without communication.

The functions take a torch.distributed process group (gloo on CPU, NCCL on
GPU); with world size 1 they reduce to local operations.
"""
from __future__ import annotations

import heapq

import numpy as np
import torch


def partition_registers(nqubits, world: int) -> list[list[int]]:
    """Register indices owned by each of `world` ranks (each list ascending)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    nq = [int(x) for x in nqubits]
    order = sorted(range(len(nq)), key=lambda r: (-nq[r], r))
    heap = [(0, rank) for rank in range(world)]
    owned: list[list[int]] = [[] for _ in range(world)]
    for r in order:
        load, rank = heapq.heappop(heap)
        owned[rank].append(r)
        heapq.heappush(heap, (load + (1 << nq[r]), rank))
    return [sorted(o) for o in owned]


def shard_cost(nqubits, owned) -> int:
    return int(sum(1 << int(nqubits[r]) for r in owned))


def gather_per_register(local_values, owned: list[int], nreg: int, group=None) -> np.ndarray:
    """Every rank passes the values of the registers it owns (same order as
    `owned`); every rank receives the full vector in register order."""
    import torch.distributed as dist
    vals = torch.as_tensor(np.asarray(local_values, dtype=np.float64)).reshape(-1)
    idx = torch.as_tensor(np.asarray(owned, dtype=np.int64)).reshape(-1)
    if vals.numel() != idx.numel():
        raise ValueError("one value per owned register")
    if not dist.is_available() or not dist.is_initialized():
        out = np.full(nreg, np.nan)
        out[idx.numpy()] = vals.numpy()
        return out
    world = dist.get_world_size(group)
    backend = dist.get_backend(group)
    dev = torch.device("cuda") if backend == "nccl" else torch.device("cpu")
    # pad to the largest shard so that all_gather sees equal sizes
    n_local = torch.tensor([idx.numel()], dtype=torch.int64, device=dev)
    sizes = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(world)]
    dist.all_gather(sizes, n_local, group=group)
    m = int(max(int(s.item()) for s in sizes))
    pv = torch.full((m,), float("nan"), dtype=torch.float64, device=dev)
    pi = torch.full((m,), -1, dtype=torch.int64, device=dev)
    pv[:vals.numel()] = vals.to(dev)
    pi[:idx.numel()] = idx.to(dev)
    gv = [torch.empty_like(pv) for _ in range(world)]
    gi = [torch.empty_like(pi) for _ in range(world)]
    dist.all_gather(gv, pv, group=group)
    dist.all_gather(gi, pi, group=group)
    out = np.full(nreg, np.nan)
    for v, i in zip(gv, gi):
        v, i = v.cpu().numpy(), i.cpu().numpy()
        keep = i >= 0
        out[i[keep]] = v[keep]
    return out


def max_over_ranks(seconds: float, group=None) -> float:
    """The slowest rank's time (a step ends when every rank has finished)."""
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return float(seconds)
    dev = torch.device("cuda") if dist.get_backend(group) == "nccl" else torch.device("cpu")
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def sum_over_ranks(value: float, group=None) -> float:
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return float(value)
    dev = torch.device("cuda") if dist.get_backend(group) == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return float(t.item())
