"""Sharding independent chains over processes (one GPU per rank).

Chains (ribbon, energy) are independent, so N ranks split the chain list with
no exchange on the data path: longest-processing-time-first assignment on the
cost KL^3 * L of each chain (KL = ceil(N/2) orbitals per column slice), each
rank evaluates its share, and one gather brings T (and status) to rank 0 in
the original chain order.  Gradients (dT/d eps per chain) travel in the same
gather; summed over chains on request (each rank sums its share first, so the
gather then carries one array per rank).
"""
from __future__ import annotations

import heapq

import numpy as np


def chain_cost(N: int, L: int) -> float:
    KL = (N + 1) // 2
    return float(KL) ** 3 * L


def lpt_partition(costs, nranks: int):
    """Assign chains to ranks, largest first to the least-loaded rank.  Returns lists of indices."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(nranks)]
    parts = [[] for _ in range(nranks)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return [sorted(p) for p in parts]


def sharded_run(chains, compute, group=None, with_grad=False, sum_grad=False):
    """Evaluate ``compute(list_of_chains)`` over all ranks.

    ``chains``: the same list on every rank, each item a dict with at least N, L.
    ``compute`` returns (T array, status array), and with ``with_grad`` also a
    list of per-chain gradient arrays.  Returns on rank 0 (None on the others):
    (T, status), or (T, status, grads) with grads the per-chain list in chain
    order, or with ``sum_grad`` their sum (all chains of one ribbon shape).
    """
    import torch.distributed as dist

    rank = dist.get_rank(group) if dist.is_initialized() else 0
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    parts = lpt_partition([chain_cost(c["N"], c["L"]) for c in chains], world)
    mine = parts[rank]
    grads = None
    if mine:
        out = compute([chains[i] for i in mine])
        T, st = out[0], out[1]
        if with_grad:
            grads = [np.asarray(g, dtype=np.float64) for g in out[2]]
    else:
        T, st = np.empty(0), np.empty(0, dtype=np.int32)
        if with_grad:
            grads = []
    if with_grad and sum_grad:
        grads = np.sum(grads, axis=0) if grads else None
    local = (mine, np.asarray(T, dtype=np.float64), np.asarray(st, dtype=np.int32), grads)
    if world == 1:
        gathered = [local]
    else:
        gathered = [None] * world if rank == 0 else None
        dist.gather_object(local, gathered, dst=0, group=group)
    if rank != 0:
        return None
    T_all = np.full(len(chains), np.nan)
    st_all = np.full(len(chains), -1, dtype=np.int32)
    for idx, T, st, _ in gathered:
        T_all[idx] = T
        st_all[idx] = st
    if not with_grad:
        return T_all, st_all
    if sum_grad:
        parts_sum = [g for _, _, _, g in gathered if g is not None]
        return T_all, st_all, (np.sum(parts_sum, axis=0) if parts_sum else None)
    g_all = [None] * len(chains)
    for idx, _, _, g in gathered:
        for i, gi in zip(idx, g):
            g_all[i] = gi
    return T_all, st_all, g_all
