"""Multi-rank chain sharding on CPU (gloo, world size 2): partition and gather."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

import workloads
from paper_1107_5300_gb300 import shard


def test_lpt_partition_balances_and_covers():
    costs = [shard.chain_cost(c["N"], c["L"]) for c in workloads.batched_uneven_chains(200, 3)]
    parts = shard.lpt_partition(costs, 4)
    assert sorted(i for p in parts for i in p) == list(range(200))
    loads = [sum(costs[i] for i in p) for p in parts]
    assert max(loads) <= 1.05 * (sum(costs) / 4) + max(costs)


def _compute_oracle(chains):
    from oracle import rgf as orgf
    T = [orgf.transmission(c["N"], c["L"], c["E"], 1e-8, 1e-8, -2.7,
                           workloads.anderson_onsite(c["N"], c["L"], 0.1, c["seed"]), None)
         for c in chains]
    return np.array(T), np.zeros(len(chains), dtype=np.int32)


def _chains():
    rng = np.random.default_rng(1)
    return [dict(N=int(rng.integers(3, 9)), L=int(rng.integers(1, 6)), E=float(rng.uniform(-1, 1)),
                 seed=100 + i) for i in range(9)]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    out = shard.sharded_run(_chains(), _compute_oracle)
    if rank == 0:
        q.put(out)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gather_equals_single_process():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    T2, st2 = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    T1, st1 = _compute_oracle(_chains())
    assert np.array_equal(T1, T2) and (st2 == 0).all()
