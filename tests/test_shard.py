"""Multi-rank chain sharding on CPU (gloo, world size 2): partition and gather
of T, status and gradients."""
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


def _compute_oracle_grad(chains):
    from oracle import gradient as ograd
    out = [ograd.two_sided(c["N"], c["L"], c["E"], 1e-8, 1e-8, -2.7,
                           workloads.anderson_onsite(c["N"], c["L"], 0.1, c["seed"]), None)
           for c in chains]
    return (np.array([o[0] for o in out]), np.zeros(len(chains), dtype=np.int32),
            [o[1] for o in out])


def _grad_chains():
    # one ribbon shape (N = 5, L = 3), several energies and disorder seeds
    return [dict(N=5, L=3, E=float(e), seed=200 + i)
            for i, e in enumerate(np.linspace(-0.9, 0.8, 7))]


def _chains():
    rng = np.random.default_rng(1)
    return [dict(N=int(rng.integers(3, 9)), L=int(rng.integers(1, 6)), E=float(rng.uniform(-1, 1)),
                 seed=100 + i) for i in range(9)]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    out = shard.sharded_run(_chains(), _compute_oracle)
    outg = shard.sharded_run(_grad_chains(), _compute_oracle_grad, with_grad=True)
    outs = shard.sharded_run(_grad_chains(), _compute_oracle_grad, with_grad=True, sum_grad=True)
    if rank == 0:
        q.put((out, outg, outs))
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
    (T2, st2), (Tg, stg, g2), (Ts, sts, gsum) = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    T1, st1 = _compute_oracle(_chains())
    assert np.array_equal(T1, T2) and (st2 == 0).all()
    T1g, _, g1 = _compute_oracle_grad(_grad_chains())
    assert np.array_equal(T1g, Tg) and (stg == 0).all()
    assert all(np.array_equal(a, b) for a, b in zip(g1, g2))
    # the sum over chains: partial sums per rank, then one gather
    assert np.allclose(gsum, np.sum(g1, axis=0), rtol=1e-13, atol=1e-15)
    assert np.array_equal(T1g, Ts)


def test_single_process_gradient_gather():
    T, st, g = shard.sharded_run(_grad_chains(), _compute_oracle_grad, with_grad=True)
    T1, _, g1 = _compute_oracle_grad(_grad_chains())
    assert np.array_equal(T, T1) and all(np.array_equal(a, b) for a, b in zip(g, g1))
    _, _, gs = shard.sharded_run(_grad_chains(), _compute_oracle_grad, with_grad=True,
                                 sum_grad=True)
    assert np.array_equal(gs, np.sum(g1, axis=0))
