"""Chain sharding driving the product: two gloo ranks, each a process on the one
GPU, evaluate their longest-processing-time share of a batch through librgf
(binary64), and one gather brings T, status and gradients to rank 0.  The
result is bit for bit that of one process evaluating every chain.  (The two
processes' kernels never wait on one another.)"""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _chains():
    rng = np.random.default_rng(7)
    return [dict(N=int(rng.integers(5, 40)), L=int(rng.integers(1, 8)), E=float(rng.uniform(-1, 1)),
                 seed=300 + i) for i in range(11)]


def _compute(chains, grad=False):
    from paper_1107_5300_gb300 import rgf
    T, st, g = [], [], []
    for c in chains:
        rib = rgf.Ribbon(c["N"], c["L"], -2.7, W=0.2, seed=c["seed"], edge_p=0.1,
                         edge_seed=c["seed"] + 1)
        if grad:
            t, gc, s = rgf.conductance_grad([rib], np.array([c["E"]]), 1e-8, 1e-8, rgf.RGF_FP64,
                                            check=False)
            g.append(gc[0])
        else:
            t, s = rgf.conductance([rib], np.array([c["E"]]), 1e-8, 1e-8, rgf.RGF_FP64, check=False)
        T.append(t[0])
        st.append(s[0])
    out = (np.array(T), np.array(st, dtype=np.int32))
    return out + (g,) if grad else out


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    from paper_1107_5300_gb300 import shard
    torch.cuda.set_device(0)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    out = shard.sharded_run(_chains(), _compute)
    outg = shard.sharded_run(_chains(), lambda cs: _compute(cs, grad=True), with_grad=True)
    if rank == 0:
        q.put((out, outg))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_on_librgf_equal_one_process(rgflib):
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    (T2, st2), (Tg, stg, g2) = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    T1, st1 = _compute(_chains())
    assert (st1 == 0).all() and np.array_equal(st1, st2) and np.array_equal(T1, T2)
    T1g, _, g1 = _compute(_chains(), grad=True)
    assert np.array_equal(T1g, Tg) and (stg == 0).all()
    assert all(np.array_equal(a, b) for a, b in zip(g1, g2))
