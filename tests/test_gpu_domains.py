"""Chains cut into more than two domains (interior domains recursed as segments
open at their first column, combined by a tree of Dyson joins across their
boundary bonds) against the oracle, in all four precisions."""
import numpy as np
import pytest

import workloads
from oracle import leads as oleads, rgf as orgf

pytestmark = pytest.mark.gpu
T_HOP = -2.7
TOL = {0: 1e-9, 1: 1e-7, 2: 1e-7, 3: 1e-9}


@pytest.fixture
def domains(rgflib):
    yield rgflib.set_domains
    rgflib.set_domains(2)
    rgflib.set_schedule(rgflib.RGF_SCHED_PHASED)


def _oracle(N, L, E, eps, rem):
    try:
        return orgf.transmission(N, L, E, 1e-8, 1e-8, T_HOP, eps, rem)
    except oleads.NoConvergence:
        return None


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
@pytest.mark.parametrize("ndom", [3, 4, 6, 9])
def test_interior_domains_vs_oracle(rgflib, domains, prec, ndom):
    # domain boundaries on every column type (ncol = 4L split in ndom parts),
    # edge vacancies, energies near and away from E = 0
    cases = [(11, 7, 0.25, 0.0), (23, 9, 0.2, 0.25), (40, 5, 0.1, 0.1), (9, 13, 0.3, 0.3)]
    domains(ndom)
    Es = np.array([-0.83, -4e-3, 0.021, 0.37])
    for N, L, W, p in cases:
        eps = workloads.anderson_onsite(N, L, W, 10 * N + L)
        rem = workloads.edge_removed(N, L, p, 10 * N + L + 1)
        rib = rgflib.Ribbon(N, L, T_HOP, onsite=eps, removed=rem)
        T, st = rgflib.conductance([rib] * len(Es), Es, 1e-8, 1e-8, prec, check=False)
        for i, e in enumerate(Es):
            ref = _oracle(N, L, e, eps, rem)
            if ref is None:
                continue
            assert st[i] == 0, (N, L, e, st[i])
            assert abs(T[i] - ref) < TOL[prec] * max(1.0, abs(ref)), (ndom, N, L, e, T[i], ref)


@pytest.mark.parametrize("prec", [0, 2])
def test_pair_fallback_inside_interior_domains(rgflib, domains, prec):
    # atoms of second columns at E (isolated-atom resonances) spread over the
    # chain, so that interior domains take single steps where pairs are unsafe
    N, L, E = 23, 16, 0.13
    eps = workloads.anderson_onsite(N, L, 0.25, 5)
    for cell, delta in ((3, 3e-5), (6, -2e-6), (9, 5e-4), (12, -1e-9), (14, 2e-5)):
        eps[cell, 2 * 4 + 1] = E + delta
        eps[cell, 2 * 5 + 1] = E - delta
    rem = workloads.edge_removed(N, L, 0.3, 9)
    rib = rgflib.Ribbon(N, L, T_HOP, onsite=eps, removed=rem)
    for ndom in (3, 5, 8, 13):
        domains(ndom)
        T, st = rgflib.conductance([rib] * 2, np.array([E, -0.4]), 1e-8, 1e-8, prec, check=False)
        assert (st == 0).all()
        for e, t in zip((E, -0.4), T):
            ref = _oracle(N, L, e, eps, rem)
            assert abs(t - ref) < TOL[prec], (ndom, e, t, ref)


def test_domain_count_is_capped_and_automatic(rgflib, domains):
    # forcing more domains than half the columns caps them (L = 2: 8 columns,
    # at most 4 domains); the automatic count for one chain of 160 columns is 5
    assert rgflib.auto_domains(1, 8, 152) == 2
    assert rgflib.auto_domains(1, 160, 152) == 5
    N, L = 15, 2
    eps = workloads.anderson_onsite(N, L, 0.2, 3)
    rib = rgflib.Ribbon(N, L, T_HOP, onsite=eps)
    domains(50)
    T, st = rgflib.conductance([rib], np.array([0.31]), 1e-8, 1e-8, rgflib.RGF_FP64)
    assert abs(T[0] - _oracle(N, L, 0.31, eps, None)) < 1e-9
    domains(0)
    N, L = 61, 40
    eps = workloads.anderson_onsite(N, L, 0.15, 4)
    rib = rgflib.Ribbon(N, L, T_HOP, onsite=eps)
    ref = _oracle(N, L, 0.22, eps, None)
    for prec in (0, 2):
        T, st = rgflib.conductance([rib], np.array([0.22]), 1e-8, 1e-8, prec)
        assert abs(T[0] - ref) < TOL[prec], (prec, T[0], ref)


def test_uneven_batch_and_graph_with_interior_domains(rgflib, domains):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(21)
    ribs, Es, host = [], [], []
    for i in range(30):
        N, L = int(rng.integers(4, 40)), int(rng.integers(3, 12))
        eps = workloads.anderson_onsite(N, L, 0.2, 500 + i)
        rem = workloads.edge_removed(N, L, 0.15, 600 + i)
        ribs.append(rgflib.Ribbon(N, L, T_HOP, onsite=eps, removed=rem))
        Es.append(float(rng.uniform(-0.9, 0.9)))
        host.append((N, L, eps, rem))
    Es = np.array(Es)
    domains(5)
    # the persistent schedule falls back to the three launches with more than
    # two domains
    rgflib.set_schedule(rgflib.RGF_SCHED_PERSISTENT)
    T, st = rgflib.conductance(ribs, Es, 1e-8, 1e-8, rgflib.RGF_MIXED_TC, check=False)
    for i in range(0, 30, 3):
        N, L, eps, rem = host[i]
        ref = _oracle(N, L, Es[i], eps, rem)
        if ref is None:
            continue
        assert st[i] == 0 and abs(T[i] - ref) < 1e-7, (i, T[i], ref)
    rgflib.set_schedule(rgflib.RGF_SCHED_PHASED)
    dE = torch.tensor(Es, dtype=torch.float64, device="cuda")
    dT = torch.empty(len(Es), dtype=torch.float64, device="cuda")
    b = rgflib.Batch(ribs, dE.data_ptr(), len(Es), dT.data_ptr(), precision=rgflib.RGF_MIXED_TC)
    b.launch(torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    T2, _ = rgflib.conductance(ribs, Es, 1e-8, 1e-8, rgflib.RGF_MIXED_TC, check=False)
    assert np.array_equal(dT.cpu().numpy(), T2)
    b.close()
