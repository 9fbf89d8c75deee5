"""The batch driver: the persistent kernel with its device work queue against
the three-launch schedule, the CUDA-graph batch, and every tuned schedule
(engine x panel width x pair steps) against the oracle."""
import numpy as np
import pytest

import workloads
from oracle import leads as oleads, rgf as orgf

pytestmark = pytest.mark.gpu
T_HOP = -2.7


@pytest.fixture
def clean_state(rgflib):
    yield
    rgflib.set_schedule(rgflib.RGF_SCHED_PHASED)
    for p in (rgflib.RGF_FP64, rgflib.RGF_MIXED, rgflib.RGF_MIXED_TC):
        rgflib.set_tuning(p, [])


def _mixed_batch(rgflib, n, seed, Nmax=40, Lmax=6):
    """n chains of uneven width and length, some with edge vacancies, at random
    energies; returns (ribbons, E, host arrays for the oracle)."""
    rng = np.random.default_rng(seed)
    ribs, Es, host = [], [], []
    for i in range(n):
        N = int(rng.integers(3, Nmax))
        L = int(rng.integers(1, Lmax))
        p = 0.2 if i % 3 == 0 else 0.0
        eps, rem = workloads.anderson_onsite(N, L, 0.2, 1000 + i), workloads.edge_removed(N, L, p, 2000 + i)
        ribs.append(rgflib.Ribbon(N, L, T_HOP, onsite=eps, removed=rem))
        Es.append(float(rng.uniform(-1.0, 1.0)))
        host.append((N, L, eps, rem))
    return ribs, np.array(Es), host


def _dev_call(rgflib, ribs, E, prec):
    """rgf_conductance_dev (device buffers: a non-finite energy reaches the
    lead kernel and comes back as that chain's RGF_EINVAL)."""
    import torch
    dE = torch.tensor(E, dtype=torch.float64, device="cuda")
    dT = torch.empty(len(E), dtype=torch.float64, device="cuda")
    dS = torch.full((len(E),), -1, dtype=torch.int32, device="cuda")
    rgflib.conductance_dev(ribs, dE.data_ptr(), len(E), dT.data_ptr(), dS.data_ptr(),
                           precision=prec, stream=torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return dT.cpu().numpy(), dS.cpu().numpy()


def _both_schedules(rgflib, ribs, E, prec):
    out = {}
    for sched in (rgflib.RGF_SCHED_PERSISTENT, rgflib.RGF_SCHED_PHASED):
        rgflib.set_schedule(sched)
        out[sched] = _dev_call(rgflib, ribs, E, prec)
    rgflib.set_schedule(rgflib.RGF_SCHED_PHASED)
    return out[rgflib.RGF_SCHED_PERSISTENT], out[rgflib.RGF_SCHED_PHASED]


# The two schedules run the same arithmetic in separately compiled kernels
# (the compiler may fuse a product and a sum into one FMA in one and not in
# the other), so they agree to rounding, not bit for bit; each is
# deterministic.
SCHED_TOL = {0: 1e-10, 1: 1e-10, 2: 1e-10, 3: 1e-10}


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_persistent_queue_equals_three_launches(rgflib, clean_state, prec):
    # more halves than SMs, uneven sizes, a non-finite energy (RGF_EINVAL from
    # the lead kernel, still counted through the queue and the join)
    ribs, E, _ = _mixed_batch(rgflib, 200, 11)
    E[17] = np.nan
    (Tp, sp), (Tq, sq) = _both_schedules(rgflib, ribs, E, prec)
    rgflib.set_schedule(rgflib.RGF_SCHED_PERSISTENT)
    Tp2, sp2 = _dev_call(rgflib, ribs, E, prec)            # persistent again
    assert np.array_equal(sp, sq) and np.array_equal(sp, sp2)
    assert sp[17] == rgflib.RGF_EINVAL and np.isnan(Tp[17])
    ok = sp == 0
    assert ok.sum() >= 190
    assert np.array_equal(Tp[ok], Tp2[ok])                 # the queue order does not matter
    d = np.abs(Tp[ok] - Tq[ok])
    assert d.max() <= SCHED_TOL[prec], (prec, d.max(), int((d > 0).sum()))


def test_persistent_queue_vs_oracle(rgflib, clean_state):
    ribs, E, host = _mixed_batch(rgflib, 320, 12, Nmax=24, Lmax=4)
    rgflib.set_schedule(rgflib.RGF_SCHED_PERSISTENT)
    for prec, tol in ((rgflib.RGF_FP64, 1e-9), (rgflib.RGF_MIXED_TC, 1e-7)):
        T, st = rgflib.conductance(ribs, E, 1e-8, 1e-8, prec, check=False)
        for i in range(0, len(ribs), 16):        # a sample the oracle does in seconds
            N, L, eps, rem = host[i]
            try:
                ref = orgf.transmission(N, L, E[i], 1e-8, 1e-8, T_HOP, eps, rem)
            except oleads.NoConvergence:
                continue
            assert st[i] == 0, (i, st[i])
            assert abs(T[i] - ref) < tol, (prec, i, T[i], ref)


def test_graph_batch_relaunch_follows_new_energies(rgflib, clean_state):
    torch = pytest.importorskip("torch")
    ribs, E, _ = _mixed_batch(rgflib, 40, 13)
    for prec, sched in ((rgflib.RGF_FP64, rgflib.RGF_SCHED_PHASED),
                        (rgflib.RGF_MIXED_TC, rgflib.RGF_SCHED_PHASED),
                        (rgflib.RGF_MIXED_TC, rgflib.RGF_SCHED_PERSISTENT)):
        rgflib.set_schedule(sched)                 # captured at creation, used by both calls
        dE = torch.tensor(E, dtype=torch.float64, device="cuda")
        dT = torch.full((len(E),), -1.0, dtype=torch.float64, device="cuda")
        dS = torch.full((len(E),), -1, dtype=torch.int32, device="cuda")
        b = rgflib.Batch(ribs, dE.data_ptr(), len(E), dT.data_ptr(), dS.data_ptr(), precision=prec)
        stream = torch.cuda.current_stream().cuda_stream
        for shift in (0.0, 0.07, -0.11):
            Es = np.clip(E + shift, -1.2, 1.2)
            dE.copy_(torch.from_numpy(Es))
            b.launch(stream)
            torch.cuda.synchronize()
            Tref, sref = rgflib.conductance(ribs, Es, 1e-8, 1e-8, prec, check=False)
            assert np.array_equal(dS.cpu().numpy(), sref)
            ok = sref == 0
            assert np.array_equal(dT.cpu().numpy()[ok], Tref[ok])
        b.close()


def _entries(engine, panel, pairs):
    return [dict(K_max=4096, engine=engine, panel=panel, pairs=pairs)]


@pytest.mark.parametrize("engine", [1, 0])
@pytest.mark.parametrize("panel", [16, 8, 4, 2])
@pytest.mark.parametrize("pairs", [1, 0])
def test_every_tuned_schedule_vs_oracle(rgflib, clean_state, engine, panel, pairs):
    # widths with columns of several panels and a ragged last panel, vacancies
    cases = [(21, 4, 0.0), (37, 3, 0.25), (50, 2, 0.1)]
    for prec, tol in ((rgflib.RGF_MIXED_TC, 1e-7), (rgflib.RGF_MIXED, 1e-7), (rgflib.RGF_FP64, 1e-9),
                      (rgflib.RGF_FP64_TC, 1e-9)):
        if engine == 0 and prec not in (rgflib.RGF_MIXED_TC, rgflib.RGF_FP64_TC):
            continue                               # the engine is read by the _TC precisions only
        rgflib.set_tuning(prec, _entries(engine, panel, pairs))
        for N, L, p in cases:
            eps = workloads.anderson_onsite(N, L, 0.25, N)
            rem = workloads.edge_removed(N, L, p, N + 1)
            rib = rgflib.Ribbon(N, L, T_HOP, onsite=eps, removed=rem)
            Es = np.array([-0.61, 0.0123, 0.37])
            T, st = rgflib.conductance([rib] * 3, Es, 1e-8, 1e-8, prec, check=False)
            for i, e in enumerate(Es):
                ref = orgf.transmission(N, L, e, 1e-8, 1e-8, T_HOP, eps, rem)
                assert st[i] == 0 and abs(T[i] - ref) < tol, (prec, N, e, T[i], ref)
        rgflib.set_tuning(prec, [])


def test_engine_groups_split_one_call(rgflib, clean_state):
    # narrow chains on the FP32 pipes, wide ones on the tensor cores: two
    # launch groups in one call, each bit-identical to the same chains run
    # alone with the same schedule
    ribs, E, _ = _mixed_batch(rgflib, 120, 14, Nmax=60)
    table = [dict(K_max=12, engine=0, panel=8, pairs=1), dict(K_max=4096, engine=1, panel=0, pairs=1)]
    rgflib.set_tuning(rgflib.RGF_MIXED_TC, table)
    (Tp, sp), (Tq, sq) = _both_schedules(rgflib, ribs, E, rgflib.RGF_MIXED_TC)
    assert np.array_equal(sp, sq) and (sp == 0).all()
    assert np.abs(Tp - Tq).max() <= SCHED_TOL[2]
    narrow = [i for i, r in enumerate(ribs) if (r.N + 1) // 2 <= 12]
    wide = [i for i, r in enumerate(ribs) if (r.N + 1) // 2 > 12]
    assert narrow and wide
    for sched, Tref in ((rgflib.RGF_SCHED_PHASED, Tq), (rgflib.RGF_SCHED_PERSISTENT, Tp)):
        rgflib.set_schedule(sched)
        for idx in (narrow, wide):
            T1, s1 = rgflib.conductance([ribs[i] for i in idx], E[idx], 1e-8, 1e-8,
                                        rgflib.RGF_MIXED_TC, check=False)
            assert np.array_equal(T1, Tref[idx])


def test_autotune_installs_a_table_that_stays_correct(rgflib, clean_state):
    prec = rgflib.RGF_MIXED_TC
    table, ms = rgflib.autotune(prec, [41, 11], cells=2, reps=1)
    assert [e["K_max"] for e in table] == [21, 6]
    assert ms.shape == (2, rgflib.RGF_TUNE_MAX_CANDIDATES)
    assert np.isfinite(ms).all() and (ms > 0).all()
    installed = rgflib.get_tuning(prec)
    assert [e["K_max"] for e in installed] == [6, 21]
    for e, row in zip(table, ms):
        # the winner is the first fastest candidate; candidates run engine
        # (tensor cores, then pipes) x panel (16, 8, 4) x pairs (1, 0)
        c = int(np.argmin(row))
        assert e == dict(K_max=e["K_max"], engine=1 - c // 6, panel=(16, 8, 4)[(c // 2) % 3],
                         pairs=(1, 0)[c % 2])
    assert rgflib.tune_lookup(prec, 11) == installed[0]
    assert rgflib.tune_lookup(prec, 41) == installed[1]
    N, L = 41, 3
    eps = workloads.anderson_onsite(N, L, 0.2, 9)
    rib = rgflib.Ribbon(N, L, T_HOP, onsite=eps)
    T, st = rgflib.conductance([rib], np.array([0.21]), 1e-8, 1e-8, prec)
    ref = orgf.transmission(N, L, 0.21, 1e-8, 1e-8, T_HOP, eps, None)
    assert abs(T[0] - ref) < 1e-7
