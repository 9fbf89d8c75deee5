"""Gradient dT/d eps (rgf_conductance_grad) against the oracle (dense closed
form, and golden values of its two-sided form on the N = 101, L = 500 ribbon)
and against finite differences of the GPU conductance."""
import json
from pathlib import Path

import numpy as np
import pytest

import workloads
from oracle import gradient as ograd

pytestmark = pytest.mark.gpu
T_HOP = -2.7
GOLDEN = Path(__file__).resolve().parent / "golden"


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-8), (2, 1e-8), (3, 1e-9)])
def test_gradient_matches_oracle_closed_form(rgflib, prec, tol):
    N, L = 11, 6
    eps = workloads.anderson_onsite(N, L, 0.3, 11)
    rem = workloads.edge_removed(N, L, 0.3, 12)
    rib = rgflib.Ribbon(N, L, T_HOP, onsite=eps, removed=rem)
    Es = np.array([-0.9, 0.31, 0.004])
    T, g, st = rgflib.conductance_grad([rib] * 3, Es, 1e-8, 1e-8, prec, ckpt_stride=2)
    assert (st == 0).all()
    for c, E in enumerate(Es):
        ref = ograd.closed_form(N, L, E, 1e-8, 1e-8, T_HOP, eps, rem)
        scale = max(1.0, np.abs(ref).max())
        assert np.abs(g[c] - ref).max() < tol * scale, (E, np.abs(g[c] - ref).max())
        assert np.all(g[c][rem.astype(bool)] == 0.0)


def test_gradient_oracle_n11_l20(rgflib):
    # Oracle gradient on an N = 11, L = 20 ribbon (Anderson +-0.15 eV).
    N, L = 11, 20
    eps = workloads.anderson_onsite(N, L, 0.15, 4)
    rib = rgflib.Ribbon(N, L, T_HOP, onsite=eps)
    Es = np.array([-0.8, -0.2, 0.45])
    for prec, tol in ((0, 1e-10), (1, 1e-8), (2, 1e-8), (3, 1e-9)):
        T, g, st = rgflib.conductance_grad([rib] * 3, Es, 1e-8, 1e-8, prec)
        for c, E in enumerate(Es):
            ref = ograd.closed_form(N, L, E, 1e-8, 1e-8, T_HOP, eps, None)
            assert np.abs(g[c] - ref).max() < tol * max(1.0, np.abs(ref).max())


def test_checkpoint_stride_does_not_change_the_gradient(rgflib):
    N, L = 12, 9
    rib = rgflib.Ribbon(N, L, T_HOP, W=0.2, seed=3, edge_p=0.2, edge_seed=4)
    Es = np.array([0.21, -0.6])
    outs = [rgflib.conductance_grad([rib] * 2, Es, ckpt_stride=s)[1] for s in (1, 2, 4, 9, 0)]
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    # the gradient sweep's own T agrees with the conductance entry point's
    T, _ = rgflib.conductance([rib] * 2, Es)
    Tg = rgflib.conductance_grad([rib] * 2, Es)[0]
    assert np.max(np.abs(T - Tg)) < 1e-12


def test_gradient_against_finite_differences_n101(rgflib):
    # N = 101, L = 500, Anderson +-0.15 eV (seed 4), 64 sites drawn from seed 44,
    # central differences with delta = 1e-6 eV; stride 23 cells.
    w = workloads.WORKLOADS["agnr101_L500_grad"]
    N, L = w["N"], w["L"]
    eps = workloads.anderson_onsite(N, L, w["W"], w["seed"])
    E = float(w["energies"]()[37])
    rib = rgflib.Ribbon(N, L, T_HOP, onsite=eps)
    u = workloads.uniform01(44, np.arange(128, dtype=np.uint64))
    sites = [(int(u[2 * i] * L), int(u[2 * i + 1] * 2 * N)) for i in range(64)]
    d = 1e-6
    ribs = []
    for (n, i) in sites:
        for sgn in (1, -1):
            e2 = eps.copy()
            e2[n, i] += sgn * d
            ribs.append(rgflib.Ribbon(N, L, T_HOP, onsite=e2))
    Tfd, st = rgflib.conductance(ribs, np.full(len(ribs), E))
    fd = (Tfd[0::2] - Tfd[1::2]) / (2 * d)
    for prec in (0, 1, 2, 3):
        T, g, st = rgflib.conductance_grad([rib], np.array([E]), 1e-8, 1e-8, prec, ckpt_stride=23)
        assert st[0] == 0
        gs = np.array([g[0, n, i] for (n, i) in sites])
        err = np.abs(gs - fd)
        assert np.all(err < 1e-5 + 1e-4 * np.abs(fd)), (prec, err.max())


@pytest.mark.parametrize("prec,tol", [(0, 1e-7), (1, 1e-5), (2, 1e-5), (3, 1e-5)])
def test_gradient_next_to_a_half_system_pole(rgflib, prec, tol):
    # N = 20, L = 40 (Anderson +-0.15 eV, seed 7) at E = -0.0764 eV, next to a
    # pole of the half systems: a reverse sweep over the column slices is off
    # by about 4e-4 of the gradient's scale here even in complex128.
    N, L = 20, 40
    eps = workloads.anderson_onsite(N, L, 0.15, 7)
    E = float(np.linspace(-0.12, 0.12, 12)[2])
    rib = rgflib.Ribbon(N, L, T_HOP, onsite=eps)
    T, g, st = rgflib.conductance_grad([rib], np.array([E]), 1e-8, 1e-8, prec, ckpt_stride=3)
    assert st[0] == 0
    ref = ograd.closed_form(N, L, E, 1e-8, 1e-8, T_HOP, eps, None)
    err = np.abs(g[0] - ref).max() / np.abs(ref).max()
    assert err < tol, (prec, err)


@pytest.mark.parametrize("prec,tol", [(0, 1e-5), (1, 2e-4), (2, 2e-4), (3, 2e-4)])
def test_gradient_near_zero_energy_matches_golden(rgflib, prec, tol):
    # The N = 101, L = 500 ribbon at three energies with |E| < 0.07 eV: the
    # largest entries, seeded random sites and sites where a reverse sweep
    # over column slices was off by 10 to 400 times the gradient's scale,
    # against oracle.gradient.two_sided (tests/golden/make_grad_golden.py).
    gold = json.loads((GOLDEN / "grad_two_sided.json").read_text())
    eps = workloads.anderson_onsite(gold["N"], gold["L"], gold["W"], gold["seed"])
    rib = rgflib.Ribbon(gold["N"], gold["L"], gold["t"], onsite=eps)
    Es = np.array([cs["E"] for cs in gold["cases"]])
    T, g, st = rgflib.conductance_grad([rib] * len(Es), Es, gold["eta_device"], gold["eta_lead"],
                                       prec, ckpt_stride=23)
    assert (st == 0).all()
    for c, cs in enumerate(gold["cases"]):
        assert abs(T[c] - cs["T"]) < 1e-7
        for n, i, v in cs["sites"]:
            assert abs(g[c, n, i] - v) < tol * cs["scale"], (prec, cs["E"], n, i, g[c, n, i], v)


def test_autograd_function(rgflib):
    import torch
    from paper_1107_5300_gb300.autograd import conductance
    N, L = 5, 4
    eps0 = workloads.anderson_onsite(N, L, 0.2, 9)
    eps = torch.tensor(eps0, dtype=torch.float64, device="cuda", requires_grad=True)
    E = torch.tensor([0.3, -0.5], dtype=torch.float64)
    T = conductance(eps, E, N)
    w = torch.tensor([1.0, -2.0], dtype=torch.float64, device="cuda")
    (T * w).sum().backward()
    ref = sum(wc * ograd.closed_form(N, L, Ec, 1e-8, 1e-8, T_HOP, eps0, None)
              for wc, Ec in zip([1.0, -2.0], [0.3, -0.5]))
    assert np.abs(eps.grad.cpu().numpy() - ref).max() < 1e-10


def test_device_gradient_entry_point(rgflib):
    # rgf_conductance_grad_dev on a stream: per-chain gradients equal the host
    # entry point's; with weights, their weighted sum over chains.
    import torch
    N, L = 12, 5
    rib = rgflib.Ribbon(N, L, T_HOP, W=0.2, seed=6, edge_p=0.2, edge_seed=7)
    Es = np.array([-0.7, 0.25, 0.9])
    T_h, g_h, _ = rgflib.conductance_grad([rib] * 3, Es, 1e-8, 1e-8, rgflib.RGF_MIXED_TC)
    s = torch.cuda.Stream()
    Ed = torch.tensor(Es, dtype=torch.float64, device="cuda")
    Td = torch.empty(3, dtype=torch.float64, device="cuda")
    Sd = torch.empty(3, dtype=torch.int32, device="cuda")
    Gd = torch.empty((3, L, 2 * N), dtype=torch.float64, device="cuda")
    s.wait_stream(torch.cuda.current_stream())
    rgflib.conductance_grad_dev([rib] * 3, Ed.data_ptr(), 3, Td.data_ptr(), Gd.data_ptr(),
                                status_ptr=Sd.data_ptr(), precision=rgflib.RGF_MIXED_TC,
                                stream=s.cuda_stream)
    w = torch.tensor([0.5, -1.0, 2.0], dtype=torch.float64, device="cuda")
    Vd = torch.empty((L, 2 * N), dtype=torch.float64, device="cuda")
    rgflib.conductance_grad_dev([rib] * 3, Ed.data_ptr(), 3, Td.data_ptr(), Vd.data_ptr(),
                                weights_ptr=w.data_ptr(), precision=rgflib.RGF_MIXED_TC,
                                stream=s.cuda_stream)
    s.synchronize()
    assert (Sd.cpu().numpy() == 0).all()
    assert np.array_equal(Gd.cpu().numpy(), g_h) and np.array_equal(Td.cpu().numpy(), T_h)
    ref = 0.5 * g_h[0] - 1.0 * g_h[1] + 2.0 * g_h[2]
    assert np.abs(Vd.cpu().numpy() - ref).max() < 1e-14 * max(1.0, np.abs(ref).max())


@pytest.mark.slow
def test_widest_ribbon_gradient_runs_on_the_pipes(rgflib):
    # N = 2047 (KL = 1024): the tensor-core layout of the two-sided sweep does
    # not fit a block's shared memory beyond KL = 980, so RGF_MIXED_TC runs the
    # same kernel as RGF_MIXED (RGF_FP64_TC as RGF_FP64, and the LDOS sweep,
    # by the same rule in the same launcher): bit-identical gradients
    N, L = 2047, 1
    eps = workloads.anderson_onsite(N, L, 0.1, 71)
    rib = rgflib.Ribbon(N, L, -2.7, onsite=eps)
    E = np.array([0.057])
    Ta, ga, sa = rgflib.conductance_grad([rib], E, 1e-8, 1e-8, rgflib.RGF_MIXED_TC)
    Tb, gb, sb = rgflib.conductance_grad([rib], E, 1e-8, 1e-8, rgflib.RGF_MIXED)
    assert (sa == 0).all() and (sb == 0).all()
    assert np.array_equal(Ta, Tb) and np.array_equal(ga, gb)
    assert np.isfinite(gb).all() and np.abs(gb).max() > 0.0
