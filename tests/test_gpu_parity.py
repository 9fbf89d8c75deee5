"""GPU path (through the C ABI) against the CPU oracle, element by element."""
import numpy as np
import pytest

import workloads
from oracle import bands, leads as oleads, rgf as orgf

pytestmark = pytest.mark.gpu
T_HOP = -2.7


def _oracle_T(N, L, E, etad, etal, eps, rem):
    try:
        return orgf.transmission(N, L, E, etad, etal, T_HOP, eps, rem)
    except oleads.NoConvergence:
        return None


@pytest.mark.parametrize("N", [2, 5, 11, 12, 24])
def test_lead_selfenergy_matches_oracle(rgflib, N):
    E = np.array([-1.3, -0.2, 0.003, 0.4, 1.7, 3.1])
    for side in (0, 1):
        sig, it = rgflib.lead_selfenergy(N, E, 1e-8, side)
        for i, e in enumerate(E):
            sL, sR, iL, iR = oleads.self_energies(N, e, 1e-8, T_HOP, return_iters=True)
            ref = sL if side == 0 else sR
            err = np.abs(sig[i] - ref).max() / max(1.0, np.abs(ref).max())
            assert err < 1e-10, (N, e, side, err)
            assert abs(int(it[i]) - (iL if side == 0 else iR)) <= 3


def test_lead_selfenergy_at_exact_charge_neutrality(rgflib):
    # The full-cell complex128 iteration of the oracle is ill-conditioned here
    # (it overflows or meets a singular block, depending on N and the BLAS);
    # compare with the same iteration in 40 digits instead.
    from oracle import mp as omp
    sig, it = rgflib.lead_selfenergy(23, np.array([0.0, 0.2]), 1e-8, 1)
    assert (it > 0).all() and np.isfinite(sig).all()
    for N in (5, 6):
        sL, sR = omp.self_energies(N, 0.0, 1e-8, T_HOP, dps=40)
        for side, ref in ((0, sL), (1, sR)):
            g, _ = rgflib.lead_selfenergy(N, np.array([0.0]), 1e-8, side)
            assert np.abs(g[0] - ref).max() / np.abs(ref).max() < 1e-12


def _run(rgflib, N, L, Es, eps, rem, prec, etad=1e-8, etal=1e-8):
    rib = rgflib.Ribbon(N, L, T_HOP, onsite=eps, removed=rem)
    T, st = rgflib.conductance([rib] * len(Es), Es, etad, etal, prec, check=False)
    return T, st


def test_pristine_n11_energy_grid_fp64(rgflib):
    # 201 energies in [-1, 1] eV, N = 11, L = 50, eta = 1e-8 eV.  At E = 0
    # exactly every partial system of a pristine ribbon carries a surface state
    # (|g| ~ 1/eta) and the column slice matrices are singular to binary64:
    # the chain reports RGF_ESINGULAR there (see the E = 0 test below).
    w = workloads.WORKLOADS["agnr11_L50_pristine"]
    N, L = w["N"], w["L"]
    Es = w["energies"]()
    T, st = _run(rgflib, N, L, Es, None, None, rgflib.RGF_FP64)
    for e, t, s in zip(Es, T, st):
        if e == 0.0:
            assert s == rgflib.RGF_ESINGULAR and np.isnan(t)
            continue
        assert s == 0
        ref = _oracle_T(N, L, e, 1e-8, 1e-8, None, None)
        assert abs(t - ref) < 1e-9, (e, t, ref)
    # quantisation: T ~ n_ch up to the eta absorption of the device
    nz = Es != 0
    assert np.all(np.abs(T[nz] - 1.0) < 1e-5)


# E = 0 exactly (eta = 1e-8 eV) against 40-digit arithmetic
# (tests/golden/mp_transmission.json).  On a disordered ribbon the leads'
# surface states are the only order-1/eta poles, and the end columns are
# handled in the leads' mode basis: the tolerance is the one measured there.
# On a pristine ribbon every partial system has a surface state at E = 0, the
# column slice matrices are singular to the working precision, and the chain
# reports RGF_ESINGULAR.  A pristine ribbon 0.1 meV from E = 0 is
# condition-limited too (|g| ~ 1/E in every column step): 1e-7, measured
# 4.9e-8 in binary64 and 2.8e-8 in double-float against 40 digits.
E0_TOL_DISORDERED = 1e-10
NEAR_E0_TOL_PRISTINE = 1e-7


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_charge_neutrality_point_vs_40_digits(rgflib, prec):
    import json
    from pathlib import Path
    gold = json.loads((Path(__file__).resolve().parent / "golden" / "mp_transmission.json").read_text())
    errs = {}
    for name, g in gold.items():
        eps = workloads.anderson_onsite(g["N"], g["L"], g["W"], g["seed"]) if g["W"] > 0 else None
        T, st = _run(rgflib, g["N"], g["L"], np.array([g["E"]]), eps, None, prec,
                     etad=g["eta_device"], etal=g["eta_lead"])
        errs[name] = (int(st[0]), abs(T[0] - g["T"]))
        print(f"E0 precision={prec} {name}: status {st[0]}, |dT| = {abs(T[0] - g['T']):.3e}")
    for name, g in gold.items():
        st, err = errs[name]
        if g["E"] == 0.0 and g["W"] == 0.0:
            assert st == rgflib.RGF_ESINGULAR, (name, st)
            continue
        assert st == 0, (name, st)
        if g["E"] == 0.0:
            tol = E0_TOL_DISORDERED
        elif g["W"] == 0.0 and abs(g["E"]) < 1e-3:
            tol = NEAR_E0_TOL_PRISTINE
        else:
            tol = 1e-9 if prec in (0, 3) else 1e-7
        assert err < tol, (name, err)


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
@pytest.mark.parametrize("N,L,W,p", [(2, 5, 0.3, 0.0), (3, 4, 0.2, 0.0), (5, 1, 0.25, 0.3),
                                     (11, 3, 0.25, 0.3), (12, 17, 0.4, 0.25), (23, 9, 0.25, 0.2),
                                     (64, 6, 0.1, 0.05), (150, 3, 0.25, 0.05)])
def test_disordered_rough_ribbons(rgflib, N, L, W, p, prec):
    eps = workloads.anderson_onsite(N, L, W, 100 + N)
    rem = workloads.edge_removed(N, L, p, 200 + N)
    Es = np.array([-1.1, -0.3, -5e-3, 1e-3, 0.02, 0.45, 2.2])
    T, st = _run(rgflib, N, L, Es, eps, rem, prec)
    tol = 1e-9 if prec in (0, 3) else 1e-7
    for e, t, s in zip(Es, T, st):
        ref = _oracle_T(N, L, e, 1e-8, 1e-8, eps, rem)
        assert s == 0
        assert abs(t - ref) < tol * max(1.0, abs(ref)), (N, L, e, t, ref)


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_pristine_quantised_without_device_absorption(rgflib, prec):
    for N in (5, 12, 17):
        Es = np.array([0.15, -0.6, 1.4, -2.3])
        T, st = _run(rgflib, N, 12, Es, None, None, prec, etad=0.0)
        for e, t in zip(Es, T):
            assert abs(t - bands.channels_closed_form(N, e)) < 1e-9


def test_batched_uneven_chains_one_call(rgflib):
    rng = np.random.default_rng(5)
    ribs, Es, refs = [], [], []
    for c in range(24):
        N = int(rng.integers(4, 70))
        L = int(rng.integers(1, 25))
        eps = workloads.anderson_onsite(N, L, 0.1, 1000 + c)
        rem = workloads.edge_removed(N, L, 0.05, 2000 + c)
        E = float(rng.uniform(-1, 1))
        ribs.append(rgflib.Ribbon(N, L, T_HOP, onsite=eps, removed=rem))
        Es.append(E)
        refs.append(_oracle_T(N, L, E, 1e-8, 1e-8, eps, rem))
    for prec, tol in ((0, 1e-9), (1, 1e-7), (2, 1e-7), (3, 1e-9)):
        T, st = rgflib.conductance(ribs, np.array(Es), 1e-8, 1e-8, prec)
        assert (st == 0).all()
        assert np.max(np.abs(T - np.array(refs))) < tol


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_two_block_pipeline_schedule(rgflib, prec):
    # 48 chains: two blocks per chain (inverse on one SM, strip product on the
    # other), the schedule of the full-size workload
    N, L = 40, 3
    eps = workloads.anderson_onsite(N, L, 0.25, 77)
    rem = workloads.edge_removed(N, L, 0.1, 78)
    Es = np.linspace(-0.9, 0.9, 48) + 1e-3
    T, st = _run(rgflib, N, L, Es, eps, rem, prec)
    tol = 1e-9 if prec in (0, 3) else 1e-7
    assert (st == 0).all()
    for e, t in zip(Es[::5], T[::5]):
        ref = _oracle_T(N, L, e, 1e-8, 1e-8, eps, rem)
        assert abs(t - ref) < tol * max(1.0, abs(ref)), (e, t, ref)


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_columns_wider_than_one_tensor_tile(rgflib, prec):
    # KL = 150 > 128 orbitals per column: the tensor-core products tile the rows
    # and split the inner dimension into exact accumulation groups
    N, L = 299, 2
    eps = workloads.anderson_onsite(N, L, 0.2, 91)
    Es = np.array([-0.35, 0.05, 0.6])
    T, st = _run(rgflib, N, L, Es, eps, None, prec)
    assert (st == 0).all()
    for e, t in zip(Es, T):
        ref = _oracle_T(N, L, e, 1e-8, 1e-8, eps, None)
        tol = 1e-9 if prec == 3 else 1e-7
        assert abs(t - ref) < tol * max(1.0, abs(ref)), (e, t, ref)


def test_failed_chain_does_not_spoil_the_batch(rgflib):
    # Fault injected on the host: a ribbon uploaded from a device buffer holding
    # a NaN on-site energy.  Its chain reports ENONFINITE; the others are exact.
    import torch
    N, L = 11, 4
    eps = workloads.anderson_onsite(N, L, 0.2, 4)
    bad = torch.tensor(eps, dtype=torch.float64, device="cuda")
    bad[2, 7] = float("nan")
    rbad = rgflib.Ribbon.from_device(N, L, T_HOP, bad.data_ptr())
    torch.cuda.synchronize()
    rok = rgflib.Ribbon(N, L, T_HOP, onsite=eps)
    T, st = rgflib.conductance([rok, rbad, rok], np.array([0.3, 0.3, -0.4]), check=False)
    assert st[1] == rgflib.RGF_ENONFINITE and np.isnan(T[1])
    assert st[0] == 0 and st[2] == 0
    assert abs(T[0] - _oracle_T(N, L, 0.3, 1e-8, 1e-8, eps, None)) < 1e-9
    with pytest.raises(rgflib.RGFError) as e:
        rgflib.conductance([rbad], np.array([0.1]))
    assert e.value.status == rgflib.RGF_ENONFINITE


def test_device_buffer_variant_on_a_stream(rgflib):
    import torch
    rib = rgflib.Ribbon(11, 8, T_HOP, W=0.2, seed=9)
    Es = np.array([-0.4, 0.1, 0.33])
    Th, _ = rgflib.conductance([rib] * 3, Es)
    s = torch.cuda.Stream()
    Ed = torch.tensor(Es, dtype=torch.float64, device="cuda")
    Td = torch.empty(3, dtype=torch.float64, device="cuda")
    Sd = torch.empty(3, dtype=torch.int32, device="cuda")
    s.wait_stream(torch.cuda.current_stream())
    rgflib.conductance_dev([rib] * 3, Ed.data_ptr(), 3, Td.data_ptr(), Sd.data_ptr(),
                           stream=s.cuda_stream)
    s.synchronize()
    assert np.array_equal(Td.cpu().numpy(), Th)
    assert (Sd.cpu().numpy() == 0).all()


def test_invalid_arguments_are_rejected(rgflib):
    with pytest.raises(rgflib.RGFError) as e:
        rgflib.Ribbon(1, 5)
    assert e.value.status == rgflib.RGF_EINVAL
    rib = rgflib.Ribbon(5, 2)
    with pytest.raises(rgflib.RGFError):
        rgflib.conductance([rib], np.array([np.nan]))
    with pytest.raises(rgflib.RGFError):
        rgflib.conductance([rib], np.array([0.1]), precision=7)
    with pytest.raises(rgflib.RGFError):
        rgflib.conductance([rib], np.array([0.1]), eta_lead=0.0)


@pytest.fixture(scope="module")
def wide_case():
    # N = 501 (KL = 251 orbitals per column): two 128-row tiles, two exact
    # accumulation groups in the strip product, a narrower Gauss-Jordan panel
    N, L = 501, 2
    eps = workloads.anderson_onsite(N, L, 0.1, 501)
    rem = workloads.edge_removed(N, L, 0.02, 502)
    Es = np.array([-0.21, 0.13])
    refs = [_oracle_T(N, L, e, 1e-8, 1e-8, eps, rem) for e in Es]
    return N, L, eps, rem, Es, refs


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_wide_columns_vs_oracle(rgflib, wide_case, prec):
    N, L, eps, rem, Es, refs = wide_case
    T, st = _run(rgflib, N, L, Es, eps, rem, prec)
    assert (st == 0).all()
    tol = 1e-9 if prec in (0, 3) else 1e-7
    for e, t, ref in zip(Es, T, refs):
        assert abs(t - ref) < tol * max(1.0, abs(ref)), (e, t, ref)


@pytest.mark.slow
def test_widest_accepted_ribbon_precisions_agree(rgflib):
    # N = 2047, the widest ribbon the ABI accepts (KL = 1024 orbitals per
    # column: eight row tiles of the tensor-core products, the narrowest
    # Gauss-Jordan panel, the largest shared-memory layout).  The oracle's
    # full-cell decimation at M = 4094 is out of reach in a test, so the four
    # precisions are checked against each other and against 0 <= T <= n_ch.
    N, L = 2047, 2
    eps = workloads.anderson_onsite(N, L, 0.1, 2047)
    rem = workloads.edge_removed(N, L, 0.05, 2048)
    Es = np.array([-0.11, 0.043])
    out = {}
    for prec in (0, 1, 2, 3):
        T, st = _run(rgflib, N, L, Es, eps, rem, prec)
        assert (st == 0).all(), (prec, st)
        out[prec] = T
    for e, t in zip(Es, out[0]):
        assert -1e-9 <= t <= bands.channels_closed_form(N, e) + 1e-9
    assert np.max(np.abs(out[1] - out[0])) < 1e-7
    assert np.max(np.abs(out[2] - out[0])) < 1e-7
    assert np.max(np.abs(out[3] - out[0])) < 1e-9


def test_config5_width_precisions_agree(rgflib):
    # N = 1001 (KL = 501, the 2002-orbital ribbon): four row tiles and four
    # accumulation groups; the four precisions agree and respect 0 <= T <= n_ch
    N, L = 1001, 3
    eps = workloads.anderson_onsite(N, L, 0.1, 5)
    rem = workloads.edge_removed(N, L, 0.02, 55)
    Es = np.array([-0.27, 0.08])
    out = {}
    for prec in (0, 1, 2, 3):
        T, st = _run(rgflib, N, L, Es, eps, rem, prec)
        assert (st == 0).all()
        out[prec] = T
    for e, t in zip(Es, out[0]):
        assert -1e-9 <= t <= bands.channels_closed_form(N, e) + 1e-9
    assert np.max(np.abs(out[1] - out[0])) < 1e-7
    assert np.max(np.abs(out[2] - out[0])) < 1e-7
    assert np.max(np.abs(out[3] - out[0])) < 1e-9


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_pair_steps_and_their_fallback_near_onsite_resonances(rgflib, prec):
    # Pairs of t I-bonded columns take one inverse; a second column with an
    # atom within 1e-4 eV of E (|z - eps| small, an isolated-atom resonance)
    # is stepped one column at a time instead.  Both against the oracle.
    N, L = 23, 12
    E = 0.13
    eps = workloads.anderson_onsite(N, L, 0.25, 5)
    for cell, delta in ((3, 3e-5), (5, -2e-6), (8, 5e-4), (9, -1e-9)):
        eps[cell, 2 * 4 + 1] = E + delta        # right atom of row 4 (second column c1)
        eps[cell, 2 * 5 + 1] = E - delta        # right atom of row 5 (second column c3)
    rem = workloads.edge_removed(N, L, 0.3, 9)
    T, st = _run(rgflib, N, L, np.array([E, -0.4]), eps, rem, prec)
    assert (st == 0).all()
    tol = 1e-9 if prec in (0, 3) else 1e-7
    for e, t in zip((E, -0.4), T):
        ref = _oracle_T(N, L, e, 1e-8, 1e-8, eps, rem)
        assert abs(t - ref) < tol, (e, t, ref)
