"""Pins of the CPU oracle against facts fixed by the paper and by the mathematics
(no GPU).  Each test names the passage or the property it checks."""
import json
from pathlib import Path

import numpy as np
import pytest

import workloads
from oracle import bands, dense, gradient, lattice, ldos, leads, mp, rgf

T_HOP = -2.7
GOLDEN = Path(__file__).resolve().parent / "golden"


def test_lattice_bonds_and_coordination():
    # Honeycomb lattice, one p orbital per atom (text around Fig. 1(a)): every atom
    # has at most 3 neighbours, interior atoms exactly 3; H01 has N-1 bonds.
    for N in (2, 5, 11, 12):
        H00, H01 = lattice.blocks(N, T_HOP)
        assert np.allclose(H00, H00.T)
        deg = (np.abs(H00) > 0).sum(1) + (np.abs(H01) > 0).sum(1) + (np.abs(H01) > 0).sum(0)
        assert deg.max() == (2 if N == 2 else 3)
        assert (np.abs(H01) > 0).sum() == N - 1
        # interior rows (1..N-2) are fully coordinated
        for j in range(1, N - 1):
            assert deg[2 * j] == 3 and deg[2 * j + 1] == 3


def test_band_edges_closed_form_vs_band_structure():
    # Step-like conductance in multiples of 2e^2/h (Fig. 3 discussion): the
    # closed-form channel count equals a brute-force band-structure count.
    for N in (2, 5, 11, 12, 13):
        _, bs = bands.band_structure(N, nk=4001)
        for E in np.linspace(-3.3, 3.3, 37):
            if np.min(np.abs(np.abs(E) - np.abs(T_HOP) * np.abs(
                    1 + 2 * np.cos(np.arange(1, N + 1) * np.pi / (N + 1))))) < 1e-2:
                continue
            assert bands.channels_closed_form(N, E) == bands.channels_band_structure(N, E, bands=bs), (N, E)


def test_metallic_armchair_has_one_channel_at_low_energy():
    # N = 3q + 2 armchair ribbons are metallic; N = 11 has one channel on [-1, 1] eV,
    # E = 0 included (the linear crossing of the metallic mode; the 40-digit
    # T(0) of tests/golden/mp_transmission.json is 0.99999985); N = 3q + 1 has a gap.
    for E in np.linspace(-1, 1, 21):
        assert bands.channels_closed_form(11, E) == 1
    assert bands.channels_closed_form(245, 0.0) == 1
    assert bands.channels_closed_form(245, 0.5) == 17
    assert bands.channels_closed_form(7, 0.0) == 0 and bands.channels_closed_form(7, 0.3) == 0


def _chain_surface(E, eta, t=T_HOP):
    # Semi-infinite monatomic chain: g = (z - sqrt(z^2 - 4 t^2)) / (2 t^2), Im g < 0.
    z = E + 1j * eta
    s = np.sqrt(z * z - 4 * t * t + 0j)
    g1, g2 = (z - s) / (2 * t * t), (z + s) / (2 * t * t)
    return g1 if g1.imag < 0 else g2


def test_decimation_matches_monatomic_chain_closed_form():
    # N = 2 is a monatomic chain (4 atoms per cell, all hoppings t): Sigma = t^2 g_chain.
    for E in (-4.0, -1.3, 0.2, 2.5, 6.0):
        sL, sR = leads.self_energies(2, E, 1e-8, T_HOP)
        ref = T_HOP ** 2 * _chain_surface(E, 1e-8)
        assert abs(sR[3, 3] - ref) < 1e-10 * max(1, abs(ref))
        assert abs(sL[0, 0] - ref) < 1e-10 * max(1, abs(ref))
        mask = np.ones_like(sR, dtype=bool)
        mask[3, 3] = False
        assert np.abs(sR[mask]).max() == 0.0


def test_decimation_fixed_point_residual_and_symmetry():
    for N in (5, 11, 12):
        H00, H01 = lattice.blocks(N, T_HOP)
        for E in (-0.9, 0.01, 0.37, 1.7):
            z = E + 1e-8j
            gR, it = leads.surface_green(H00, H01, H01.T, z)
            assert it < 60
            assert leads.fixed_point_residual(gR, H00, H01, H01.T, z) < 1e-10
            assert np.abs(gR - gR.T).max() < 1e-10 * np.abs(gR).max()


def test_eq2_forms_agree_and_rgf_equals_dense_definition():
    # Eq. 2 as printed (Tr[G_L G^a G_R G^r]) equals Tr[G_L G_1L G_R G_1L^+]; the
    # recursion of Eqs. 4-5 reaches the dense inverse of Eq. 1.
    N, L = 11, 7
    eps = workloads.anderson_onsite(N, L, 0.25, 3)
    rem = workloads.edge_removed(N, L, 0.3, 4)
    assert rem.sum() > 0
    for E in (-0.77, -0.1, 0.003, 0.45):
        Td = dense.transmission_dense(N, L, E, 1e-8, 1e-8, T_HOP, eps, rem)
        Tp = dense.transmission_dense_paper_form(N, L, E, 1e-8, 1e-8, T_HOP, eps, rem)
        Tr = rgf.transmission(N, L, E, 1e-8, 1e-8, T_HOP, eps, rem)
        assert abs(Tp - Td) < 1e-12
        assert abs(Tr - Td) < 1e-11
        assert 0.0 <= Tr <= bands.channels_closed_form(N, E) + 1e-12


def test_reciprocity():
    N, L = 12, 6
    eps = workloads.anderson_onsite(N, L, 0.4, 9)
    rem = workloads.edge_removed(N, L, 0.2, 10)
    for E in (-1.1, 0.2, 0.9):
        a = rgf.transmission(N, L, E, 1e-8, 1e-8, T_HOP, eps, rem)
        b = rgf.transmission_right_to_left(N, L, E, 1e-8, 1e-8, T_HOP, eps, rem)
        assert abs(a - b) < 1e-12


def test_pristine_ribbon_is_quantised():
    # Ideal ribbon: T is the number of propagating channels (Fig. 3 discussion),
    # exactly when no absorption is added inside the device (eta_device = 0).
    for N in (5, 11, 12):
        for E in (0.15, -0.6, 1.4, -2.3):
            n = bands.channels_closed_form(N, E)
            T = rgf.transmission(N, 15, E, 0.0, 1e-8, T_HOP)
            assert abs(T - n) < 1e-9, (N, E, T, n)


def test_eta_absorption_is_linear_in_eta_and_length():
    # With eta_device > 0 the device absorbs: n_ch - T = O(eta * L).
    N, E = 11, 0.5
    d1 = 1.0 - rgf.transmission(N, 20, E, 1e-8, 1e-8, T_HOP)
    d2 = 1.0 - rgf.transmission(N, 20, E, 2e-8, 1e-8, T_HOP)
    d3 = 1.0 - rgf.transmission(N, 40, E, 1e-8, 1e-8, T_HOP)
    assert d1 > 0
    assert abs(d2 / d1 - 2.0) < 1e-3
    assert abs(d3 / d1 - 2.0) < 1e-3


def test_gradient_adjoint_closed_form_and_finite_differences():
    N, L, E = 11, 6, 0.31
    eps = workloads.anderson_onsite(N, L, 0.3, 11)
    rem = workloads.edge_removed(N, L, 0.3, 12)
    T, gadj = gradient.adjoint(N, L, E, 1e-8, 1e-8, T_HOP, eps, rem)
    gcf = gradient.closed_form(N, L, E, 1e-8, 1e-8, T_HOP, eps, rem)
    assert np.abs(gadj - gcf).max() < 1e-12 * max(1.0, np.abs(gcf).max())
    assert np.all(gcf[rem.astype(bool)] == 0.0)
    rng = np.random.default_rng(0)
    d = 1e-6
    for _ in range(6):
        n, i = rng.integers(L), rng.integers(2 * N)
        if rem[n, i]:
            continue
        ep, em = eps.copy(), eps.copy()
        ep[n, i] += d
        em[n, i] -= d
        fd = (rgf.transmission(N, L, E, 1e-8, 1e-8, T_HOP, ep, rem)
              - rgf.transmission(N, L, E, 1e-8, 1e-8, T_HOP, em, rem)) / (2 * d)
        assert abs(fd - gcf[n, i]) < 1e-8 + 1e-5 * abs(gcf[n, i])


@pytest.mark.parametrize("E,eta_d", [(0.31, 1e-8), (-0.9, 1e-8), (0.004, 1e-8), (0.52, 0.0)])
def test_gradient_two_sided_matches_closed_form(E, eta_d):
    # The Dyson-assembled blocks (Eq. 3 with one bond cut) against the dense G
    # of Eq. 1, with removed atoms (ragged slices).
    N, L = 11, 6
    eps = workloads.anderson_onsite(N, L, 0.3, 11)
    rem = workloads.edge_removed(N, L, 0.3, 12)
    T, g = gradient.two_sided(N, L, E, eta_d, 1e-8, T_HOP, eps, rem)
    gcf = gradient.closed_form(N, L, E, eta_d, 1e-8, T_HOP, eps, rem)
    assert np.abs(g - gcf).max() < 1e-12 * max(1.0, np.abs(gcf).max())
    assert np.all(g[rem.astype(bool)] == 0.0)
    assert abs(T - dense.transmission_dense(N, L, E, eta_d, 1e-8, T_HOP, eps, rem)) < 1e-12


def test_gradient_two_sided_near_half_system_poles():
    # Near E = 0 the ends of the half systems left and right of a cut carry
    # nearly bound states; the two-sided form stays at the dense closed form
    # (here within 1e-8 of the gradient's scale; the reverse sweep of the same
    # recursion is off by about 2.5e-5 of it on this ribbon)
    N, L = 20, 40
    eps = workloads.anderson_onsite(N, L, 0.15, 7)
    E = float(np.linspace(-0.12, 0.12, 12)[2])
    _, g = gradient.two_sided(N, L, E, 1e-8, 1e-8, T_HOP, eps)
    gcf = gradient.closed_form(N, L, E, 1e-8, 1e-8, T_HOP, eps)
    assert np.abs(g - gcf).max() < 1e-8 * np.abs(gcf).max()


@pytest.mark.parametrize("E", [0.31, -0.9])
def test_ldos_matches_dense_diagonal(E):
    # -Im G_ii / pi from the Dyson-assembled diagonal blocks against the dense
    # G of Eq. 1 (disorder, removed atoms)
    N, L = 11, 6
    eps = workloads.anderson_onsite(N, L, 0.3, 11)
    rem = workloads.edge_removed(N, L, 0.3, 12)
    r = ldos.ldos(N, L, E, 1e-8, 1e-8, T_HOP, eps, rem)
    G, off, keep, _, _ = dense.green_dense(N, L, E, 1e-8, 1e-8, T_HOP, eps, rem)
    ref = np.zeros((L, 2 * N))
    for n in range(L):
        ref[n, keep[n]] = -np.imag(np.diag(G)[off[n]:off[n + 1]]) / np.pi
    assert np.abs(r - ref).max() < 1e-12 * np.abs(ref).max()
    assert np.all(r[rem.astype(bool)] == 0.0) and np.all(r >= 0.0)


@pytest.mark.parametrize("N,E", [(5, 0.9), (7, -1.3), (6, 2.2)])
def test_ldos_of_pristine_ribbon_is_the_bloch_ldos(N, E):
    # A pristine device between pristine leads (eta_device = 0) is a piece of
    # the infinite ribbon: every cell has the LDOS of its Bloch states at E,
    # computed from the band structure (band crossings, Hellmann-Feynman slopes)
    b = bands.bloch_ldos(N, E)
    r = ldos.ldos(N, 5, E, 0.0, 1e-8, T_HOP)
    assert np.abs(r - b[None, :]).max() < 1e-6 * b.max()


def test_gradient_sums_to_uniform_shift_derivative():
    # The derivative along a uniform shift of every device on-site energy is the
    # sum of the gradient.
    N, L, E = 5, 5, 0.4
    eps = workloads.anderson_onsite(N, L, 0.2, 5)
    _, g = gradient.adjoint(N, L, E, 0.0, 1e-8, T_HOP, eps, None)
    d = 1e-6
    Tp = rgf.transmission(N, L, E, 0.0, 1e-8, T_HOP, eps + d)
    Tm = rgf.transmission(N, L, E, 0.0, 1e-8, T_HOP, eps - d)
    assert abs(g.sum() - (Tp - Tm) / (2 * d)) < 1e-7


def test_complex128_against_arbitrary_precision_golden():
    # 40-digit values written by tests/golden/make_golden.py (oracle.mp only).
    g = json.loads((GOLDEN / "mp_transmission.json").read_text())
    for name, v in g.items():
        eps = workloads.anderson_onsite(v["N"], v["L"], v["W"], v["seed"]) if v["W"] > 0 else None
        T = rgf.transmission(v["N"], v["L"], v["E"], v["eta_device"], v["eta_lead"], T_HOP, eps)
        if v["E"] == 0.0:
            # E = 0 exactly is condition-limited in complex128 (edge-state pole of
            # the leads): the error is large but bounded.
            assert abs(T - v["T"]) < 5e-3, name
        else:
            assert abs(T - v["T"]) < 1e-10, name


def test_mp_recursion_matches_complex128_when_well_conditioned():
    N, L, E = 5, 4, 0.37
    eps = workloads.anderson_onsite(N, L, 0.2, 2)
    a = mp.transmission(N, L, E, 1e-8, 1e-8, T_HOP, eps, dps=30)
    b = rgf.transmission(N, L, E, 1e-8, 1e-8, T_HOP, eps)
    assert abs(a - b) < 1e-12


# ---------------------------------------------------------------------------
# Lead self-energies in the transverse-mode basis (oracle.modes) and the
# recursion with the end slices in that basis (oracle.rgf.transmission_modes).
# ---------------------------------------------------------------------------
from oracle import modes  # noqa: E402


@pytest.mark.parametrize("N", [2, 3, 5, 11, 12, 24])
def test_mode_self_energies_equal_full_cell_decimation(N):
    # The closed form (root of the mode chain's surface Dyson equation) is the
    # value the full-cell Sancho-Rubio iteration converges to (text after
    # Eqs. 4-5: the self-energies enter at the first and the last slice).
    for E in (-1.3, -0.2, 0.003, 0.4, 1.7, 3.1):
        a = modes.self_energies(N, E, 1e-8, T_HOP)
        b = leads.self_energies(N, E, 1e-8, T_HOP)
        for x, y in zip(a, b):
            assert np.abs(x - y).max() < 1e-10 * max(1.0, np.abs(y).max()), (N, E)


def test_mode_surface_green_function_special_cases():
    # tau = t: the mode chain is the monatomic chain (textbook closed form);
    # every root is the retarded one (Im g < 0) and a fixed point of the
    # surface Dyson equation.
    for E in (-3.0, -0.7, 0.0, 0.4, 5.5):
        g = modes.surface_green(E + 1e-8j, T_HOP, T_HOP)
        assert abs(g - _chain_surface(E, 1e-8)) < 1e-12 * abs(g)
    for N in (5, 11, 24):
        for E in (0.0, 1e-3, 0.4, 2.0):
            assert modes.dyson_residual(N, E, 1e-8, T_HOP) < 1e-13
            assert np.all(modes.mode_self_energies(N, E, 1e-8, T_HOP).imag <= 0.0)


def test_mode_vectors_diagonalise_the_decimated_self_energy():
    N, E = 12, 0.37
    UL, UR = modes.mode_vectors(N)
    assert np.abs(UL.T @ UL - np.eye(UL.shape[0])).max() < 1e-13
    assert np.abs(UR.T @ UR - np.eye(UR.shape[0])).max() < 1e-13
    sL, sR = leads.self_energies(N, E, 1e-8, T_HOP)
    iL, iR = modes.left_orbitals(N), modes.right_orbitals(N)
    w = modes.mode_self_energies(N, E, 1e-8, T_HOP)
    dL = UL.T @ sL[np.ix_(iL, iL)] @ UL
    dR = UR.T @ sR[np.ix_(iR, iR)] @ UR
    assert np.abs(dL - np.diag(w)).max() < 1e-10 * np.abs(w).max()
    assert np.abs(dR - np.diag(w[:UR.shape[0]])).max() < 1e-10 * np.abs(w).max()


def test_mode_self_energies_at_charge_neutrality_vs_40_digits():
    # At E = 0 the surface-state modes give |Sigma| ~ 1e9 eV; the closed form
    # keeps full relative accuracy against 40-digit decimation (oracle.mp).
    for N in (5, 6):
        sL, sR = mp.self_energies(N, 0.0, 1e-8, T_HOP, dps=40)
        a = modes.self_energies(N, 0.0, 1e-8, T_HOP)
        assert np.abs(a[0] - sL).max() < 1e-13 * np.abs(sL).max()
        assert np.abs(a[1] - sR).max() < 1e-13 * np.abs(sR).max()


def test_mp_self_energies_match_decimation_when_well_conditioned():
    sL, sR = mp.self_energies(5, 0.37, 1e-8, T_HOP, dps=30)
    a, b = leads.self_energies(5, 0.37, 1e-8, T_HOP)
    assert np.abs(sL - a).max() < 1e-12 * np.abs(a).max()
    assert np.abs(sR - b).max() < 1e-12 * np.abs(b).max()


@pytest.mark.parametrize("N,L,p", [(5, 1, 0.0), (11, 3, 0.0), (12, 7, 0.0), (23, 5, 0.3), (2, 3, 0.0)])
def test_transmission_modes_equals_recursion_and_dense(N, L, p):
    # An orthogonal change of basis on the lead-attached atoms of the end slices
    # changes neither G_1L's trace (Eq. 2) nor the recursion (Eqs. 4-5).
    eps = workloads.anderson_onsite(N, L, 0.25, 100 + N)
    rem = None
    if p > 0:
        rem = workloads.edge_removed(N, L, p, 7)
        rem[0, modes.left_orbitals(N)] = 0
        rem[-1, modes.right_orbitals(N)] = 0
    for E in (-1.1, -0.3, 0.02, 0.45):
        a = rgf.transmission_modes(N, L, E, 1e-8, 1e-8, T_HOP, eps, rem)
        b = rgf.transmission(N, L, E, 1e-8, 1e-8, T_HOP, eps, rem)
        c = dense.transmission_dense(N, L, E, 1e-8, 1e-8, T_HOP, eps, rem)
        assert abs(a - b) < 1e-11 and abs(a - c) < 1e-11, (N, L, E, a, b, c)


def test_transmission_modes_at_charge_neutrality_vs_40_digits():
    # E = 0 exactly (eta = 1e-8 eV): with the end slices in the mode basis the
    # complex128 recursion meets the 40-digit values to 1e-9 on the disordered
    # ribbon (measured 3.1e-10; the site-basis recursion is off by 7.5e-5) and to
    # 2e-7 on the pristine one, whose every partial system carries a surface
    # state at E = 0 (measured 5.2e-8; site basis: 1.6e-3).
    g = json.loads((GOLDEN / "mp_transmission.json").read_text())
    for name, tol in (("agnr5_L8_anderson_E0", 1e-9), ("agnr11_L10_pristine_E0", 2e-7),
                      ("agnr5_L8_anderson_E1e-3", 1e-12), ("agnr11_L10_pristine_E1e-4", 1e-12)):
        v = g[name]
        eps = workloads.anderson_onsite(v["N"], v["L"], v["W"], v["seed"]) if v["W"] > 0 else None
        T = rgf.transmission_modes(v["N"], v["L"], v["E"], v["eta_device"], v["eta_lead"], T_HOP, eps)
        assert abs(T - v["T"]) < tol, (name, T - v["T"])


def test_removed_atom_is_the_infinite_onsite_limit():
    # Dropping an atom (its orbital removed from its slice) is the limit of an
    # infinite on-site energy on it: T and the gradient at the other sites
    # approach the dropped values as 1/eps.
    N, L, E = 11, 4, 0.31
    eps = workloads.anderson_onsite(N, L, 0.2, 8)
    rem = np.zeros((L, 2 * N), dtype=np.uint8)
    sites = [(1, 0), (2, 2 * N - 1), (3, 1)]
    for n, o in sites:
        rem[n, o] = 1
    T_drop = rgf.transmission(N, L, E, 1e-8, 1e-8, T_HOP, eps, rem)
    g_drop = gradient.closed_form(N, L, E, 1e-8, 1e-8, T_HOP, eps, rem)
    devs = []
    for big in (1e6, 1e7):
        e2 = eps.copy()
        for n, o in sites:
            e2[n, o] = big
        T_big = rgf.transmission(N, L, E, 1e-8, 1e-8, T_HOP, e2, None)
        g_big = gradient.closed_form(N, L, E, 1e-8, 1e-8, T_HOP, e2, None)
        devs.append(abs(T_big - T_drop))
        assert np.abs(g_big - g_drop).max() < 100.0 / big * max(1.0, np.abs(g_drop).max())
    assert devs[1] < 1e-5 and devs[1] < 0.2 * devs[0] + 1e-12
