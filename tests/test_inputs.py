"""Seeded input generators (no GPU)."""
import numpy as np

import workloads


def test_splitmix64_reference_output():
    # First output of SplitMix64 seeded with 0 (Steele, Lea, Flood 2014;
    # the value of the public reference implementation).
    assert int(workloads.splitmix64(0, 0)) == 0xE220A8397B1DCDAF
    assert int(workloads.splitmix64(0, 1)) == 0x6E789E6AA1B965F4


def test_anderson_range_and_moments():
    eps = workloads.anderson_onsite(245, 40, 0.25, 1)
    assert eps.shape == (40, 490)
    assert eps.min() >= -0.25 and eps.max() <= 0.25
    assert abs(eps.mean()) < 0.01
    assert abs(eps.var() - 0.25 ** 2 / 3) < 0.002


def test_edge_roughness_only_outer_rows():
    N, L, p = 51, 400, 0.05
    rem = workloads.edge_removed(N, L, p, 8)
    rows = np.arange(2 * N) // 2
    assert rem[:, (rows != 0) & (rows != N - 1)].sum() == 0
    frac = rem[:, (rows == 0) | (rows == N - 1)].mean()
    assert abs(frac - p) < 0.015


def test_batched_chain_ranges():
    ch = workloads.batched_uneven_chains(256, 3)
    Ns = np.array([c["N"] for c in ch])
    Ls = np.array([c["L"] for c in ch])
    Es = np.array([c["E"] for c in ch])
    assert Ns.min() >= 51 and Ns.max() <= 401
    assert Ls.min() >= 100 and Ls.max() <= 2000
    assert Es.min() >= -1 and Es.max() <= 1
