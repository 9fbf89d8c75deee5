"""The bench workload at its full size, in the launch the benchmark times (69
chains, two-block clusters): the W = 30 nm ribbon (N = 245, M = 490 orbitals
per cell), L = 4000 cells, Anderson disorder +-0.25 eV, 69 energies.  The
oracle cannot sweep 4000 cells of this ribbon in a test, so every chain is
checked against the binary64 GPU path (|dT| <= 1e-6 per energy, the target of
the mixed-precision paths) and against the bounds 0 <= T <= n_ch(E); both
mixed paths must report the same status as binary64 (E = 0 exactly is
condition-limited and is flagged RGF_EBOUNDS rather than returned)."""
import numpy as np
import pytest

import workloads
from oracle import bands

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bench_case(rgflib):
    w = workloads.WORKLOADS["agnr245_L4000_anderson"]
    N, L = w["N"], w["L"]
    eps = workloads.anderson_onsite(N, L, w["W"], w["seed"])
    Es = w["energies"]()
    rib = rgflib.Ribbon(N, L, -2.7, onsite=eps)
    T64, s64 = rgflib.conductance([rib] * len(Es), Es, 1e-8, 1e-8, rgflib.RGF_FP64, check=False)
    return rib, N, Es, T64, s64


@pytest.mark.parametrize("prec", [1, 2])
def test_mixed_paths_match_binary64_at_full_size(rgflib, bench_case, prec):
    rib, N, Es, T64, s64 = bench_case
    T, st = rgflib.conductance([rib] * len(Es), Es, 1e-8, 1e-8, prec, check=False)
    assert np.array_equal(st, s64)
    ok = s64 == 0
    assert ok.sum() >= len(Es) - 1                      # only E = 0 may be flagged
    assert np.all(s64[Es != 0.0] == 0)
    d = np.abs(T[ok] - T64[ok])
    assert d.max() <= 1e-6, d.max()
    nch = np.array([bands.channels_closed_form(N, e) for e in Es[ok]])
    assert np.all(T64[ok] >= -1e-9) and np.all(T64[ok] <= nch + 1e-9)
