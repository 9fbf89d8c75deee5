"""Local density of states -Im G_ii / pi (rgf_ldos) against the oracle, element
by element: the Dyson-assembled diagonal blocks of oracle.ldos (disorder and
removed atoms) and, for a pristine device, the Bloch-state LDOS of the
infinite ribbon from its band structure (oracle.bands)."""
import numpy as np
import pytest

import workloads
from oracle import bands, ldos as oldos

pytestmark = pytest.mark.gpu
T_HOP = -2.7


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-8), (2, 1e-8), (3, 1e-9)])
def test_ldos_matches_oracle(rgflib, prec, tol):
    N, L = 11, 6
    eps = workloads.anderson_onsite(N, L, 0.3, 11)
    rem = workloads.edge_removed(N, L, 0.3, 12)
    rib = rgflib.Ribbon(N, L, T_HOP, onsite=eps, removed=rem)
    Es = np.array([-0.9, 0.31, 0.05])
    T, rho, st = rgflib.ldos([rib] * 3, Es, 1e-8, 1e-8, prec, ckpt_stride=2)
    assert (st == 0).all()
    for c, E in enumerate(Es):
        ref = oldos.ldos(N, L, E, 1e-8, 1e-8, T_HOP, eps, rem)
        err = np.abs(rho[c] - ref).max() / np.abs(ref).max()
        print(f"ldos precision={prec} E={E}: max rel |d rho| = {err:.2e}")
        assert err < tol, (E, err)
        assert np.all(rho[c][rem.astype(bool)] == 0.0)


@pytest.mark.parametrize("prec", [0, 2, 3])
def test_ldos_wider_ribbon_and_checkpoint_strides(rgflib, prec):
    # N = 40 (KL = 20): a tensor-core tile per product; strides 1 and 3 give
    # the same values, and the oracle agrees
    N, L = 40, 7
    eps = workloads.anderson_onsite(N, L, 0.2, 40)
    rem = workloads.edge_removed(N, L, 0.1, 41)
    rib = rgflib.Ribbon(N, L, T_HOP, onsite=eps, removed=rem)
    Es = np.array([-0.45, 0.62])
    _, r1, st1 = rgflib.ldos([rib] * 2, Es, 1e-8, 1e-8, prec, ckpt_stride=1)
    _, r3, st3 = rgflib.ldos([rib] * 2, Es, 1e-8, 1e-8, prec, ckpt_stride=3)
    assert (st1 == 0).all() and (st3 == 0).all()
    assert np.array_equal(r1, r3)
    tol = {0: 1e-10, 2: 1e-8, 3: 1e-9}[prec]
    for c, E in enumerate(Es):
        ref = oldos.ldos(N, L, E, 1e-8, 1e-8, T_HOP, eps, rem)
        assert np.abs(r1[c] - ref).max() < tol * np.abs(ref).max()


@pytest.mark.parametrize("N,E", [(5, 0.9), (7, -1.3), (6, 2.2)])
def test_ldos_of_pristine_ribbon_is_the_bloch_ldos(rgflib, N, E):
    # A pristine device between pristine leads (eta_device = 0) is a piece of
    # the infinite ribbon: every cell carries the LDOS of the Bloch states at E.
    b = bands.bloch_ldos(N, E)
    rib = rgflib.Ribbon(N, 5, T_HOP)
    _, rho, st = rgflib.ldos([rib], np.array([E]), 0.0, 1e-8, rgflib.RGF_FP64)
    assert st[0] == 0
    assert np.abs(rho[0] - b[None, :]).max() < 1e-6 * b.max()
