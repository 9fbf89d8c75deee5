"""Failure detection, with every failure made on the host: a lowered iteration
cap or residual tolerance of the lead decimation, a non-finite energy, and a
slice matrix made exactly singular by the input.  Each comes back as a status
word; no test faults, traps or hangs the GPU."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu
T_HOP = -2.7


@pytest.fixture
def lead_controls(rgflib):
    yield rgflib.set_lead_controls
    rgflib.set_lead_controls(200, 1e-10)      # the defaults


def test_iteration_cap_gives_enoconv(rgflib, lead_controls):
    E = np.array([-0.4, 0.2])
    lead_controls(1, 1e-10)
    with pytest.raises(rgflib.RGFError) as e:
        rgflib.lead_selfenergy(11, E, 1e-8, 0)
    assert e.value.status == rgflib.RGF_ENOCONV
    sig, it = rgflib.lead_selfenergy(11, E, 1e-8, 1, check=False)
    assert np.all(it == -1) and np.isnan(sig).all()
    rib = rgflib.Ribbon(11, 3, T_HOP, W=0.2, seed=1)
    T, st = rgflib.conductance([rib] * 2, E, check=False)
    assert np.all(st == rgflib.RGF_ENOCONV) and np.isnan(T).all()
    lead_controls(200, 1e-10)
    T, st = rgflib.conductance([rib] * 2, E)
    assert np.all(st == 0)


def test_zero_residual_tolerance_gives_enoconv(rgflib, lead_controls):
    # every decimated g_p misses the surface Dyson equation by some rounding
    lead_controls(200, 0.0)
    _, it = rgflib.lead_selfenergy(24, np.array([0.37]), 1e-8, 0, check=False)
    assert it[0] == -1
    lead_controls(200, 1e-10)
    _, it = rgflib.lead_selfenergy(24, np.array([0.37]), 1e-8, 0)
    assert 0 < it[0] < 200


def test_controls_reject_bad_values(rgflib):
    for args in ((0, 1e-10), (200, -1.0), (200, float("nan"))):
        with pytest.raises(rgflib.RGFError) as e:
            rgflib.set_lead_controls(*args)
        assert e.value.status == rgflib.RGF_EINVAL


def test_nonfinite_energy_is_einval_per_chain(rgflib):
    import torch
    rib = rgflib.Ribbon(11, 4, T_HOP, W=0.2, seed=3)
    Es = np.array([0.3, np.nan, -0.2, np.inf])
    Ed = torch.tensor(Es, dtype=torch.float64, device="cuda")
    Td = torch.empty(4, dtype=torch.float64, device="cuda")
    Sd = torch.empty(4, dtype=torch.int32, device="cuda")
    rgflib.conductance_dev([rib] * 4, Ed.data_ptr(), 4, Td.data_ptr(), Sd.data_ptr())
    torch.cuda.synchronize()
    st, T = Sd.cpu().numpy(), Td.cpu().numpy()
    assert list(st) == [0, rgflib.RGF_EINVAL, 0, rgflib.RGF_EINVAL]
    ref, _ = rgflib.conductance([rib] * 2, Es[[0, 2]])
    assert np.array_equal(T[[0, 2]], ref) and np.isnan(T[[1, 3]]).all()


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_exactly_singular_slice_gives_esingular(rgflib, prec):
    # With no broadening in the device (eta_device = 0) and the left atom of
    # row 0 in the first cell removed, the right atom of row 0 has no bond to
    # the left: its row of the second column's slice matrix is z - eps, exactly
    # zero when its on-site energy equals E.  The left-connected recursion
    # meets an exactly singular matrix (the whole system does not).
    N, L, E = 8, 3, 0.3
    eps = np.zeros((L, 2 * N))
    eps[0, 1] = E
    rem = np.zeros((L, 2 * N), dtype=np.uint8)
    rem[0, 0] = 1
    bad = rgflib.Ribbon(N, L, T_HOP, onsite=eps, removed=rem)
    good = rgflib.Ribbon(N, L, T_HOP, onsite=workloads.anderson_onsite(N, L, 0.1, 2))
    T, st = rgflib.conductance([bad, good], np.array([E, E]), 0.0, 1e-8, prec, check=False)
    assert st[0] == rgflib.RGF_ESINGULAR and np.isnan(T[0])
    assert st[1] == 0 and -1e-9 <= T[1] <= 1.0 + 1e-9
