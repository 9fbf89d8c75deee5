"""The allocation-free entry point, called through the C ABI, gives the same
conductances as the allocating one, on two calls in a row.  (Collected last so
that a run stopping at the first failure has run everything else.)"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def test_noalloc_matches_allocating_entry_point(rgflib):
    import torch
    N, L = 23, 7
    eps = workloads.anderson_onsite(N, L, 0.25, 21)
    rem = workloads.edge_removed(N, L, 0.2, 22)
    Es = np.array([-0.8, -0.05, 0.003, 0.27, 1.3])
    rib = rgflib.Ribbon(N, L, -2.7, onsite=eps, removed=rem)
    eps_d = torch.tensor(eps, dtype=torch.float64, device="cuda")
    rem_d = torch.tensor(rem, dtype=torch.uint8, device="cuda")
    E_d = torch.tensor(Es, dtype=torch.float64, device="cuda")
    T_d = torch.empty(len(Es), dtype=torch.float64, device="cuda")
    S_d = torch.empty(len(Es), dtype=torch.int32, device="cuda")
    for prec, tol in ((rgflib.RGF_FP64, 1e-9), (rgflib.RGF_MIXED, 1e-7)):
        T_ref, st_ref = rgflib.conductance([rib] * len(Es), Es, 1e-8, 1e-8, prec)
        for _ in range(2):
            T_d.fill_(float("nan"))
            S_d.fill_(-1)
            torch.cuda.synchronize()
            rgflib.conductance_noalloc(N, L, -2.7, eps_d.data_ptr(), rem_d.data_ptr(),
                                       E_d.data_ptr(), len(Es), T_d.data_ptr(), S_d.data_ptr(),
                                       1e-8, 1e-8, prec)
            torch.cuda.synchronize()
            assert (S_d.cpu().numpy() == st_ref).all()
            assert np.max(np.abs(T_d.cpu().numpy() - T_ref)) < tol


def test_noalloc_rejects_sizes_beyond_its_scratch(rgflib):
    import torch
    N, L, n = 1001, 2, 64
    eps_d = torch.zeros((L, 2 * N), dtype=torch.float64, device="cuda")
    E_d = torch.zeros(n, dtype=torch.float64, device="cuda")
    T_d = torch.empty(n, dtype=torch.float64, device="cuda")
    st = rgflib.conductance_noalloc(N, L, -2.7, eps_d.data_ptr(), 0, E_d.data_ptr(), n,
                                    T_d.data_ptr(), check=False)
    assert st == rgflib.RGF_EINVAL
    assert "64 MiB" in rgflib.lib.rgf_last_error().decode()
