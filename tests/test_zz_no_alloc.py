"""The allocation-free entry point, called through the C ABI, gives the same
conductances as the allocating one, on two calls in a row, and allocates no
device memory.  (Collected last so that a run stopping at the first failure
has run everything else.)

It serves callers that may not allocate device memory (a host that reserved
the device memory for its own pool, a plugin handed only pre-allocated
buffers, a loop that must avoid the synchronisation of cudaMalloc): its
scratch is a fixed 64 MiB array inside the library."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def _bufs(torch, n):
    return (torch.empty(n, dtype=torch.float64, device="cuda"),
            torch.empty(n, dtype=torch.int32, device="cuda"))


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
    T_d, S_d = _bufs(torch, len(Es))
    for prec, tol in ((rgflib.RGF_FP64, 1e-9), (rgflib.RGF_MIXED, 1e-7), (rgflib.RGF_MIXED_TC, 1e-7),
                      (rgflib.RGF_FP64_TC, 1e-9)):
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


def test_noalloc_allocates_nothing_and_takes_null_options(rgflib):
    import torch
    N, L = 31, 5
    eps = workloads.anderson_onsite(N, L, 0.2, 3)
    Es = np.array([-0.3, 0.11, 0.6])
    rib = rgflib.Ribbon(N, L, -2.7, onsite=eps)
    T_ref, _ = rgflib.conductance([rib] * 3, Es, 1e-8, 1e-8, rgflib.RGF_FP64)
    eps_d = torch.tensor(eps, dtype=torch.float64, device="cuda")
    E_d = torch.tensor(Es, dtype=torch.float64, device="cuda")
    T_d, _ = _bufs(torch, 3)
    call = lambda: rgflib.conductance_noalloc(N, L, -2.7, eps_d.data_ptr(), 0, E_d.data_ptr(), 3,
                                              T_d.data_ptr(), 0, 1e-8, 1e-8, rgflib.RGF_FP64)
    call()                                   # first call on the device: the array is set up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    T_d.fill_(float("nan"))
    call()                                   # removed and status pointers NULL
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert np.max(np.abs(T_d.cpu().numpy() - T_ref)) < 1e-9


def test_noalloc_at_its_limit(rgflib):
    # N = 245 (the bench ribbon's width): 21 energies fill the 64 MiB scratch
    # array to its end and give the allocating entry point's values; 22 do
    # not fit and are refused.
    import torch
    N, L, n = 245, 3, 21
    eps = workloads.anderson_onsite(N, L, 0.25, 1)
    Es = np.linspace(-0.5, 0.5, n)
    rib = rgflib.Ribbon(N, L, -2.7, onsite=eps)
    eps_d = torch.tensor(eps, dtype=torch.float64, device="cuda")
    E_d = torch.tensor(Es, dtype=torch.float64, device="cuda")
    T_ref, S_ref = _bufs(torch, n)
    T_d, S_d = _bufs(torch, n)
    rgflib.conductance_dev([rib] * n, E_d.data_ptr(), n, T_ref.data_ptr(), S_ref.data_ptr(),
                           precision=rgflib.RGF_MIXED_TC)
    rgflib.conductance_noalloc(N, L, -2.7, eps_d.data_ptr(), 0, E_d.data_ptr(), n, T_d.data_ptr(),
                               S_d.data_ptr(), 1e-8, 1e-8, rgflib.RGF_MIXED_TC)
    torch.cuda.synchronize()
    assert (S_d.cpu().numpy() == 0).all() and (S_ref.cpu().numpy() == 0).all()
    assert np.array_equal(T_d.cpu().numpy(), T_ref.cpu().numpy())
    E22 = torch.zeros(n + 1, dtype=torch.float64, device="cuda")
    T22, _ = _bufs(torch, n + 1)
    st = rgflib.conductance_noalloc(N, L, -2.7, eps_d.data_ptr(), 0, E22.data_ptr(), n + 1,
                                    T22.data_ptr(), check=False)
    assert st == rgflib.RGF_EINVAL
    assert "64 MiB" in rgflib.lib.rgf_last_error().decode()


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
