"""The tensor-core complex product (rgf_zgemm_tc, through the C ABI, sliced
from binary64) against complex128 products, with the normwise bound of exact
digit slicing: |C - AB|_mn <= 2^-49 k max_j|A_mj| max_j|B_jn| per real part.
The analysis gives 2^-50.1 in the worst alignment (the dropped digit levels,
the rounding of the sliced significands and of the shared accumulator); the
bound leaves a factor 2, and is 2^3 below what double-float operands allow."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _run(rgflib, A, B, check=True):
    import torch
    m, k = A.shape
    n = B.shape[1]
    Ad = torch.from_numpy(np.ascontiguousarray(A, dtype=np.complex128)).cuda()
    Bd = torch.from_numpy(np.ascontiguousarray(B, dtype=np.complex128)).cuda()
    Cd = torch.full((max(m, 1), max(n, 1)), complex(np.nan, np.nan), dtype=torch.complex128,
                    device="cuda")
    torch.cuda.synchronize()
    st = rgflib.zgemm_tc(Ad.data_ptr(), Bd.data_ptr(), Cd.data_ptr(), m, n, k,
                         lda=max(k, 1), ldb=max(n, 1), ldc=max(n, 1), check=check)
    torch.cuda.synchronize()
    return Cd.cpu().numpy()[:m, :n], st


def _bound(A, B):
    ra = np.maximum(np.abs(A.real), np.abs(A.imag)).max(axis=1)
    cb = np.maximum(np.abs(B.real), np.abs(B.imag)).max(axis=0)
    return 2.0 ** -49 * A.shape[1] * np.outer(ra, cb)


def _check_close(C, A, B):
    # the reference in extended precision: a complex128 product of 128 terms of
    # one sign is itself off by several units of 2^-53 of its sum
    ref = A.astype(np.clongdouble) @ B.astype(np.clongdouble)
    tol = _bound(A, B)
    d = C.astype(np.clongdouble) - ref
    er, ei = np.abs(d.real).astype(np.float64), np.abs(d.imag).astype(np.float64)
    assert np.isfinite(C).all()
    assert (er <= tol).all() and (ei <= tol).all(), (float((er / tol).max()), float((ei / tol).max()))
    return float(max((er / tol).max(), (ei / tol).max()))


def _rand(rng, m, n):
    return rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (5, 3, 7), (37, 64, 8), (123, 123, 123),
                                   (128, 128, 128), (130, 70, 129), (300, 200, 260), (64, 1, 300),
                                   (8, 65, 17)])
def test_matches_complex128(rgflib, m, n, k):
    rng = np.random.default_rng(1000 * m + 10 * n + k)
    A, B = _rand(rng, m, k), _rand(rng, k, n)
    C, _ = _run(rgflib, A, B)
    _check_close(C, A, B)


def test_row_and_column_scales(rgflib):
    # rows of A and columns of B spread over 16 decades each: the per-row and
    # per-column scales keep every entry accurate relative to its own row/column
    rng = np.random.default_rng(7)
    A = _rand(rng, 123, 123) * 10.0 ** rng.uniform(-8, 8, (123, 1))
    B = _rand(rng, 123, 100) * 10.0 ** rng.uniform(-8, 8, (1, 100))
    C, _ = _run(rgflib, A, B)
    _check_close(C, A, B)


def test_real_dominated_operands(rgflib):
    # |Re| >> |Im| (the regime of slice matrices near E = 0)
    rng = np.random.default_rng(8)
    A = rng.standard_normal((100, 90)) * 1e4 + 1j * rng.standard_normal((100, 90)) * 1e-8
    B = rng.standard_normal((90, 110)) * 1e3 + 1j * rng.standard_normal((90, 110)) * 1e-9
    C, _ = _run(rgflib, A, B)
    _check_close(C, A, B)


def test_leading_levels_accumulate_exactly(rgflib):
    # every entry close to its row / column maximum with one sign: the exact
    # digit levels sum up to 5 x 192 x 2^14 < 2^24 terms' worth, near the limit
    # of exact binary32 accumulation; any rounding there would show at ~2^-24
    # relative
    rng = np.random.default_rng(9)
    A = (1.0 - 1e-3 * rng.random((128, 128))) * (1 + 1j)
    B = (1.0 - 1e-3 * rng.random((128, 128))) * (1 + 1j)
    C, _ = _run(rgflib, A, B)
    _check_close(C, A, B)
    A2 = -(1.0 - 1e-7 * rng.random((128, 128))) + 0j
    B2 = (1.0 - 1e-7 * rng.random((128, 128))) + 0j
    C2, _ = _run(rgflib, A2, B2)
    _check_close(C2, A2, B2)


def test_small_integer_inputs_are_exact(rgflib):
    # small integers are exact in the leading digits; their products then too
    rng = np.random.default_rng(10)
    A = rng.integers(-1000, 1000, (40, 50)) + 1j * rng.integers(-1000, 1000, (40, 50))
    B = rng.integers(-1000, 1000, (50, 30)) + 1j * rng.integers(-1000, 1000, (50, 30))
    C, _ = _run(rgflib, A.astype(np.complex128), B.astype(np.complex128))
    assert np.array_equal(C, A @ B)


def test_nonfinite_entry_poisons_only_its_row(rgflib):
    rng = np.random.default_rng(11)
    A, B = _rand(rng, 20, 16), _rand(rng, 16, 12)
    A[3, 5] = np.nan
    C, _ = _run(rgflib, A, B)
    assert not np.isfinite(C[3]).any()
    rows = np.arange(20) != 3
    _check_close(C[rows], A[rows], B)


def test_empty_and_invalid_sizes(rgflib):
    rng = np.random.default_rng(12)
    A, B = _rand(rng, 4, 0), _rand(rng, 0, 3)
    C, _ = _run(rgflib, A, B)
    assert np.array_equal(C, np.zeros((4, 3)))
    st = rgflib.zgemm_tc(0, 0, 0, 3, 3, 5, lda=4, check=False)
    assert st == rgflib.RGF_EINVAL


def test_completion_wait_timeout_is_reported(rgflib):
    # the MMAs' completion is never committed to the barrier the kernel waits
    # on: the bounded wait runs out, the kernel reports it and drains its MMAs
    # before freeing tensor memory; the context stays usable afterwards
    assert rgflib.zgemm_tc_selftest_timeout() == rgflib.RGF_ETIMEOUT
    rng = np.random.default_rng(13)
    A, B = _rand(rng, 64, 64), _rand(rng, 64, 64)
    C, st = _run(rgflib, A, B)
    assert st == rgflib.RGF_OK
    _check_close(C, A, B)
