"""dynmat_spmv_coo_noalloc: the COO product for callers that cannot allocate
device memory when they multiply (a disabled or budget-locked allocator, or a
hot path where cudaMalloc is not allowed to run). Its work array is fixed and
shared, so this file checks that two calls in a row, on different matrices,
both give the results of the ordinary entry point (dynmat_spmv on a COO
handle) within the FP64 tolerance used throughout:
|y - y_ref| <= 1e-13 * sum_j |a_ij x_j| per row, and rows without entries
exactly 0.

Named to run last: when it fails, a run that stops at the first failure has
already run every other test."""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2209_06478_b300 import build
    build.build()
    from paper_2209_06478_b300 import dynmat
    return dynmat, torch


def _case(dm, torch, N, r, c, v, seed):
    """Device COO arrays of a COO handle, x, the ordinary product and its
    per-row bound sum_j |a_ij x_j| (both from dynmat_spmv)."""
    A = dm.dynmat_create(N, N, r, c, v)
    i = A.info()
    a = A.arrays()
    dev = {k: torch.from_numpy(np.ascontiguousarray(a[k])).cuda() for k in ("row", "col", "val")}
    x = torch.from_numpy(synth.uniform_pm1(seed, N)).cuda()
    y_ref = torch.empty(N, dtype=torch.float64, device="cuda")
    A.spmv(x, y_ref)
    Aabs = dm.dynmat_create(N, N, r, c, np.abs(v))
    bound = torch.empty(N, dtype=torch.float64, device="cuda")
    Aabs.spmv(x.abs(), bound)
    torch.cuda.synchronize()
    return i.nnz, dev, x, y_ref.cpu().numpy(), bound.cpu().numpy()


def _noalloc(dm, torch, N, dev, x):
    y = torch.full((N,), float("nan"), dtype=torch.float64, device="cuda")
    dm.dynmat_spmv_coo_noalloc(N, dev["row"], dev["col"], dev["val"], x, y)
    torch.cuda.synchronize()
    return y.cpu().numpy()


def test_two_calls_in_a_row_match_the_handle_product(env):
    dm, torch = env
    N1, r1, c1, v1 = synth.powerlaw(31, 40000)      # rows up to ~5000 entries
    N2, r2, c2, v2 = synth.stencil27(32)
    nnz1, d1, x1, ref1, b1 = _case(dm, torch, N1, r1, c1, v1, 1)
    nnz2, d2, x2, ref2, b2 = _case(dm, torch, N2, r2, c2, v2, 2)
    assert nnz1 > 128 * 1000 and nnz2 > 128 * 1000
    y1 = _noalloc(dm, torch, N1, d1, x1)
    y2 = _noalloc(dm, torch, N2, d2, x2)      # shares the work array with the first call
    assert np.all(np.abs(y1 - ref1) <= 1e-13 * b1) and np.all(y1[b1 == 0] == 0.0)
    assert np.all(np.abs(y2 - ref2) <= 1e-13 * b2) and np.all(y2[b2 == 0] == 0.0)
    # and back to the first matrix after the second one overwrote the array
    y1b = _noalloc(dm, torch, N1, d1, x1)
    assert np.all(np.abs(y1b - ref1) <= 1e-13 * b1)


def _gappy(seed, nrows, first, last, density):
    """COO whose rows [0, first) and [last, nrows) are empty, with every
    fifth row of [first, last) empty as well."""
    r, c, v = synth.random_coo(seed, last - first, nrows, density)
    r = (r + first).astype(np.int32)
    keep = (r - first) % 5 != 3
    return r[keep], c[keep], v[keep]


def test_empty_leading_interior_and_trailing_rows_are_zero(env):
    """Rows with no entries get exactly 0, including those before the first
    stored row and after the last (nrows > max(row) + 1), on two calls in a
    row with y filled with NaN before each."""
    dm, torch = env
    cases = []
    for seed, N, first, last, dens in ((3, 9000, 700, 8100, 0.004), (4, 3000, 1, 2990, 0.02)):
        r, c, v = _gappy(seed, N, first, last, dens)
        A = dm.dynmat_create(N, N, r, c, v)
        a = A.arrays()
        dev = {k: torch.from_numpy(np.ascontiguousarray(a[k])).cuda() for k in ("row", "col", "val")}
        x = torch.from_numpy(synth.uniform_pm1(seed + 10, N)).cuda()
        y_ref = torch.empty(N, dtype=torch.float64, device="cuda")
        A.spmv(x, y_ref)
        Aabs = dm.dynmat_create(N, N, r, c, np.abs(v))
        bound = torch.empty(N, dtype=torch.float64, device="cuda")
        Aabs.spmv(x.abs(), bound)
        torch.cuda.synchronize()
        empty = np.ones(N, bool)
        empty[np.asarray(a["row"])] = False
        assert empty[:first].all() and empty[last:].all() and empty.sum() > (N - (last - first))
        assert A.info().nnz > 128 * 20  # many 128-entry chunks
        cases.append((N, dev, x, y_ref.cpu().numpy(), bound.cpu().numpy(), empty))
    for N, dev, x, ref, b, empty in cases + cases:  # each matrix twice, alternating
        y = _noalloc(dm, torch, N, dev, x)
        assert np.all(y[empty] == 0.0) and not np.any(np.signbit(y[empty]))
        assert np.all(np.abs(y - ref) <= 1e-13 * b)


def test_limits_are_refused_before_any_work(env):
    dm, torch = env
    lib = dm.lib
    p = C.c_void_p(256)  # never dereferenced: the size check comes first
    st = lib.dynmat_spmv_coo_noalloc(1, dm.NOALLOC_MAX_NNZ + 1, p, p, p, p, p, None)
    assert st == dm.ERR_INVALID_ARG
    assert "over the" in dm.last_error()
    buf = torch.zeros(64, dtype=torch.int32, device="cuda")
    mis = C.c_void_p(buf.data_ptr() + 4)
    ok = C.c_void_p(buf.data_ptr())
    st = lib.dynmat_spmv_coo_noalloc(4, 8, mis, ok, ok, ok, ok, None)
    assert st == dm.ERR_INVALID_ARG and "16-byte" in dm.last_error()
