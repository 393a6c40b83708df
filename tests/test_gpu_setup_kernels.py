"""Edge cases of the setup kernels behind create, convert and the SpMV plan
(§III-B), through the C ABI:
- the COO check reads four entries per thread and takes each group's
  successor from the next lane (or a plain load at the end of a warp), so
  duplicates, inversions and out-of-range indices are planted at every
  kind of boundary and the status must be the oracle's;
- the COO plan's longest row decides the automatic kernel (stream kernel
  when the longest row is at most 2 x mean + 32), so rows one entry either
  side of that threshold, placed at the start, across 128-entry tiles and at
  the end, must pick the variant the exact length implies;
- the FP32-exactness flag is decided on the bits; it must equal numpy's
  float32 round trip on normal, subnormal, overflowing and special values."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2209_06478_b300 import build
    build.build()
    from paper_2209_06478_b300 import dynmat
    return dynmat


def _create_status(dm, N, M, r, c, v):
    try:
        A = dm.dynmat_create(N, M, r, c, v)
    except dm.DynmatError as e:
        return e.status, None
    return dm.OK, A


BOUNDARIES = (1, 2, 3, 4, 5, 126, 127, 128, 129, 255, 256, 511)


def _sorted_coo(n):
    N, r, c, v = synth.stencil27(n)
    return N, r.copy(), c.copy(), v.copy()


@pytest.mark.parametrize("p", BOUNDARIES + (-2,))
def test_check_finds_duplicates_at_group_and_warp_boundaries(dm, orc, p):
    N, r, c, v = _sorted_coo(8)  # 5832 entries
    p = p % r.size
    r[p + 1], c[p + 1] = r[p], c[p]  # entry p + 1 repeats entry p
    want = orc.canonical(N, N, r, c, v)[0]
    assert want == orc.DUPLICATE
    assert _create_status(dm, N, N, r, c, v)[0] == want


@pytest.mark.parametrize("p", BOUNDARIES + (-2,))
def test_check_finds_inversions_at_group_and_warp_boundaries(dm, orc, p):
    """Entries p and p + 1 swapped: not sorted, so the library sorts, and the
    result must be the canonical arrays bit for bit."""
    N, r, c, v = _sorted_coo(8)
    p = p % r.size
    for a in (r, c, v):
        a[p], a[p + 1] = a[p + 1], a[p]
    st, A = _create_status(dm, N, N, r, c, v)
    ref = orc.canonical(N, N, r, c, v)
    assert st == ref[0] == orc.OK
    got = A.arrays()
    assert np.array_equal(got["row"], ref[1]) and np.array_equal(got["col"], ref[2])
    assert np.array_equal(got["val"].view(np.int64), ref[3].view(np.int64))


@pytest.mark.parametrize("p", BOUNDARIES + (-1,))
@pytest.mark.parametrize("what", ["row", "col", "negative"])
def test_check_finds_out_of_range_indices_anywhere(dm, orc, p, what):
    N, r, c, v = _sorted_coo(8)
    p = p % r.size
    if what == "row":
        r[p] = N
    elif what == "col":
        c[p] = N + 7
    else:
        c[p] = -1
    want = orc.canonical(N, N, r, c, v)[0]
    assert want == orc.INDEX_RANGE
    assert _create_status(dm, N, N, r, c, v)[0] == want


def _rows_with_one_long(N, base_len, k, L, ncols):
    """Rows of base_len entries except row k with L, columns 0, 1, ..."""
    lens = np.full(N, base_len, np.int64)
    lens[k] = L
    r = np.repeat(np.arange(N, dtype=np.int32), lens)
    c = np.concatenate([np.arange(n, dtype=np.int32) for n in lens])
    v = synth.uniform_pm1(k + 3, r.size) + 2.0
    return r, c, v, ncols


@pytest.mark.parametrize("k", [0, 31, 500, 999])
def test_longest_row_decides_the_coo_kernel_to_the_entry(dm, k):
    """999 rows of 4 and one of 40 (mean 4.036: 40 <= 40.072, stream kernel)
    or 41 (mean 4.037: 41 > 40.074, segmented kernel); row 31 crosses the
    first 128-entry tile boundary, row 999 runs to the last entry."""
    N = 1000
    for L, want in ((40, 2), (41, 1)):
        r, c, v, M = _rows_with_one_long(N, 4, k, L, 64)
        A = dm.dynmat_create(N, M, r, c, v)
        assert A.info().spmv_variant == want, (k, L)


@pytest.mark.parametrize("k", [0, 7, 999])
def test_longest_row_across_several_tiles(dm, k):
    """999 rows of 200 and one of 432 (fits 2 x 200.232 + 32 = 432.46) or
    433 (does not): the long row spans four 128-entry tiles."""
    N = 1000
    for L, want in ((432, 2), (433, 1)):
        r, c, v, M = _rows_with_one_long(N, 200, k, L, 1000)
        A = dm.dynmat_create(N, M, r, c, v)
        assert A.info().spmv_variant == want, (k, L)


SPECIAL = [
    0.0, -0.0, 1.0, -2.5, 3.0 + 2.0 ** -20, 0.1, 1.0 + 2.0 ** -23, 1.0 + 2.0 ** -24,
    float(np.finfo(np.float32).max), float(np.finfo(np.float32).max) * (1 + 2.0 ** -40),
    2.0 ** 127, 2.0 ** 128, -(2.0 ** 128), float("inf"), float("-inf"),
    2.0 ** -126, 2.0 ** -127, 2.0 ** -149, 3 * 2.0 ** -149, 2.0 ** -150, 2.0 ** -149 * 1.5,
    2.0 ** -130 + 2.0 ** -149, 2.0 ** -130 + 2.0 ** -150, 5e-324, 2.2250738585072014e-308,
    1e-40, 1e-45, 1e300, -1e-300,
]


@pytest.mark.parametrize("value", SPECIAL)
def test_fp32_exactness_flag_matches_float32_round_trip(dm, value):
    v = np.array([1.0, value, -4.0])
    r = np.array([0, 1, 2], np.int32)
    A = dm.dynmat_create(3, 3, r, r.copy(), v)
    with np.errstate(over="ignore"):
        exact = bool(np.float64(np.float32(value)) == value) or np.isnan(value)
    assert A.info().values_exact_in_f32 == int(exact), value


def test_fp32_exactness_flag_on_a_large_array(dm):
    """One inexact value anywhere in 3M exact ones clears the flag."""
    n = 3_000_001
    r = np.arange(n, dtype=np.int32)
    v = (synth.uniform_pm1(9, n).astype(np.float32)).astype(np.float64)
    A = dm.dynmat_create(n, n, r, r.copy(), v)
    assert A.info().values_exact_in_f32 == 1
    v[n - 2] += 2.0 ** -40
    A = dm.dynmat_create(n, n, r, r.copy(), v)
    assert A.info().values_exact_in_f32 == 0
