"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer and layout results (create, every conversion, the selector's
features and choice) must be bit-identical. FP64 SpMV must satisfy
|y_i - y_ref,i| <= 1e-13 * sum_j |a_ij x_j| per row, with rows whose bound is
0 exactly 0. FP32 results are compared with the FP64 oracle against a stated
bound. CG is compared with the oracle's iterates and with its defining
properties."""
import json
import math
import os

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
FMTS = ("coo", "csr", "dia", "ell", "hyb")
GOLD = os.path.join(os.path.dirname(__file__), "golden", "tiny_formats.json")


@pytest.fixture(scope="module")
def dm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2209_06478_b300 import build
    build.build()
    from paper_2209_06478_b300 import dynmat
    return dynmat


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    return torch


def _golden():
    g = json.load(open(GOLD))
    s = g["matrix"]["coo_shuffled"]
    return (g["matrix"]["nrows"], g["matrix"]["ncols"], np.array(s["row"], np.int32),
            np.array(s["col"], np.int32), np.array(s["val"], np.float64))


def _zeros_matrix():
    r, c, v = synth.random_coo(41, 90, 70, 0.12)
    v = v.copy()
    v[::7] = 0.0
    v[3::11] = -0.0
    return 90, 70, r, c, v


def _long_rows():
    # rows of 300..700 entries (cross several 128-entry chunks), some empty rows
    N, M = 40, 2000
    lens = synth.randint(5, N, 0, 700)
    lens[::5] = 0
    rows, cols = [], []
    for i, L in enumerate(lens.tolist()):
        cc = np.sort(np.unique(synth.randint(100 + i, 3 * L + 3, 0, M)))[:L]
        rows.append(np.full(cc.size, i))
        cols.append(cc)
    r = np.concatenate(rows).astype(np.int32)
    c = np.concatenate(cols).astype(np.int32)
    return N, M, r, c, synth.uniform_pm1(77, r.size)


def _dense_row():
    M = 3001
    return 3, M, np.ones(M, np.int32), np.arange(M, dtype=np.int32), synth.uniform_pm1(5, M)


def matrices():
    out = {}
    out["golden"] = _golden()
    N, r, c, v = synth.stencil27(8)[0], *synth.stencil27(8)[1:]
    out["stencil8"] = (N, N, r, c, v)
    N, r, c, v = synth.stencil27(16)[0], *synth.stencil27(16)[1:]
    out["stencil16"] = (N, N, r, c, v)
    N, r, c, v = synth.stencil7(11)[0], *synth.stencil7(11)[1:]
    out["stencil7_11"] = (N, N, r, c, v)
    out["rect_tall"] = (1000, 37, *synth.random_coo(6, 1000, 37, 0.1))
    out["rect_wide"] = (37, 1000, *synth.random_coo(7, 37, 1000, 0.1))
    out["random_4097"] = (4097, 4097, *synth.random_coo(8, 4097, 4097, 0.003))
    N, r, c, v = synth.powerlaw(9, 6000)
    out["powerlaw"] = (N, N, r, c, v)
    N, r, c, v = synth.banded(10, 5003, 21)
    out["banded"] = (N, N, r, c, v)
    out["zeros"] = _zeros_matrix()
    out["long_rows"] = _long_rows()
    out["dense_row"] = _dense_row()
    e = np.zeros(0, np.int32)
    out["empty"] = (17, 9, e, e.copy(), np.zeros(0))
    out["one"] = (1, 1, np.zeros(1, np.int32), np.zeros(1, np.int32), np.array([2.5]))
    return out


MATS = matrices()


def make(dm, name, shuffle=False):
    N, M, r, c, v = MATS[name]
    if shuffle and r.size:
        p = np.argsort(synth.uniform01(3, r.size), kind="stable")
        r, c, v = r[p], c[p], v[p]
    return dm.dynmat_create(N, M, np.ascontiguousarray(r), np.ascontiguousarray(c),
                            np.ascontiguousarray(v))


def canonical(orc, name):
    N, M, r, c, v = MATS[name]
    st, r, c, v = orc.canonical(N, M, r, c, v)
    assert st == orc.OK
    return N, M, r, c, v


def assert_arrays_equal(got, want, ctx):
    for k, w in want.items():
        g = got[k]
        assert g.shape == w.shape, (ctx, k, g.shape, w.shape)
        if w.dtype.kind == "f":
            assert np.array_equal(g.view(np.uint64 if g.itemsize == 8 else np.uint32),
                                  np.ascontiguousarray(w).view(np.uint64 if w.itemsize == 8 else np.uint32)), (ctx, k)
        else:
            assert np.array_equal(g, w), (ctx, k)


# ---------------------------------------------------------------------------
# Create and convert: bit-exact
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", sorted(MATS))
def test_create_canonical_bit_exact(dm, orc, name):
    N, M, r, c, v = canonical(orc, name)
    A = make(dm, name, shuffle=True)
    i = A.info()
    assert (i.format, i.nrows, i.ncols, i.nnz) == (dm.COO, N, M, r.size)
    assert_arrays_equal(A.arrays(), {"row": r, "col": c, "val": v}, name)


def test_create_shuffled_wide_keys_bit_exact(dm, orc):
    """Keys of 38 bits (row: 17 bits, column: 21 bits, for 70,000 x 1,048,579
    cells): five radix passes of 8-bit digits over 59 tiles of 4096 keys, the
    last one ragged; the upper digits are shared by long runs of keys, so the
    passes' stability decides the order. Compared with the oracle's canonical
    order (taken from the shuffled triplets as well)."""
    N, M = 70000, (1 << 20) + 3
    r, c, v = synth.random_coo(21, N, M, 4.1e-6)
    assert 4096 * 58 < r.size < 4096 * 59
    p = np.argsort(synth.uniform01(22, r.size), kind="stable")
    r, c, v = (np.ascontiguousarray(a[p]) for a in (r, c, v))
    st, wr, wc, wv = orc.canonical(N, M, r, c, v)
    assert st == orc.OK
    A = dm.dynmat_create(N, M, r, c, v)
    assert_arrays_equal(A.arrays(), {"row": wr, "col": wc, "val": wv}, "wide keys")


@pytest.mark.parametrize("name", ["stencil16", "random_4097", "powerlaw"])
def test_create_shuffled_f32_bit_exact(dm, orc, name):
    """FP32 values travel through the sort as a 32-bit payload (FP64 values
    as a 64-bit one): a shuffled FP32 create gives the oracle's canonical
    order with the values' bits unchanged."""
    N, M, r, c, v = MATS[name]
    p = np.argsort(synth.uniform01(4, r.size), kind="stable")
    r, c = np.ascontiguousarray(r[p]), np.ascontiguousarray(c[p])
    v32 = np.ascontiguousarray(v[p].astype(np.float32))
    st, wr, wc, wv = orc.canonical(N, M, r, c, v32.astype(np.float64))
    assert st == orc.OK
    A = dm.dynmat_create(N, M, r, c, v32)
    assert_arrays_equal(A.arrays(), {"row": wr, "col": wc, "val": wv.astype(np.float32)},
                        (name, "f32"))


def test_create_errors_match_oracle(dm, orc):
    cases = [
        (3, 3, [0, 3], [0, 0], [1.0, 2.0]),
        (3, 3, [0, 1], [0, -1], [1.0, 2.0]),
        (3, 3, [1, 0, 1], [2, 0, 2], [1.0, 2.0, 3.0]),
        (3, 3, [1, 1, 5], [2, 2, 0], [1.0, 2.0, 3.0]),
        (4, 4, [3, 2, 1, 0, 2], [0, 0, 0, 0, 0], [1.0] * 5),
    ]
    for N, M, r, c, v in cases:
        st = orc.canonical(N, M, r, c, v)[0]
        r, c, v = np.array(r, np.int32), np.array(c, np.int32), np.array(v)
        if st == orc.OK:
            dm.dynmat_create(N, M, r, c, v)
        else:
            with pytest.raises(dm.DynmatError) as e:
                dm.dynmat_create(N, M, r, c, v)
            assert e.value.status == st


@pytest.fixture
def no_pad_limit(dm):
    """Lifts the padding guard so that every pair can be compared (the
    irregular matrices here are small enough for any padding)."""
    dm.dynmat_set_pad_limit(1e9)
    yield
    dm.dynmat_set_pad_limit(16.0)


@pytest.mark.parametrize("name", sorted(MATS))
def test_every_conversion_pair_bit_exact(dm, orc, name, no_pad_limit):
    N, M, r, c, v = canonical(orc, name)
    for src in FMTS:
        A = make(dm, name)
        A.convert(src)
        want_src = orc.to_format(src, N, M, r, c, v)
        assert_arrays_equal(A.arrays(), want_src, (name, src))
        for dst in FMTS:
            B = make(dm, name)
            B.convert(src)
            B.convert(dst)
            want = orc.convert(src, dst, N, M, want_src)
            assert_arrays_equal(B.arrays(), want, (name, src, dst))


@pytest.mark.parametrize("name", ["stencil16", "powerlaw", "zeros", "golden", "rect_wide"])
def test_f32_conversions(dm, orc, name, no_pad_limit):
    N, M, r, c, v = canonical(orc, name)
    for fmt in FMTS:
        A = make(dm, name)
        A.convert(fmt, dm.F32)
        want = orc.to_format(fmt, N, M, r, c, v.astype(np.float32).astype(np.float64), vbytes=4)
        for k in want:
            if want[k].dtype == np.float64:
                want[k] = want[k].astype(np.float32)
        assert_arrays_equal(A.arrays(), want, (name, fmt))
        assert A.info().values_exact_in_f32 == 1
        # and back to F64 through COO: the FP32 values widened exactly, DIA's
        # stored zeros dropped by its COO view, HYB re-split with the FP64
        # byte model
        A.convert(fmt, dm.F64)
        want_w = {k: (w.astype(np.float64) if w.dtype == np.float32 else w) for k, w in want.items()}
        r2, c2, v2 = orc.to_coo(fmt, N, M, want_w)
        want64 = orc.to_format(fmt, N, M, r2, c2, v2, vbytes=8)
        assert_arrays_equal(A.arrays(), want64, (name, fmt, "f64"))


def test_format_too_large_leaves_matrix_valid(dm, orc):
    dm.dynmat_set_pad_limit(3.0)
    try:
        A = make(dm, "random_4097")
        A.convert("csr")
        with pytest.raises(dm.DynmatError) as e:
            A.convert("dia")
        assert e.value.status == dm.ERR_FORMAT_TOO_LARGE
        assert A.info().format == dm.CSR
        N, M, r, c, v = canonical(orc, "random_4097")
        assert_arrays_equal(A.arrays(), orc.to_format("csr", N, M, r, c, v), "after failure")
    finally:
        dm.dynmat_set_pad_limit(16.0)


def test_memory_limit_gives_oom_and_keeps_matrix(dm):
    A = make(dm, "stencil16")
    used = dm.dynmat_memory_in_use()
    dm.dynmat_set_memory_limit(used + 1024)
    try:
        with pytest.raises(dm.DynmatError) as e:
            A.convert("ell")
        assert e.value.status == dm.ERR_OOM
        assert A.info().format == dm.COO
    finally:
        dm.dynmat_set_memory_limit(0)
    A.convert("ell")


# ---------------------------------------------------------------------------
# Features and the rule: bit-exact
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", sorted(MATS))
def test_features_and_choice_match_oracle(dm, orc, name, no_pad_limit):
    N, M, r, c, v = canonical(orc, name)
    want = orc.features(N, M, r, c, vbytes=8, guard=3)
    for fmt in ("coo", "dia", "hyb"):
        A = make(dm, name)
        A.convert(fmt)
        got = A.features()
        if fmt == "dia" and np.any(v == 0):
            continue  # DIA dropped the stored zeros: a different COO view
        assert got == want, (name, fmt)
        assert A.select_format(dm.SELECT_FEATURES) == want["choice"]
    A = make(dm, name)
    A.convert("csr", dm.F32)
    assert A.features() == orc.features(N, M, r, c, vbytes=4, guard=3)


# ---------------------------------------------------------------------------
# SpMV
# ---------------------------------------------------------------------------

def spmv_ref(orc, name, x):
    N, M, r, c, v = canonical(orc, name)
    a = orc.to_format("csr", N, M, r, c, v)
    y = orc.spmv("csr", N, M, a, x)
    bound = orc.spmv("csr", N, M, {"rowptr": a["rowptr"], "col": c, "val": np.abs(v)}, np.abs(x))
    return y, bound


def run_spmv(dm, torch, A, x, vdt=np.float64):
    i = A.info()
    xt = torch.from_numpy(np.ascontiguousarray(x.astype(vdt))).cuda()
    yt = torch.full((i.nrows,), float("nan"), dtype=xt.dtype, device="cuda")
    A.spmv(xt, yt)
    torch.cuda.synchronize()
    return yt.cpu().numpy()


@pytest.mark.parametrize("name", sorted(MATS))
def test_spmv_f64_every_format(dm, orc, torch_mod, name, no_pad_limit):
    N, M = MATS[name][:2]
    x = synth.uniform_pm1(1, M)
    y_ref, bound = spmv_ref(orc, name, x)
    for fmt in FMTS:
        A = make(dm, name)
        A.convert(fmt)
        variants = {"csr": [1, 2, 3, 4, 5, 6, 7, 8], "dia": [1, 2, 3, 4, 5, 6, 7], "coo": [1, 2],
                    "ell": [1, 2], "hyb": [1, 2]}[fmt]
        for var in variants:
            if var:
                A.set_variant(var)
            y = run_spmv(dm, torch_mod, A, x)
            assert np.all(np.abs(y - y_ref) <= 1e-13 * bound), (name, fmt, var)
            assert np.all(y[bound == 0] == 0.0), (name, fmt, var)


@pytest.mark.parametrize("name", ["stencil16", "stencil8", "banded", "stencil7_11", "random_4097"])
def test_dia_runs_variant_same_bits_as_variant_1(dm, orc, torch_mod, name, no_pad_limit):
    """Variant 6 groups the diagonals in runs but adds them in the same order
    with the same multiply-adds: the products are bit-identical to variant 1
    (matrices with too many runs fall back to variant 1)."""
    N, M = MATS[name][:2]
    x = synth.uniform_pm1(5, M)
    A = make(dm, name)
    A.convert("dia")
    A.set_variant(1)
    y1 = run_spmv(dm, torch_mod, A, x)
    A.set_variant(6)
    y6 = run_spmv(dm, torch_mod, A, x)
    assert np.array_equal(y1.view(np.int64), y6.view(np.int64))


@pytest.mark.parametrize("n", [3, 4, 9, 16])
def test_stencil_ones_exact_every_format_and_precision(dm, orc, torch_mod, n):
    N, r, c, v = synth.stencil27(n)
    expect = {19.0: 8, 15.0: 12 * (n - 2), 9.0: 6 * (n - 2) ** 2, 0.0: (n - 2) ** 3}
    expect = {k: m for k, m in expect.items() if m}
    for fmt in FMTS:
        for vdt, xdt in ((dm.F64, np.float64), (dm.F32, np.float32), (dm.F32, np.float64)):
            A = dm.dynmat_create(N, N, r, c, v)
            A.convert(fmt, vdt)
            y = run_spmv(dm, torch_mod, A, np.ones(N), xdt)
            vals, counts = np.unique(y, return_counts=True)
            assert dict(zip(vals.tolist(), counts.tolist())) == expect, (fmt, vdt, xdt)


@pytest.mark.parametrize("name", ["stencil16", "powerlaw", "banded", "long_rows", "random_4097"])
def test_spmv_f32_error_stated(dm, orc, torch_mod, name, no_pad_limit):
    """FP32 values and vectors with FP32 sums: error vs the FP64 oracle is
    bounded by (len_i + 2) * 2^-24 * sum_j |a_ij x_j| (one rounding each for
    a and x, and one for each of the row's len_i multiply-adds)."""
    N, M, r, c, v = canonical(orc, name)
    x = synth.uniform_pm1(2, M)
    y_ref, bound = spmv_ref(orc, name, x)
    lens = np.bincount(r, minlength=N)
    worst = 0.0
    for fmt in FMTS:
        A = make(dm, name)
        A.convert(fmt, dm.F32)
        y = run_spmv(dm, torch_mod, A, x, np.float32).astype(np.float64)
        err = np.abs(y - y_ref)
        assert np.all(err <= (lens + 2) * 2.0 ** -24 * bound + 1e-30), (name, fmt)
        nz = bound > 0
        if nz.any():
            worst = max(worst, float((err[nz] / bound[nz]).max()))
        # FP32 values with FP64 vectors: FP64 sums of the rounded values
        y64 = run_spmv(dm, torch_mod, A, x, np.float64)
        a32 = orc.to_format("csr", N, M, r, c, v.astype(np.float32).astype(np.float64))
        y32ref = orc.spmv("csr", N, M, a32, x)
        assert np.all(np.abs(y64 - y32ref) <= 1e-13 * bound + 1e-300), (name, fmt)
    print("%s: max FP32 relative error %.3e" % (name, worst))


def test_spmv_is_deterministic(dm, torch_mod, no_pad_limit):
    for name in ("powerlaw", "long_rows", "stencil16"):
        for fmt in FMTS:
            A = make(dm, name)
            A.convert(fmt)
            x = synth.uniform_pm1(3, MATS[name][1])
            y1 = run_spmv(dm, torch_mod, A, x)
            y2 = run_spmv(dm, torch_mod, A, x)
            assert np.array_equal(y1.view(np.uint64), y2.view(np.uint64)), (name, fmt)


@pytest.mark.parametrize("fmt,vdt", [("dia", "f64"), ("ell", "f64"), ("dia", "f32"), ("csr", "f64"),
                                     ("coo", "f64"), ("hyb", "f64")])
def test_spmv_host_pipelined_matches_device_product(dm, orc, torch_mod, fmt, vdt):
    """Host buffers on a matrix large enough for the pipelined path (x up in
    pieces, the product in row chunks, y down per chunk; DIA, ELL, CSR's
    stream kernel, COO's stream kernel) give the same bits as the device
    product, and HYB, whose stencil has no COO overflow, runs as its ELL part."""
    N, r, c, v = synth.stencil27(96)
    A = dm.dynmat_create(N, N, r, c, v)
    A.convert(fmt, dm.F64 if vdt == "f64" else dm.F32)
    xh = synth.uniform_pm1(9, N)  # FP64 vectors (with FP32 values for "f32")
    x = torch_mod.from_numpy(xh).pin_memory()
    y = torch_mod.empty_like(x).pin_memory()
    A.spmv_host(x.numpy(), y.numpy())
    y_dev = run_spmv(dm, torch_mod, A, xh, xh.dtype.type)
    assert np.array_equal(y.numpy().view(np.uint8), y_dev.view(np.uint8))
    # twice in a row: the pipeline's streams and events are reused
    y2 = torch_mod.zeros_like(y).pin_memory()
    A.spmv_host(x.numpy(), y2.numpy())
    assert np.array_equal(y2.numpy().view(np.uint8), y_dev.view(np.uint8))


def _device_product(torch_mod, A, xh):
    """y = A x on the device (y sized by A's rows, x by its columns)."""
    i = A.info()
    assert xh.shape == (i.ncols,)
    x = torch_mod.from_numpy(xh).cuda()
    y = torch_mod.empty(i.nrows, dtype=x.dtype, device=x.device)
    A.spmv(x, y)
    torch_mod.cuda.synchronize()
    return y.cpu().numpy()


def test_host_alloc_contract(dm):
    """dynmat_host_alloc: 2 MiB-aligned, zeroed, usable as the source of a
    device copy; a second free of the same block and a pointer inside a
    block are refused without touching the mapping."""
    import ctypes as C
    import torch
    p = C.c_void_p()
    nbytes = (3 << 20) + 5
    assert dm.lib.dynmat_host_alloc(nbytes, C.byref(p)) == dm.OK
    assert p.value % (2 << 20) == 0
    view = np.ctypeslib.as_array((C.c_uint8 * nbytes).from_address(p.value))
    assert not view.any()
    view[:] = 7
    d = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    d.copy_(torch.from_numpy(view), non_blocking=True)
    torch.cuda.synchronize()
    assert int(d.sum().item()) == 7 * nbytes
    assert dm.lib.dynmat_host_free(C.c_void_p(p.value + 64)) == dm.ERR_INVALID_ARG
    assert dm.lib.dynmat_host_free(p) == dm.OK
    assert dm.lib.dynmat_host_free(p) == dm.ERR_INVALID_ARG


def test_spmv_host_follows_changes(dm, torch_mod):
    """Host buffers from dynmat_host_alloc through the pipelined product: new
    contents of the same buffers, a variant change, format switches (the ELL
    chunks' column reach is measured again) and a new buffer all give the
    device product's bits."""
    N, r, c, v = synth.stencil27(96)
    A = dm.dynmat_create(N, N, r, c, v)
    A.convert("dia")
    xh = dm.dynmat_host_alloc(N)
    yh = dm.dynmat_host_alloc(N)
    assert xh.ctypes.data % (2 << 20) == 0 and not yh.any()
    for seed, change in ((1, None), (2, None), (3, "variant"), (4, "ell"), (5, "f32"),
                         (6, "dia"), (7, "new y")):
        if change == "variant":
            A.set_variant(1)
        elif change == "ell":
            A.convert("ell")
        elif change == "f32":
            A.convert("ell", dm.F32)
        elif change == "dia":
            A.convert("dia")
        elif change == "new y":
            yh = dm.dynmat_host_alloc(N)
        xh[:] = synth.uniform_pm1(seed, N)
        A.spmv_host(xh, yh)
        assert np.array_equal(yh.view(np.uint64), _device_product(torch_mod, A, xh).view(np.uint64)), change
    # FP32 vectors through the same buffers' memory
    A.convert("dia", dm.F32)
    x32 = dm.dynmat_host_alloc(N, np.float32)
    y32 = dm.dynmat_host_alloc(N, np.float32)
    x32[:] = synth.uniform_pm1(8, N).astype(np.float32)
    A.spmv_host(x32, y32)
    assert np.array_equal(y32.view(np.uint32), _device_product(torch_mod, A, x32).view(np.uint32))


def test_spmv_host_every_csr_coo_ell_and_dia_variant(dm, torch_mod):
    """CSR, COO, ELL and DIA kernel variants through the host-buffer product:
    the tile-based ones (CSR 1-5 and 7, COO 2, ELL 1 and 2, DIA) run
    pipelined in row chunks, the others whole; all give the device product's
    bits."""
    N, r, c, v = synth.stencil27(96)
    xh = dm.dynmat_host_alloc(N)
    yh = dm.dynmat_host_alloc(N)
    xh[:] = synth.uniform_pm1(13, N)
    for fmt, variants in (("csr", range(1, 9)), ("coo", (1, 2)), ("ell", (1, 2)),
                          ("dia", (1, 3, 6, 7))):
        A = dm.dynmat_create(N, N, r, c, v)
        A.convert(fmt)
        for var in variants:
            A.set_variant(var)
            yh[:] = np.nan
            A.spmv_host(xh, yh)
            want = _device_product(torch_mod, A, xh)
            assert np.array_equal(yh.view(np.uint64), want.view(np.uint64)), (fmt, var)


def test_spmv_host_dia_runs_on_small_tiles(dm, torch_mod):
    """Above about 909k rows the automatic DIA variant (6) takes 512-row tiles
    dealt out over every resident block, and a row chunk of the host-buffer
    product keeps two tiles per block. At 100^3 and 128^3 the pipelined
    product gives the device product's bits; the stencil's largest offset,
    n^2 + n + 1, makes a chunk read x past its own rows."""
    for n in (100, 128):
        N, r, c, v = synth.stencil27(n)
        A = dm.dynmat_create(N, N, r, c, v)
        A.convert("dia")
        assert A.info().spmv_variant == 6
        xh = dm.dynmat_host_alloc(N)
        yh = dm.dynmat_host_alloc(N)
        xh[:] = synth.uniform_pm1(21, N)
        yh[:] = np.nan
        A.spmv_host(xh, yh)
        want = _device_product(torch_mod, A, xh)
        assert np.array_equal(yh.view(np.uint64), want.view(np.uint64)), n


def test_spmv_host_ell_chunks_wait_for_their_columns(dm, torch_mod):
    """Rows whose columns reach far ahead (and far behind) of their own row,
    in ELL, CSR and COO: each row chunk of the pipeline waits for the x piece
    of the largest column stored in it, so the result is exact whether x
    comes up before or after the chunk's own rows."""
    N = 1 << 20
    rng = np.random.default_rng(11)
    i = np.arange(N, dtype=np.int64)
    far = rng.integers(0, N, N)
    ahead = np.where(i % 4096 == 0, N - 1 - (i // 4096), i)  # a few rows read the very end
    r = np.concatenate([i, i, i])
    c = np.concatenate([i, np.where(i < N // 2, far % (i + 1), far), ahead])
    key = np.unique(r * N + c)
    r, c = (key // N).astype(np.int32), (key % N).astype(np.int32)
    v = rng.uniform(-1, 1, r.size)
    for fmt in ("ell", "csr", "coo", "hyb"):  # ELL slots; CSR and COO entry ranges; HYB (overflow: whole)
        A = dm.dynmat_create(N, N, r, c, v)
        A.convert(fmt)
        for buffers in ("registered", "pageable"):
            xh = dm.dynmat_host_alloc(N) if buffers == "registered" else np.empty(N)
            yh = dm.dynmat_host_alloc(N) if buffers == "registered" else np.empty(N)
            xh[:] = synth.uniform_pm1(12, N)
            A.spmv_host(xh, yh)
            want = _device_product(torch_mod, A, xh)
            assert np.array_equal(yh.view(np.uint64), want.view(np.uint64)), (fmt, buffers)


@pytest.mark.parametrize("shape", [(1_500_000, 700_000), (600_000, 1_400_000)])
def test_spmv_host_rectangular(dm, torch_mod, shape):
    """Tall and wide matrices through the pipelined host product: x pieces
    cover the columns and row chunks the rows, so the two differ in length;
    every tile-based format gives the device product's bits."""
    N, M = shape
    rng = np.random.default_rng(21)
    i = np.repeat(np.arange(N, dtype=np.int64), 4)
    band = (i * M) // N  # each row's entries near its scaled diagonal
    c = np.clip(band + rng.integers(-3000, 3000, i.size), 0, M - 1)
    key = np.unique(i * M + c)
    r, c = (key // M).astype(np.int32), (key % M).astype(np.int32)
    v = rng.uniform(-1, 1, r.size)
    xh = dm.dynmat_host_alloc(M)
    yh = dm.dynmat_host_alloc(N)
    xh[:] = synth.uniform_pm1(22, M)
    for fmt in ("ell", "csr", "coo"):
        A = dm.dynmat_create(N, M, r, c, v)
        A.convert(fmt)
        yh[:] = np.nan
        A.spmv_host(xh, yh)
        want = _device_product(torch_mod, A, xh)
        assert np.array_equal(yh.view(np.uint64), want.view(np.uint64)), (fmt, shape)


def test_spmv_host_f32_vectors_pipelined(dm, torch_mod):
    """FP32 values and FP32 vectors at 128^3 (16.8 MB of x and y, above the
    pipeline's threshold): the pipelined product has the device product's
    bits in DIA, ELL and CSR."""
    A = dm.dynmat_create_stencil(128, 27, "dia", dm.F32)
    N = 128 ** 3
    xh = dm.dynmat_host_alloc(N, np.float32)
    yh = dm.dynmat_host_alloc(N, np.float32)
    xh[:] = synth.uniform_pm1(23, N).astype(np.float32)
    for fmt in ("dia", "ell", "csr"):
        A.convert(fmt, dm.F32)
        yh[:] = np.nan
        A.spmv_host(xh, yh)
        want = _device_product(torch_mod, A, xh)
        assert np.array_equal(yh.view(np.uint32), want.view(np.uint32)), fmt


def test_spmv_host_buffers(dm, orc):
    name = "stencil16"
    A = make(dm, name)
    A.convert("dia")
    x = synth.uniform_pm1(4, MATS[name][1])
    y = np.empty(MATS[name][0])
    A.spmv_host(x, y)
    y_ref, bound = spmv_ref(orc, name, x)
    assert np.all(np.abs(y - y_ref) <= 1e-13 * bound)


def test_profile_selection_and_autotune(dm, orc, torch_mod):
    for name in ("stencil16", "powerlaw", "banded"):
        A = make(dm, name)
        f = A.select_format(dm.SELECT_PROFILE)
        assert 0 <= f <= 4
        assert A.info().format == dm.COO  # select does not convert
        fmt, var = A.autotune()
        assert A.info().format == fmt
        x = synth.uniform_pm1(6, MATS[name][1])
        y_ref, bound = spmv_ref(orc, name, x)
        y = run_spmv(dm, torch_mod, A, x)
        assert np.all(np.abs(y - y_ref) <= 1e-13 * bound), (name, fmt, var)


# ---------------------------------------------------------------------------
# CG
# ---------------------------------------------------------------------------

def cg_gpu(dm, torch, A, b, **kw):
    bt = torch.from_numpy(b).cuda()
    xt = torch.zeros_like(bt)
    res = A.cg_solve(bt, xt, **kw)
    return res, xt.cpu().numpy()


def test_cg_16cubed_50_iterations_matches_oracle(dm, orc, torch_mod):
    N, r, c, v = synth.stencil27(16)
    rp = orc.coo_to_csr(N, r)
    b = orc.spmv("csr", N, N, {"rowptr": rp, "col": c, "val": v}, np.ones(N))
    ref = orc.cg(N, rp, c, v, b, tol=0.0, max_iters=50)
    for fmt in FMTS:
        A = dm.dynmat_create(N, N, r, c, v)
        A.convert(fmt)
        res, x = cg_gpu(dm, torch_mod, A, b, tol=0.0, max_iters=50, check_every=7)
        assert res["status"] == dm.ERR_NOT_CONVERGED and res["iterations"] == 50, fmt
        assert np.linalg.norm(x - ref["x"]) / np.linalg.norm(ref["x"]) <= 1e-10, fmt
        assert abs(res["rel_residual"] - ref["rel_residual"]) <= 1e-8 * ref["rel_residual"] + 1e-14


@pytest.mark.parametrize("fmt", FMTS)
def test_cg_to_tolerance_recovers_ones(dm, orc, torch_mod, fmt):
    n = 24
    N, r, c, v = synth.stencil27(n)
    rp = orc.coo_to_csr(N, r)
    b = orc.spmv("csr", N, N, {"rowptr": rp, "col": c, "val": v}, np.ones(N))
    ref = orc.cg(N, rp, c, v, b, tol=1e-9, max_iters=1000)
    A = dm.dynmat_create(N, N, r, c, v)
    A.convert(fmt)
    res, x = cg_gpu(dm, torch_mod, A, b, tol=1e-9, max_iters=1000)
    assert res["status"] == dm.OK
    assert abs(res["iterations"] - ref["iterations"]) <= 2
    true = np.linalg.norm(b - orc.spmv("csr", N, N, {"rowptr": rp, "col": c, "val": v}, x)) / np.linalg.norm(b)
    assert true <= 2e-9 and abs(true - res["true_rel_residual"]) <= 1e-12
    t1 = 1 + 2 * math.cos(math.pi / (n + 1))
    tn = 1 + 2 * math.cos(n * math.pi / (n + 1))
    kappa = (27 - t1 * t1 * tn) / (27 - t1 ** 3)
    assert np.linalg.norm(x - 1) / math.sqrt(N) <= kappa * 1e-9


def test_cg_edge_cases(dm, torch_mod):
    i = np.arange(10, dtype=np.int32)
    A = dm.dynmat_create(10, 10, i, i, -np.ones(10))
    res, _ = cg_gpu(dm, torch_mod, A, np.ones(10), tol=1e-9, max_iters=5)
    assert res["status"] == dm.ERR_BREAKDOWN and res["iterations"] == 0
    A = dm.dynmat_create(10, 10, i, i, np.ones(10))
    res, x = cg_gpu(dm, torch_mod, A, np.zeros(10), tol=1e-9, max_iters=5)
    assert res["status"] == dm.OK and res["iterations"] == 0 and np.all(x == 0)
    d = np.array([2.0, 5.0, 11.0] * 20)
    i = np.arange(60, dtype=np.int32)
    A = dm.dynmat_create(60, 60, i, i, d)
    b = synth.uniform_pm1(12, 60)
    res, x = cg_gpu(dm, torch_mod, A, b, tol=1e-13, max_iters=10)
    assert res["status"] == dm.OK and res["iterations"] == 3
    assert np.allclose(x, b / d, rtol=1e-12, atol=0)


def test_cg_is_deterministic(dm, torch_mod):
    N, r, c, v = synth.stencil27(20)
    b = synth.uniform_pm1(9, N)
    for fmt in ("dia", "csr", "coo", "ell"):  # 20^3 ELL: the split-slot form (variant 2)
        A = dm.dynmat_create(N, N, r, c, v)
        A.convert(fmt)
        _, x1 = cg_gpu(dm, torch_mod, A, b, tol=1e-10, max_iters=500)
        _, x2 = cg_gpu(dm, torch_mod, A, b, tol=1e-10, max_iters=500)
        assert np.array_equal(x1.view(np.uint64), x2.view(np.uint64)), fmt


@pytest.mark.parametrize("fmt,vdt", [("dia", 1), ("csr", 0), ("ell", 1), ("coo", 0), ("hyb", 1)])
def test_mixed_precision_reaches_1e10(dm, orc, torch_mod, fmt, vdt):
    n = 20
    N, r, c, v = synth.stencil27(n)
    rp = orc.coo_to_csr(N, r)
    b = orc.spmv("csr", N, N, {"rowptr": rp, "col": c, "val": v}, np.ones(N))
    A = dm.dynmat_create(N, N, r, c, v)
    A.convert(fmt, vdt)
    res, x = cg_gpu(dm, torch_mod, A, b, tol=1e-10, max_iters=1000, precision=dm.CG_MIXED,
                    inner_tol=1e-5)
    assert res["status"] == dm.OK and res["outer_iterations"] >= 2
    true = np.linalg.norm(b - orc.spmv("csr", N, N, {"rowptr": rp, "col": c, "val": v}, x)) / np.linalg.norm(b)
    assert true <= 1e-10
    ref = orc.ir_mixed(N, rp, c, v, b, tol=1e-10, inner_tol=1e-5)
    assert abs(res["outer_iterations"] - ref["outer"]) <= 1
    assert np.linalg.norm(x - ref["x"]) / np.linalg.norm(ref["x"]) <= 1e-8


@pytest.mark.parametrize("fmt,vdt", [("dia", 1), ("csr", 0), ("ell", 1), ("coo", 0), ("hyb", 0)])
def test_reliable_mixed_matches_oracle(dm, orc, torch_mod, fmt, vdt):
    n = 20
    N, r, c, v = synth.stencil27(n)
    rp = orc.coo_to_csr(N, r)
    b = synth.uniform_pm1(33, N)
    A = dm.dynmat_create(N, N, r, c, v)
    A.convert(fmt, vdt)
    res, x = cg_gpu(dm, torch_mod, A, b, tol=1e-10, max_iters=2000,
                    precision=dm.CG_MIXED_RELIABLE, delta=0.1)
    ref = orc.cg_reliable(N, rp, c, v, b, tol=1e-10, delta=0.1)
    assert res["status"] == dm.OK and ref["status"] == orc.OK
    assert abs(res["iterations"] - ref["iterations"]) <= 3
    assert abs(res["outer_iterations"] - ref["folds"]) <= 2
    true = np.linalg.norm(b - orc.spmv("csr", N, N, {"rowptr": rp, "col": c, "val": v}, x)) / np.linalg.norm(b)
    assert true <= 1e-10 and abs(true - res["true_rel_residual"]) <= 1e-13
    assert np.linalg.norm(x - ref["x"]) / np.linalg.norm(ref["x"]) <= 1e-8
    fp64 = orc.cg(N, rp, c, v, b, tol=1e-10, max_iters=2000)
    assert res["iterations"] <= 1.15 * fp64["iterations"] + 5


def test_reliable_mixed_edge_cases(dm, torch_mod):
    i = np.arange(10, dtype=np.int32)
    A = dm.dynmat_create(10, 10, i, i, -np.ones(10))
    res, _ = cg_gpu(dm, torch_mod, A, np.ones(10), tol=1e-9, max_iters=5,
                    precision=dm.CG_MIXED_RELIABLE)
    assert res["status"] == dm.ERR_BREAKDOWN and res["iterations"] == 0
    A = dm.dynmat_create(10, 10, i, i, np.ones(10))
    res, x = cg_gpu(dm, torch_mod, A, np.zeros(10), tol=1e-9, max_iters=5,
                    precision=dm.CG_MIXED_RELIABLE)
    assert res["status"] == dm.OK and res["iterations"] == 0 and np.all(x == 0)
    N, r, c, v = synth.stencil27(8)
    A = dm.dynmat_create(N, N, r, c, v)
    res, _ = cg_gpu(dm, torch_mod, A, synth.uniform_pm1(2, N), tol=1e-30, max_iters=7,
                    precision=dm.CG_MIXED_RELIABLE)
    assert res["status"] == dm.ERR_NOT_CONVERGED and res["iterations"] == 7


def test_mixed_precision_general_matrix_uses_fp64_residual(dm, orc, torch_mod):
    N, r, c, v = synth.banded(21, 3000, 15, spd=True)
    st, r, c, v = orc.canonical(N, N, r, c, v)
    A = dm.dynmat_create(N, N, r, c, v)
    A.convert("dia")
    assert A.info().values_exact_in_f32 == 0
    rp = orc.coo_to_csr(N, r)
    b = synth.uniform_pm1(22, N)
    res, x = cg_gpu(dm, torch_mod, A, b, tol=1e-10, max_iters=500, precision=dm.CG_MIXED)
    assert res["status"] == dm.OK
    true = np.linalg.norm(b - orc.spmv("csr", N, N, {"rowptr": rp, "col": c, "val": v}, x)) / np.linalg.norm(b)
    assert true <= 1e-10


# ---------------------------------------------------------------------------
# Full-size workload (27-point stencil, 128^3) in the benchmark's configuration
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def big(orc):
    n = 128
    N, r, c, v = synth.stencil27(n)
    return n, N, r, c, v


def test_full_size_spmv_every_format(dm, orc, torch_mod, big):
    n, N, r, c, v = big
    x = synth.uniform_pm1(2, N)
    rp = orc.coo_to_csr(N, r)
    y_ref = orc.spmv("csr", N, N, {"rowptr": rp, "col": c, "val": v}, x)
    bound = orc.spmv("csr", N, N, {"rowptr": rp, "col": c, "val": np.abs(v)}, np.abs(x))
    A = dm.dynmat_create(N, N, r, c, v)
    feats = A.features()
    assert feats == orc.features(N, N, r, c)
    assert feats["choice"] == dm.DIA and feats["ndiag"] == 27
    for fmt in FMTS:
        A.convert(fmt)
        y = run_spmv(dm, torch_mod, A, x)
        assert np.all(np.abs(y - y_ref) <= 1e-13 * bound), fmt
    # DIA arrays bit-exact at full size
    A.convert("dia")
    want = orc.to_format("dia", N, N, r, c, v)
    got = A.arrays()
    assert np.array_equal(got["offsets"], want["offsets"])
    assert np.array_equal(got["val"], want["val"])


def test_full_size_every_kernel_variant(dm, orc, torch_mod, big):
    """Every kernel variant of CSR (1-8), DIA (1-7), COO (1-2) and ELL (1-2) at 128^3
    against the oracle's product; DIA's variants agree bit for bit (one DFMA
    per slot in offset order)."""
    n, N, r, c, v = big
    x = synth.uniform_pm1(2, N)
    rp = orc.coo_to_csr(N, r)
    y_ref = orc.spmv("csr", N, N, {"rowptr": rp, "col": c, "val": v}, x)
    bound = orc.spmv("csr", N, N, {"rowptr": rp, "col": c, "val": np.abs(v)}, np.abs(x))
    A = dm.dynmat_create(N, N, r, c, v)
    for fmt, variants in (("csr", range(1, 9)), ("dia", range(1, 8)), ("coo", (1, 2)),
                          ("ell", (1, 2))):
        A.convert(fmt)
        ys = {}
        for var in variants:
            A.set_variant(var)
            ys[var] = run_spmv(dm, torch_mod, A, x)
            assert np.all(np.abs(ys[var] - y_ref) <= 1e-13 * bound), (fmt, var)
        if fmt == "dia":
            for var in (2, 3, 6):  # one chain per row: the same sums as variant 1
                assert np.array_equal(ys[var].view(np.int64), ys[1].view(np.int64)), var


def test_full_size_cg_to_1e9(dm, orc, torch_mod, big):
    n, N, r, c, v = big
    rp = orc.coo_to_csr(N, r)
    b = orc.spmv("csr", N, N, {"rowptr": rp, "col": c, "val": v}, np.ones(N))
    A = dm.dynmat_create(N, N, r, c, v)
    A.convert("dia")
    res, x = cg_gpu(dm, torch_mod, A, b, tol=1e-9, max_iters=3000)
    assert res["status"] == dm.OK
    true = np.linalg.norm(b - orc.spmv("csr", N, N, {"rowptr": rp, "col": c, "val": v}, x)) / np.linalg.norm(b)
    assert true <= 2e-9
    t1 = 1 + 2 * math.cos(math.pi / (n + 1))
    tn = 1 + 2 * math.cos(n * math.pi / (n + 1))
    kappa = (27 - t1 * t1 * tn) / (27 - t1 ** 3)
    assert np.linalg.norm(x - 1) / math.sqrt(N) <= kappa * 1e-9
