"""Pins the CPU oracle to facts that do not come from the oracle itself.

Each test compares the oracle against a hand-derived fixture, brute force,
exact rational arithmetic, a closed form of the 27-point stencil (§II-B), or
an invariant of the format definitions (§II-A) and of CG. A dropped term, a
wrong sign or index, or a transposed operand in the oracle fails at least
one of them.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden", "tiny_formats.json")
FMTS = ("coo", "csr", "dia", "ell", "hyb")


def dense_of(nrows, ncols, row, col, val):
    A = np.zeros((nrows, ncols))
    A[np.asarray(row), np.asarray(col)] = val
    return A


def kron_stencil(n):
    """27 I - T (x) T (x) T with T = tridiag(1, 1, 1): an independent dense
    construction of the 27-point operator."""
    T = np.eye(n) + np.eye(n, k=1) + np.eye(n, k=-1)
    return 27.0 * np.eye(n ** 3) - np.kron(T, np.kron(T, T))


# --------------------------------------------------------------------------
# Hand-derived golden arrays
# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def gold():
    with open(GOLD) as f:
        return json.load(f)


def test_golden_canonical_and_formats(orc, gold):
    m = gold["matrix"]
    N, M = m["nrows"], m["ncols"]
    s = m["coo_shuffled"]
    st, r, c, v = orc.canonical(N, M, s["row"], s["col"], s["val"])
    assert st == orc.OK
    assert r.tolist() == gold["coo"]["row"]
    assert c.tolist() == gold["coo"]["col"]
    assert v.tolist() == gold["coo"]["val"]
    csr = orc.to_format("csr", N, M, r, c, v)
    assert csr["rowptr"].tolist() == gold["csr"]["rowptr"]
    dia = orc.to_format("dia", N, M, r, c, v)
    assert dia["offsets"].tolist() == gold["dia"]["offsets"]
    assert dia["val"].tolist() == gold["dia"]["val"]
    ell = orc.to_format("ell", N, M, r, c, v)
    assert ell["col"].tolist() == gold["ell"]["col"]
    assert ell["val"].tolist() == gold["ell"]["val"]
    for key, vb in (("hyb_f64", 8), ("hyb_f32", 4)):
        h = orc.to_format("hyb", N, M, r, c, v, vbytes=vb)
        g = gold[key]
        assert h["ell_col"].shape[0] == g["K"]
        assert h["coo_row"].size == g["over"]
        if g["K"]:
            assert h["ell_col"].tolist() == g["ell_col"]
            assert h["ell_val"].tolist() == g["ell_val"]
        assert h["coo_row"].tolist() == g["coo_row"]
        assert h["coo_col"].tolist() == g["coo_col"]
        assert h["coo_val"].tolist() == g["coo_val"]
    f = orc.features(N, M, r, c, vbytes=8, guard=3)
    for k, val in gold["features_f64"].items():
        assert f[k] == val, k


def test_golden_spmv_every_format(orc, gold):
    m = gold["matrix"]
    N, M = m["nrows"], m["ncols"]
    c0 = gold["coo"]
    x = np.array(gold["spmv"]["x"], float)
    for fmt in FMTS:
        a = orc.to_format(fmt, N, M, c0["row"], c0["col"], c0["val"])
        assert orc.spmv(fmt, N, M, a, x).tolist() == gold["spmv"]["y"], fmt
    assert (np.array(m["dense"]) @ x).tolist() == gold["spmv"]["y"]


def test_golden_hyb_width(orc, gold):
    g = gold["hyb_width_case"]
    row = np.repeat(np.arange(len(g["lengths"])), g["lengths"])
    assert orc.hyb_width(len(g["lengths"]), row, 8) == (g["K"], g["over"])


# --------------------------------------------------------------------------
# Canonical COO: validation and ordering
# --------------------------------------------------------------------------

def test_canonical_rejects_out_of_range_and_duplicates(orc):
    assert orc.canonical(3, 3, [0, 3], [0, 0], [1.0, 2.0])[0] == orc.INDEX_RANGE
    assert orc.canonical(3, 3, [0, 1], [0, -1], [1.0, 2.0])[0] == orc.INDEX_RANGE
    assert orc.canonical(3, 3, [1, 0, 1], [2, 0, 2], [1.0, 2.0, 3.0])[0] == orc.DUPLICATE
    # out-of-range wins over a duplicate
    assert orc.canonical(3, 3, [1, 1, 5], [2, 2, 0], [1.0, 2.0, 3.0])[0] == orc.INDEX_RANGE
    assert orc.canonical(-1, 3, [], [], [])[0] == orc.INVALID_ARG
    st, r, c, v = orc.canonical(0, 0, [], [], [])
    assert st == orc.OK and r.size == 0


def test_canonical_sorts_any_permutation(orc):
    r0, c0, v0 = synth.random_coo(5, 40, 30, 0.2)
    rs, cs, vs = synth.random_coo(5, 40, 30, 0.2, shuffle=True)
    st, r, c, v = orc.canonical(40, 30, rs, cs, vs)
    assert st == orc.OK
    assert np.array_equal(r, r0) and np.array_equal(c, c0) and np.array_equal(v, v0)


# --------------------------------------------------------------------------
# SpMV against brute force and exact arithmetic
# --------------------------------------------------------------------------

SHAPES = [(1, 1, 1.0), (7, 3, 0.5), (3, 9, 0.4), (33, 33, 0.1), (64, 50, 0.07), (64, 64, 0.3),
          (20, 20, 0.0)]


@pytest.mark.parametrize("shape", SHAPES)
def test_spmv_matches_dense_bruteforce(orc, shape):
    N, M, dens = shape
    r, c, v = synth.random_coo(11 + N, N, M, dens)
    x = synth.uniform_pm1(3, M)
    yd = dense_of(N, M, r, c, v) @ x
    bound = np.abs(dense_of(N, M, r, c, v)) @ np.abs(x)
    for fmt in FMTS:
        a = orc.to_format(fmt, N, M, r, c, v)
        y = orc.spmv(fmt, N, M, a, x)
        assert np.all(np.abs(y - yd) <= 1e-13 * bound), fmt
        assert np.all(y[bound == 0] == 0.0), fmt


@pytest.mark.parametrize("shape", SHAPES[:6])
def test_spmv_integer_inputs_are_exact(orc, shape):
    N, M, dens = shape
    r, c, v = synth.random_coo(17 + N, N, M, dens, int_values=True)
    x = synth.randint(9, M, -3, 4).astype(float)
    yd = dense_of(N, M, r, c, v) @ x
    for fmt in FMTS:
        a = orc.to_format(fmt, N, M, r, c, v)
        assert np.array_equal(orc.spmv(fmt, N, M, a, x), yd), fmt


@pytest.mark.parametrize("kind", ["random", "stencil"])
def test_openmp_build_matches_serial_bit_for_bit(orc, kind):
    """The multi-core baseline (the same source built with -fopenmp) splits
    rows across threads; every row's sum keeps its order, so each product is
    bit-identical to the serial build's and within the brute-force bound."""
    if kind == "random":
        N = M = 3000
        r, c, v = synth.random_coo(5, N, M, 0.004)
    else:
        N, r, c, v = synth.stencil27(9)
        M = N
    x = synth.uniform_pm1(4, M)
    A = dense_of(N, M, r, c, v)
    yd, bound = A @ x, np.abs(A) @ np.abs(x)
    assert orc.threads(omp=False) == 1
    for fmt in FMTS:
        a = orc.to_format(fmt, N, M, r, c, v)
        y1 = orc.spmv(fmt, N, M, a, x)
        yp = orc.spmv(fmt, N, M, a, x, omp=True)
        assert np.array_equal(y1.view(np.int64), yp.view(np.int64)), fmt
        assert np.all(np.abs(yp - yd) <= 1e-13 * bound), fmt


def test_spmv_within_rounding_bound_of_exact_sum(orc):
    N, M = 24, 40
    r, c, v = synth.random_coo(23, N, M, 0.35)
    x = synth.uniform_pm1(4, M)
    u = 2.0 ** -53
    for fmt in FMTS:
        a = orc.to_format(fmt, N, M, r, c, v)
        y = orc.spmv(fmt, N, M, a, x)
        for i in range(N):
            sel = np.nonzero(r == i)[0]
            exact = sum((Fraction(float(v[e])) * Fraction(float(x[c[e]])) for e in sel), Fraction(0))
            n_terms = max(1, sel.size)
            # DIA also adds its padded zeros, which are exact (+0.0 * x).
            gamma = n_terms * u / (1 - n_terms * u)
            s_abs = sum(abs(float(v[e]) * float(x[c[e]])) for e in sel)
            assert abs(Fraction(float(y[i])) - exact) <= Fraction(gamma) * Fraction(s_abs) + Fraction(0), (fmt, i)


def test_spmv_f32_error_scale(orc):
    N = 300
    Nn, r, c, v = synth.stencil27(5)[0], *synth.stencil27(5)[1:]
    N = Nn
    x = synth.uniform_pm1(5, N)
    rp = orc.coo_to_csr(N, r)
    y32 = orc.spmv_csr_f32(N, rp, c, v.astype(np.float32), x.astype(np.float32))
    A = dense_of(N, N, r, c, v)
    yd = A @ x.astype(np.float32).astype(np.float64)
    bound = np.abs(A) @ np.abs(x)
    err = np.abs(y32 - yd) / bound
    # 27 terms, each step rounds to float: |err| <= 27 * 2^-24 comfortably.
    assert err.max() <= 27 * 2.0 ** -24
    assert err.max() > 0  # it really is float arithmetic


# --------------------------------------------------------------------------
# 27-point stencil closed forms
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n", [3, 4, 5])
def test_stencil_generator_matches_kron(n):
    N, r, c, v = synth.stencil27(n)
    assert r.size == (3 * n - 2) ** 3
    assert np.array_equal(dense_of(N, N, r, c, v), kron_stencil(n))


@pytest.mark.parametrize("n", [3, 4, 5, 7])
def test_stencil_row_sums_every_format(orc, n):
    N, r, c, v = synth.stencil27(n)
    ones = np.ones(N)
    expect = {19.0: 8, 15.0: 12 * (n - 2), 9.0: 6 * (n - 2) ** 2, 0.0: (n - 2) ** 3}
    for fmt in FMTS:
        a = orc.to_format(fmt, N, N, r, c, v)
        y = orc.spmv(fmt, N, N, a, ones)
        vals, counts = np.unique(y, return_counts=True)
        got = dict(zip(vals.tolist(), counts.tolist()))
        assert got == {k: cnt for k, cnt in expect.items() if cnt}, fmt


@pytest.mark.parametrize("n,abc", [(5, (1, 1, 1)), (5, (5, 5, 5)), (6, (2, 3, 5)), (6, (6, 1, 4))])
def test_stencil_eigenpairs(orc, n, abc):
    N, r, c, v = synth.stencil27(n)
    i = np.arange(1, n + 1)
    s = [np.sin(k * i * math.pi / (n + 1)) for k in abc]
    t = [1 + 2 * math.cos(k * math.pi / (n + 1)) for k in abc]
    lam = 27 - t[0] * t[1] * t[2]
    # row index = ix + n*(iy + n*iz): x fastest, so the Kronecker order is z, y, x
    vec = np.kron(s[2], np.kron(s[1], s[0]))
    bound = 27 * np.abs(vec).max() * 2
    for fmt in FMTS:
        a = orc.to_format(fmt, N, N, r, c, v)
        res = orc.spmv(fmt, N, N, a, vec) - lam * vec
        assert np.abs(res).max() <= 1e-13 * bound, fmt


@pytest.mark.parametrize("n", [3, 4, 9])
def test_stencil_dia_and_ell_shape(orc, n):
    N, r, c, v = synth.stencil27(n)
    dia = orc.to_format("dia", N, N, r, c, v)
    expect = sorted(dz * n * n + dy * n + dx for dz in (-1, 0, 1) for dy in (-1, 0, 1)
                    for dx in (-1, 0, 1))
    assert dia["offsets"].tolist() == expect
    ell = orc.to_format("ell", N, N, r, c, v)
    assert ell["col"].shape[0] == 27
    # DIA padding: 27 N slots hold (3n-2)^3 entries
    assert int((dia["val"] != 0).sum()) == (3 * n - 2) ** 3


# --------------------------------------------------------------------------
# Conversions: round trips through COO, explicit zeros
# --------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(1, 1, 1.0), (9, 4, 0.5), (4, 9, 0.5), (40, 40, 0.15), (57, 31, 0.2)])
def test_round_trip_every_pair(orc, shape):
    N, M, dens = shape
    r, c, v = synth.random_coo(31 + N, N, M, dens)
    assert np.all(v != 0)
    for src in FMTS:
        a = orc.to_format(src, N, M, r, c, v)
        for dst in FMTS:
            b = orc.convert(src, dst, N, M, a)
            r2, c2, v2 = orc.to_coo(dst, N, M, b)
            assert np.array_equal(r2, r) and np.array_equal(c2, c) and np.array_equal(v2, v), (src, dst)


def test_explicit_zeros_kept_except_through_dia(orc):
    r = np.array([0, 0, 1, 2], np.int32)
    c = np.array([0, 1, 1, 0], np.int32)
    v = np.array([1.0, 0.0, -0.0, 2.0])
    for fmt in ("coo", "csr", "ell", "hyb"):
        r2, c2, v2 = orc.to_coo(fmt, 3, 2, orc.to_format(fmt, 3, 2, r, c, v))
        assert r2.tolist() == r.tolist() and c2.tolist() == c.tolist()
    r2, c2, v2 = orc.to_coo("dia", 3, 2, orc.to_format("dia", 3, 2, r, c, v))
    assert r2.tolist() == [0, 2] and c2.tolist() == [0, 0] and v2.tolist() == [1.0, 2.0]


def test_empty_and_degenerate(orc):
    e = np.zeros(0, np.int32)
    for fmt in FMTS:
        a = orc.to_format(fmt, 5, 4, e, e, np.zeros(0))
        assert orc.spmv(fmt, 5, 4, a, np.ones(4)).tolist() == [0.0] * 5
        r2, c2, v2 = orc.to_coo(fmt, 5, 4, a)
        assert r2.size == 0
    # one dense row
    r = np.zeros(6, np.int32)
    c = np.arange(6, dtype=np.int32)
    v = np.arange(1.0, 7.0)
    for fmt in FMTS:
        a = orc.to_format(fmt, 3, 6, r, c, v)
        assert orc.spmv(fmt, 3, 6, a, np.ones(6)).tolist() == [21.0, 0.0, 0.0]


# --------------------------------------------------------------------------
# HYB width and the format rule
# --------------------------------------------------------------------------

def test_hyb_width_invariants(orc):
    # every row the same length L: pure ELL (k = L) is cheapest
    for L in (1, 4, 9):
        row = np.repeat(np.arange(50), L)
        assert orc.hyb_width(50, row, 8) == (L, 0)
        assert orc.hyb_width(50, row, 4) == (L, 0)
    # one long row among short ones: the width follows the short rows
    lens = [2] * 99 + [400]
    row = np.repeat(np.arange(100), lens)
    assert orc.hyb_width(100, row, 8) == (2, 398)
    # empty matrix
    assert orc.hyb_width(10, np.zeros(0, np.int32), 8) == (0, 0)


def test_hyb_never_costs_more_than_coo_or_ell(orc):
    for seed in range(5):
        N, r, c, v = synth.powerlaw(200 + seed, 3000)
        f = orc.features(N, N, r, c)
        assert f["bytes"][orc.HYB] <= f["bytes"][orc.COO]
        assert f["bytes"][orc.HYB] <= f["bytes"][orc.ELL]


def test_selector_hand_checked_cases(orc):
    N, r, c, v = synth.stencil27(16)
    f = orc.features(N, N, r, c)
    assert f["ndiag"] == 27 and f["maxlen"] == 27 and f["nnz"] == 97336
    assert f["choice"] == orc.DIA
    # identity: one diagonal
    i = np.arange(100, dtype=np.int32)
    assert orc.features(100, 100, i, i)["choice"] == orc.DIA
    # uniform random rows: DIA and ELL padding are out of bounds or dearer
    N, r, c, v = synth.uniform(7, 5000)
    f = orc.features(N, N, r, c)
    assert f["ndiag"] > 1000 and f["choice"] == orc.CSR
    # power-law rows: ELL is excluded by the guard, HYB or CSR wins
    N, r, c, v = synth.powerlaw(8, 5000)
    f = orc.features(N, N, r, c)
    assert f["bytes"][orc.ELL] > 3 * f["bytes"][orc.CSR]
    assert f["choice"] in (orc.CSR, orc.HYB)


# --------------------------------------------------------------------------
# CG and mixed-precision refinement
# --------------------------------------------------------------------------

def stencil_kappa(n):
    t1 = 1 + 2 * math.cos(math.pi / (n + 1))
    tn = 1 + 2 * math.cos(n * math.pi / (n + 1))
    lmin = 27 - t1 ** 3
    lmax = 27 - t1 * t1 * tn
    return lmax / lmin


def test_cg_recovers_all_ones_16cubed(orc):
    N, r, c, v = synth.stencil27(16)
    rp = orc.coo_to_csr(N, r)
    b = orc.spmv("csr", N, N, {"rowptr": rp, "col": c, "val": v}, np.ones(N))
    out = orc.cg(N, rp, c, v, b, tol=1e-9, max_iters=500)
    assert out["status"] == orc.OK
    A = kron_stencil(16) if N <= 4096 else None
    res = np.linalg.norm(b - A @ out["x"]) / np.linalg.norm(b)
    assert res <= 2e-9
    assert abs(res - out["true_rel_residual"]) <= 1e-12
    kappa = stencil_kappa(16)
    assert 38.5 < kappa < 39.5
    assert np.linalg.norm(out["x"] - 1) / math.sqrt(N) <= kappa * 1e-9


def test_cg_obeys_spectral_bound(orc):
    n = 6
    N, r, c, v = synth.stencil27(n)
    A = kron_stencil(n)
    rp = orc.coo_to_csr(N, r)
    b = A @ np.ones(N)
    kappa = stencil_kappa(n)
    rate = (math.sqrt(kappa) - 1) / (math.sqrt(kappa) + 1)
    e0 = np.ones(N)
    e0A = math.sqrt(e0 @ A @ e0)
    for k in (1, 2, 4, 8, 12):
        out = orc.cg(N, rp, c, v, b, tol=0.0, max_iters=k)
        assert out["iterations"] == k and out["status"] == orc.NOT_CONVERGED
        e = out["x"] - 1
        assert math.sqrt(e @ A @ e) <= 2 * rate ** k * e0A * (1 + 1e-12)
    # and the relative residual history is what the iterates give
    out = orc.cg(N, rp, c, v, b, tol=1e-12, max_iters=200, history=True)
    assert out["history"][0] == 1.0 and out["history"][-1] <= 1e-12


def test_cg_distinct_eigenvalues_finish_in_that_many_steps(orc):
    d = np.array([2.0, 5.0, 11.0] * 20)
    i = np.arange(60, dtype=np.int32)
    rp = orc.coo_to_csr(60, i)
    b = synth.uniform_pm1(12, 60)
    out = orc.cg(60, rp, i, d, b, tol=1e-13, max_iters=10)
    assert out["status"] == orc.OK and out["iterations"] == 3
    assert np.allclose(out["x"], b / d, rtol=1e-12, atol=0)


def test_cg_edge_cases(orc):
    i = np.arange(10, dtype=np.int32)
    rp = orc.coo_to_csr(10, i)
    out = orc.cg(10, rp, i, -np.ones(10), np.ones(10), tol=1e-9, max_iters=5)
    assert out["status"] == orc.BREAKDOWN and out["iterations"] == 0
    out = orc.cg(10, rp, i, np.ones(10), np.zeros(10), tol=1e-9, max_iters=5)
    assert out["status"] == orc.OK and out["iterations"] == 0
    N, r, c, v = synth.stencil27(8)
    rp = orc.coo_to_csr(N, r)
    out = orc.cg(N, rp, c, v, np.ones(N), tol=1e-14, max_iters=3)
    assert out["status"] == orc.NOT_CONVERGED and out["iterations"] == 3


def test_ir_mixed_reaches_fp64_accuracy(orc):
    n = 12
    N, r, c, v = synth.stencil27(n)
    rp = orc.coo_to_csr(N, r)
    A = kron_stencil(n)
    b = A @ np.ones(N)
    out = orc.ir_mixed(N, rp, c, v, b, tol=1e-10, inner_tol=1e-5)
    assert out["status"] == orc.OK
    res = np.linalg.norm(b - A @ out["x"]) / np.linalg.norm(b)
    assert res <= 1e-10
    # FP32 alone cannot reach 1e-10: the refinement really iterates
    assert out["outer"] >= 2
    assert np.linalg.norm(out["x"] - 1) / math.sqrt(N) <= stencil_kappa(n) * 1e-10 * 2


def test_ir_mixed_gives_up_after_max_outer(orc):
    N, r, c, v = synth.stencil27(6)
    rp = orc.coo_to_csr(N, r)
    b = synth.uniform_pm1(3, N)
    out = orc.ir_mixed(N, rp, c, v, b, tol=1e-30, inner_tol=1e-3, max_outer=2)
    assert out["status"] == orc.NOT_CONVERGED and out["outer"] == 2


# --------------------------------------------------------------------------
# Mixed precision with reliable updates
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n", [16, 24])
def test_reliable_mixed_reaches_1e10_at_about_fp64_iterations(orc, n):
    N, r, c, v = synth.stencil27(n)
    rp = orc.coo_to_csr(N, r)
    A = kron_stencil(n) if n <= 16 else None
    b = synth.uniform_pm1(n, N)
    out = orc.cg_reliable(N, rp, c, v, b, tol=1e-10)
    assert out["status"] == orc.OK and out["folds"] >= 2
    y = orc.spmv("csr", N, N, {"rowptr": rp, "col": c, "val": v}, out["x"])
    res = np.linalg.norm(b - y) / np.linalg.norm(b)
    assert res <= 1e-10 and abs(res - out["true_rel_residual"]) <= 1e-14
    if A is not None:
        assert np.linalg.norm(b - A @ out["x"]) / np.linalg.norm(b) <= 1e-10
    ref = orc.cg(N, rp, c, v, b, tol=1e-10, max_iters=5000)
    # the direction survives each fold: no restart, so the count stays near FP64 CG's
    assert out["iterations"] <= 1.15 * ref["iterations"] + 5
    # restarted refinement loses the direction at each restart: more iterations
    ir = orc.ir_mixed(N, rp, c, v, b, tol=1e-10, inner_tol=1e-5)
    assert ir["inner_total"] > out["iterations"]


def test_reliable_mixed_without_folds_stalls_in_fp32(orc):
    N, r, c, v = synth.stencil27(16)
    rp = orc.coo_to_csr(N, r)
    b = synth.uniform_pm1(5, N)
    # delta = 0 and an unreachable tolerance: the only fold is the final one
    out = orc.cg_reliable(N, rp, c, v, b, tol=1e-30, delta=0.0, max_iters=60)
    assert out["status"] == orc.NOT_CONVERGED and out["folds"] == 1
    assert out["true_rel_residual"] > 1e-8  # FP32 alone stalls far from FP64 accuracy
    ok = orc.cg_reliable(N, rp, c, v, b, tol=1e-30, delta=0.1, max_iters=60)
    assert ok["folds"] > 5 and ok["true_rel_residual"] < 1e-13


def test_reliable_mixed_edge_cases(orc):
    d = np.array([2.0, 5.0, 11.0] * 20)
    i = np.arange(60, dtype=np.int32)
    rp = orc.coo_to_csr(60, i)
    b = synth.uniform_pm1(12, 60)
    out = orc.cg_reliable(60, rp, i, d, b, tol=1e-12)
    assert out["status"] == orc.OK and out["iterations"] <= 8
    assert np.allclose(out["x"], b / d, rtol=1e-12, atol=0)
    out = orc.cg_reliable(10, orc.coo_to_csr(10, i[:10]), i[:10], -np.ones(10), np.ones(10))
    assert out["status"] == orc.BREAKDOWN and out["iterations"] == 0
    out = orc.cg_reliable(10, orc.coo_to_csr(10, i[:10]), i[:10], np.ones(10), np.zeros(10))
    assert out["status"] == orc.OK and out["iterations"] == 0


# ---------------------------------------------------------------------------
# Diagonal extraction / update (§III-D, §IV-B)
# ---------------------------------------------------------------------------

def test_diagonal_against_dense(orc):
    for seed, (nr, nc) in ((31, (12, 12)), (32, (9, 14)), (33, (15, 7))):
        r, c, v = synth.random_coo(seed, nr, nc, 0.3)
        st, r2, c2, v2 = orc.canonical(nr, nc, r, c, v)
        dense = np.zeros((nr, nc))
        dense[r2, c2] = v2
        d, stored = orc.diagonal(nr, nc, r2, c2, v2)
        n = min(nr, nc)
        assert np.array_equal(d, np.diag(dense)[:n])
        assert stored == int(np.sum(r2 == c2))
        newd = synth.uniform_pm1(seed + 1, n) + 2.0
        v3, k = orc.set_diagonal(r2, c2, v2, newd)
        assert k == stored
        dense3 = np.zeros((nr, nc))
        dense3[r2, c2] = v3
        want = dense.copy()
        idx = np.arange(n)
        has = np.zeros(n, bool)
        has[r2[r2 == c2]] = True
        want[idx[has], idx[has]] = newd[has]     # only stored entries change
        assert np.array_equal(dense3, want)
        # off-diagonal values untouched, bit for bit
        assert np.array_equal(v3[r2 != c2], v2[r2 != c2])


def test_diagonal_of_stencil_is_26(orc):
    N, r, c, v = synth.stencil27(5)
    d, stored = orc.diagonal(N, N, r, c, v)
    assert stored == N and np.all(d == 26.0)


# ---------------------------------------------------------------------------
# HPCG's preconditioned CG: coloured symmetric Gauss-Seidel and multigrid
# ---------------------------------------------------------------------------

def test_colouring_separates_stencil_neighbours():
    N, r, c, v = synth.stencil(6, 27, 4, 8)
    nx, ny = 6, 4
    col = lambda i: 7 - ((i % nx & 1) + 2 * ((i // nx) % ny & 1) + 4 * (i // (nx * ny) & 1))
    off = r != c
    assert not np.any(col(r[off]) == col(c[off]))


def test_symgs_solves_a_diagonal_matrix_exactly(orc):
    n = 4 * 6 * 2
    d = synth.uniform_pm1(3, n) + 3.0
    level = {"dims": (4, 6, 2), "n": n, "rowptr": np.arange(n + 1, dtype=np.int32),
             "col": np.arange(n, dtype=np.int32), "val": d}
    r = synth.uniform_pm1(4, n)
    z = orc.symgs(level, r, np.zeros(n))
    assert np.array_equal(z, r / d)


def test_symgs_reduces_to_gauss_seidel_by_hand(orc):
    # 2 x 1 x 1 grid: row 1 (odd x) is colour 6, row 0 (even) colour 7; the
    # forward pass updates row 1 then row 0, the backward pass row 0 then
    # row 1
    level = {"dims": (2, 1, 1), "n": 2, "rowptr": np.array([0, 2, 4], np.int32),
             "col": np.array([0, 1, 0, 1], np.int32), "val": np.array([4.0, 1.0, 1.0, 3.0])}
    r = np.array([1.0, 2.0])
    z1 = (2.0 - 1.0 * 0.0) / 3.0
    z0 = (1.0 - 1.0 * z1) / 4.0
    z0b = (1.0 - 1.0 * z1) / 4.0
    z1b = (2.0 - 1.0 * z0b) / 3.0
    assert np.array_equal(orc.symgs(level, r, np.zeros(2)), np.array([z0b, z1b]))
    assert z0 == z0b


@pytest.mark.parametrize("nlev", [1, 2, 3])
def test_preconditioner_is_symmetric_positive_definite(orc, nlev):
    levels = orc.stencil_levels((8, 8, 8), nlev)
    n = levels[0]["n"]
    u, w = synth.uniform_pm1(5, n), synth.uniform_pm1(6, n)
    Mu, Mw = orc.mg_apply(levels, u), orc.mg_apply(levels, w)
    assert abs(np.dot(w, Mu) - np.dot(u, Mw)) <= 1e-12 * np.linalg.norm(u) * np.linalg.norm(Mw)
    assert np.dot(u, Mu) > 0 and np.dot(w, Mw) > 0


def test_pcg_without_preconditioner_is_cg(orc):
    levels = orc.stencil_levels((12, 12, 12), 1)
    L = levels[0]
    b = synth.uniform_pm1(7, L["n"])
    p = orc.pcg(levels, b, nlev=0, tol=1e-10, max_iters=300)
    c = orc.cg(L["n"], L["rowptr"], L["col"], L["val"], b, tol=1e-10, max_iters=300)
    assert p["iterations"] == c["iterations"]
    assert np.array_equal(p["x"], c["x"])


def test_pcg_converges_in_far_fewer_iterations(orc):
    levels = orc.stencil_levels((16, 16, 16), 3)
    L = levels[0]
    ones = np.ones(L["n"])
    b = orc.spmv("csr", L["n"], L["n"], L, ones)
    plain = orc.pcg(levels, b, nlev=0, tol=1e-9, max_iters=500)
    mg = orc.pcg(levels, b, tol=1e-9, max_iters=500)
    assert mg["status"] == 0 and plain["status"] == 0
    assert mg["iterations"] * 1.7 <= plain["iterations"]
    assert mg["true_rel_residual"] <= 1e-8
    assert np.max(np.abs(mg["x"] - 1.0)) < 1e-6


def test_coarse_levels_contribute(orc):
    """The coarse grids get a nonzero right-hand side (the last colour of a
    sweep has zero residual, so it must not be the injected points) and a
    deeper hierarchy converges faster than a single smoother."""
    levels = orc.stencil_levels((32, 32, 32), 4)
    r = synth.uniform_pm1(8, levels[0]["n"])
    assert np.max(np.abs(orc.mg_apply(levels[:3], r) - orc.mg_apply(levels[:2], r))) > 1e-6
    L = levels[0]
    b = orc.spmv("csr", L["n"], L["n"], L, np.ones(L["n"]))
    one = orc.pcg(levels, b, nlev=1, tol=1e-9, max_iters=500)
    four = orc.pcg(levels, b, nlev=4, tol=1e-9, max_iters=500)
    assert four["iterations"] * 1.4 <= one["iterations"]
