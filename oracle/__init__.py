"""CPU oracle — test infrastructure only.

A ctypes view of ``orc.c``: the plain single-threaded FP64 statement of the
method (formats and conversions of §II-A / §III-B, SpMV of §III-D, the
deterministic format rule, CG of §II-B / §IV-B and mixed-precision
refinement). Only the tests, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg import this package; the product library never does, and
this package never imports the product.

Arrays are numpy; DIA values come back as a (ndiag, nrows) array and ELL
arrays as (K, nrows), i.e. slot-major as the C code stores them.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "orc.c")
LIB = os.path.join(HERE, "liborc.so")
LIB_OMP = os.path.join(HERE, "liborc_omp.so")

OK, INVALID_ARG, INDEX_RANGE, DUPLICATE, OOM, FORMAT_TOO_LARGE = 0, 1, 2, 3, 4, 5
BREAKDOWN, NOT_CONVERGED = 7, 8
COO, CSR, DIA, ELL, HYB = 0, 1, 2, 3, 4
FORMATS = ("coo", "csr", "dia", "ell", "hyb")

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC"]


def build(force: bool = False, omp: bool = False) -> str:
    """Compiles orc.c into liborc.so, or with -fopenmp into liborc_omp.so
    (the multi-core baseline); skipped when up to date."""
    out = LIB_OMP if omp else LIB
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(SRC)):
        return out
    tmp = out + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", *CFLAGS, *(["-fopenmp"] if omp else []), SRC, "-o", tmp, "-lm"])
    os.replace(tmp, out)
    return out


_lib = None
_lib_omp = None


class Features(C.Structure):
    _fields_ = [("nrows", C.c_int64), ("ncols", C.c_int64), ("nnz", C.c_int64),
                ("ndiag", C.c_int64), ("maxlen", C.c_int64), ("hyb_k", C.c_int64),
                ("hyb_over", C.c_int64), ("bytes", C.c_int64 * 5), ("choice", C.c_int64)]


def lib(omp: bool = False):
    """The serial oracle, or with omp=True the same source built with -fopenmp."""
    global _lib, _lib_omp
    if omp:
        if _lib_omp is None:
            _lib_omp = _declare(C.CDLL(build(omp=True)))
        return _lib_omp
    if _lib is None:
        _lib = _declare(C.CDLL(build()))
    return _lib


def _declare(L):
    i64, vp, dbl = C.c_int64, C.c_void_p, C.c_double
    sig = {
        "orc_coo_canonical": (C.c_int, [i64, i64, i64, vp, vp, vp, vp, vp, vp]),
        "orc_coo_to_csr": (None, [i64, i64, vp, vp]),
        "orc_csr_to_coo": (None, [i64, vp, vp]),
        "orc_dia_ndiag": (i64, [i64, i64, i64, vp, vp]),
        "orc_coo_to_dia": (None, [i64, i64, i64, vp, vp, vp, vp, vp]),
        "orc_dia_to_coo": (i64, [i64, i64, i64, vp, vp, vp, vp, vp]),
        "orc_max_row_length": (i64, [i64, i64, vp]),
        "orc_coo_to_ell": (None, [i64, i64, vp, vp, vp, i64, vp, vp]),
        "orc_ell_to_coo": (i64, [i64, i64, vp, vp, vp, vp, vp]),
        "orc_hyb_width": (i64, [i64, i64, vp, i64, vp]),
        "orc_coo_to_hyb": (None, [i64, i64, vp, vp, vp, i64, vp, vp, vp, vp, vp]),
        "orc_hyb_to_coo": (i64, [i64, i64, vp, vp, i64, vp, vp, vp, vp, vp, vp]),
        "orc_features_select": (None, [i64, i64, i64, vp, vp, i64, i64, vp]),
        "orc_threads": (i64, []),
        "orc_spmv_coo": (None, [i64, i64, vp, vp, vp, vp, vp]),
        "orc_spmv_csr": (None, [i64, vp, vp, vp, vp, vp]),
        "orc_spmv_dia": (None, [i64, i64, i64, vp, vp, vp, vp]),
        "orc_spmv_ell": (None, [i64, i64, vp, vp, vp, vp]),
        "orc_spmv_hyb": (None, [i64, i64, vp, vp, i64, vp, vp, vp, vp, vp]),
        "orc_spmv_csr_f32": (None, [i64, vp, vp, vp, vp, vp]),
        "orc_diagonal": (i64, [i64, i64, i64, vp, vp, vp, vp]),
        "orc_symgs": (None, [i64, i64, i64, vp, vp, vp, vp, vp]),
        "orc_mg_apply": (None, [i64, vp, vp, vp, vp, vp, vp]),
        "orc_pcg": (C.c_int, [i64, vp, vp, vp, vp, vp, vp, C.c_double, i64, vp, vp, vp,
                              vp]),
        "orc_set_diagonal": (i64, [i64, vp, vp, vp, vp]),
        "orc_cg_csr": (C.c_int, [i64, vp, vp, vp, vp, vp, dbl, i64, vp, vp, vp, vp]),
        "orc_ir_mixed_csr": (C.c_int, [i64, vp, vp, vp, vp, vp, dbl, dbl, i64, i64,
                                       vp, vp, vp]),
        "orc_cg_reliable_csr": (C.c_int, [i64, vp, vp, vp, vp, vp, dbl, dbl, i64, vp, vp,
                                          vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


def threads(omp: bool = False) -> int:
    """Threads the SpMV row loops use: 1 for the serial build, the OpenMP
    team size (OMP_NUM_THREADS, else all cores) for the other."""
    return int(lib(omp).orc_threads())


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------
# Formats and conversions (every conversion goes through COO, §III-B)
# ---------------------------------------------------------------------------

def canonical(nrows, ncols, row, col, val):
    """(status, row, col, val) sorted by (row, col); status != OK on
    out-of-range indices or duplicate positions."""
    row, col, val = _i32(row), _i32(col), _f64(val)
    nnz = row.size
    o = (np.empty(nnz, np.int32), np.empty(nnz, np.int32), np.empty(nnz, np.float64))
    st = lib().orc_coo_canonical(nrows, ncols, nnz, _p(row), _p(col), _p(val), *map(_p, o))
    return (st,) + (o if st == OK else (None, None, None))


def coo_to_csr(nrows, row):
    row = _i32(row)
    rp = np.empty(nrows + 1, np.int32)
    lib().orc_coo_to_csr(nrows, row.size, _p(row), _p(rp))
    return rp


def csr_to_coo(nrows, rowptr):
    rowptr = _i32(rowptr)
    row = np.empty(int(rowptr[-1]), np.int32)
    lib().orc_csr_to_coo(nrows, _p(rowptr), _p(row))
    return row


def coo_to_dia(nrows, ncols, row, col, val):
    row, col, val = _i32(row), _i32(col), _f64(val)
    nd = lib().orc_dia_ndiag(nrows, ncols, row.size, _p(row), _p(col))
    off = np.empty(nd, np.int32)
    dval = np.empty((nd, nrows), np.float64)
    lib().orc_coo_to_dia(nrows, ncols, row.size, _p(row), _p(col), _p(val), _p(off), _p(dval))
    return off, dval


def dia_to_coo(nrows, ncols, offsets, dval):
    offsets, dval = _i32(offsets), _f64(dval)
    nd = offsets.size
    m = lib().orc_dia_to_coo(nrows, ncols, nd, _p(offsets), _p(dval), None, None, None)
    o = (np.empty(m, np.int32), np.empty(m, np.int32), np.empty(m, np.float64))
    lib().orc_dia_to_coo(nrows, ncols, nd, _p(offsets), _p(dval), *map(_p, o))
    return o


def max_row_length(nrows, row):
    row = _i32(row)
    return lib().orc_max_row_length(nrows, row.size, _p(row))


def coo_to_ell(nrows, row, col, val):
    row, col, val = _i32(row), _i32(col), _f64(val)
    K = lib().orc_max_row_length(nrows, row.size, _p(row))
    ecol = np.empty((K, nrows), np.int32)
    evl = np.empty((K, nrows), np.float64)
    lib().orc_coo_to_ell(nrows, row.size, _p(row), _p(col), _p(val), K, _p(ecol), _p(evl))
    return ecol, evl


def ell_to_coo(nrows, ecol, evl):
    ecol, evl = _i32(ecol), _f64(evl)
    K = ecol.shape[0] if ecol.ndim == 2 else 0
    m = lib().orc_ell_to_coo(nrows, K, _p(ecol), _p(evl), None, None, None)
    o = (np.empty(m, np.int32), np.empty(m, np.int32), np.empty(m, np.float64))
    lib().orc_ell_to_coo(nrows, K, _p(ecol), _p(evl), *map(_p, o))
    return o


def hyb_width(nrows, row, vbytes=8):
    row = _i32(row)
    over = C.c_int64(0)
    k = lib().orc_hyb_width(nrows, row.size, _p(row), vbytes, C.byref(over))
    return int(k), int(over.value)


def coo_to_hyb(nrows, row, col, val, vbytes=8):
    row, col, val = _i32(row), _i32(col), _f64(val)
    Kh, over = hyb_width(nrows, row, vbytes)
    ecol = np.empty((Kh, nrows), np.int32)
    evl = np.empty((Kh, nrows), np.float64)
    crow, ccol, cval = np.empty(over, np.int32), np.empty(over, np.int32), np.empty(over, np.float64)
    lib().orc_coo_to_hyb(nrows, row.size, _p(row), _p(col), _p(val), Kh, _p(ecol), _p(evl),
                         _p(crow), _p(ccol), _p(cval))
    return ecol, evl, crow, ccol, cval


def hyb_to_coo(nrows, ecol, evl, crow, ccol, cval):
    ecol, evl = _i32(ecol), _f64(evl)
    crow, ccol, cval = _i32(crow), _i32(ccol), _f64(cval)
    Kh = ecol.shape[0] if ecol.ndim == 2 else 0
    args = (nrows, Kh, _p(ecol), _p(evl), crow.size, _p(crow), _p(ccol), _p(cval))
    m = lib().orc_hyb_to_coo(*args, None, None, None)
    o = (np.empty(m, np.int32), np.empty(m, np.int32), np.empty(m, np.float64))
    lib().orc_hyb_to_coo(*args, *map(_p, o))
    return o


def to_format(fmt, nrows, ncols, row, col, val, vbytes=8):
    """Canonical COO -> the arrays of `fmt` as a dict."""
    fmt = FORMATS[fmt] if isinstance(fmt, int) else fmt
    if fmt == "coo":
        return {"row": _i32(row), "col": _i32(col), "val": _f64(val)}
    if fmt == "csr":
        return {"rowptr": coo_to_csr(nrows, row), "col": _i32(col), "val": _f64(val)}
    if fmt == "dia":
        off, dval = coo_to_dia(nrows, ncols, row, col, val)
        return {"offsets": off, "val": dval}
    if fmt == "ell":
        ecol, evl = coo_to_ell(nrows, row, col, val)
        return {"col": ecol, "val": evl}
    if fmt == "hyb":
        ecol, evl, crow, ccol, cval = coo_to_hyb(nrows, row, col, val, vbytes)
        return {"ell_col": ecol, "ell_val": evl, "coo_row": crow, "coo_col": ccol,
                "coo_val": cval}
    raise ValueError(fmt)


def to_coo(fmt, nrows, ncols, a):
    """The arrays of `fmt` -> canonical COO (row, col, val)."""
    fmt = FORMATS[fmt] if isinstance(fmt, int) else fmt
    if fmt == "coo":
        return a["row"], a["col"], a["val"]
    if fmt == "csr":
        return csr_to_coo(nrows, a["rowptr"]), a["col"], a["val"]
    if fmt == "dia":
        return dia_to_coo(nrows, ncols, a["offsets"], a["val"])
    if fmt == "ell":
        return ell_to_coo(nrows, a["col"], a["val"])
    if fmt == "hyb":
        return hyb_to_coo(nrows, a["ell_col"], a["ell_val"], a["coo_row"], a["coo_col"],
                          a["coo_val"])
    raise ValueError(fmt)


def convert(src_fmt, dst_fmt, nrows, ncols, a, vbytes=8):
    """X -> COO -> Y (§III-B proxy policy). Converting to the format that is
    already active changes nothing (§III-A: activate() of the active state)."""
    src_name = FORMATS[src_fmt] if isinstance(src_fmt, int) else src_fmt
    dst_name = FORMATS[dst_fmt] if isinstance(dst_fmt, int) else dst_fmt
    if src_name == dst_name:
        return {k: v.copy() for k, v in a.items()}
    row, col, val = to_coo(src_fmt, nrows, ncols, a)
    return to_format(dst_fmt, nrows, ncols, row, col, val, vbytes)


def features(nrows, ncols, row, col, vbytes=8, guard=3):
    row, col = _i32(row), _i32(col)
    f = Features()
    lib().orc_features_select(nrows, ncols, row.size, _p(row), _p(col), vbytes, guard, C.byref(f))
    return {"nrows": f.nrows, "ncols": f.ncols, "nnz": f.nnz, "ndiag": f.ndiag,
            "maxlen": f.maxlen, "hyb_k": f.hyb_k, "hyb_over": f.hyb_over,
            "bytes": list(f.bytes), "choice": f.choice}


# ---------------------------------------------------------------------------
# SpMV (§III-D)
# ---------------------------------------------------------------------------

def diagonal(nrows, ncols, row, col, val):
    """(d, stored) of a canonical COO matrix: d[i] = a(i, i) or 0, for
    i < min(nrows, ncols); stored = number of stored diagonal entries."""
    n = min(nrows, ncols)
    d = np.empty(n, np.float64)
    found = lib().orc_diagonal(nrows, ncols, row.size, _p(_i32(row)), _p(_i32(col)),
                               _p(_f64(val)), _p(d))
    return d, int(found)


def set_diagonal(row, col, val, d):
    """COO values with every stored (i, i) entry set to d[i]; (val', count)."""
    v = np.array(val, dtype=np.float64, copy=True)
    n = lib().orc_set_diagonal(row.size, _p(_i32(row)), _p(_i32(col)), _p(v), _p(_f64(d)))
    return v, int(n)


def spmv(fmt, nrows, ncols, a, x, omp=False):
    """y = A x in the format's natural order; omp=True runs the OpenMP build
    (CSR, DIA and ELL rows split across threads; same result)."""
    fmt = FORMATS[fmt] if isinstance(fmt, int) else fmt
    x = _f64(x)
    y = np.empty(nrows, np.float64)
    L = lib(omp)
    if fmt == "coo":
        L.orc_spmv_coo(nrows, a["row"].size, _p(_i32(a["row"])), _p(_i32(a["col"])),
                       _p(_f64(a["val"])), _p(x), _p(y))
    elif fmt == "csr":
        L.orc_spmv_csr(nrows, _p(_i32(a["rowptr"])), _p(_i32(a["col"])), _p(_f64(a["val"])),
                       _p(x), _p(y))
    elif fmt == "dia":
        off = _i32(a["offsets"])
        L.orc_spmv_dia(nrows, ncols, off.size, _p(off), _p(_f64(a["val"])), _p(x), _p(y))
    elif fmt == "ell":
        ecol = _i32(a["col"])
        K = ecol.shape[0] if ecol.ndim == 2 else 0
        L.orc_spmv_ell(nrows, K, _p(ecol), _p(_f64(a["val"])), _p(x), _p(y))
    elif fmt == "hyb":
        ecol = _i32(a["ell_col"])
        K = ecol.shape[0] if ecol.ndim == 2 else 0
        crow = _i32(a["coo_row"])
        L.orc_spmv_hyb(nrows, K, _p(ecol), _p(_f64(a["ell_val"])), crow.size, _p(crow),
                       _p(_i32(a["coo_col"])), _p(_f64(a["coo_val"])), _p(x), _p(y))
    else:
        raise ValueError(fmt)
    return y


def spmv_csr_f32(nrows, rowptr, col, val32, x32):
    y = np.empty(nrows, np.float32)
    lib().orc_spmv_csr_f32(nrows, _p(_i32(rowptr)), _p(_i32(col)),
                           _p(np.ascontiguousarray(val32, np.float32)),
                           _p(np.ascontiguousarray(x32, np.float32)), _p(y))
    return y


# ---------------------------------------------------------------------------
# Solvers
# ---------------------------------------------------------------------------

def cg(nrows, rowptr, col, val, b, x0=None, tol=1e-9, max_iters=1000, history=False):
    """Textbook CG (§II-B with the preconditioner disabled, §IV-B)."""
    b = _f64(b)
    x = np.zeros(nrows) if x0 is None else _f64(x0).copy()
    it, rel, trel = C.c_int64(0), C.c_double(0), C.c_double(0)
    hist = np.zeros(max_iters + 1) if history else None
    st = lib().orc_cg_csr(nrows, _p(_i32(rowptr)), _p(_i32(col)), _p(_f64(val)), _p(b), _p(x),
                          tol, max_iters, C.byref(it), C.byref(rel), C.byref(trel), _p(hist))
    out = {"status": st, "x": x, "iterations": it.value, "rel_residual": rel.value,
           "true_rel_residual": trel.value}
    if history:
        out["history"] = hist[: it.value + 1]
    return out


def stencil_levels(dims, nlev, kind=27):
    """The multigrid hierarchy of HPCG's problem: level l is the `kind`-point
    stencil on dims / 2^l, as canonical CSR. Returns a list of dicts."""
    import synth
    out = []
    nx, ny, nz = dims
    for _ in range(nlev):
        N, r, c, v = synth.stencil(nx, kind, ny, nz)
        st, r2, c2, v2 = canonical(N, N, r, c, v)
        out.append({"dims": (nx, ny, nz), "n": N, "rowptr": coo_to_csr(N, r2), "col": c2,
                    "val": v2})
        nx, ny, nz = nx // 2, ny // 2, nz // 2
    return out


def _level_args(levels):
    dims = np.array([d for L in levels for d in L["dims"]], dtype=np.int64)
    keep = [(_i32(L["rowptr"]), _i32(L["col"]), _f64(L["val"])) for L in levels]
    n = max(len(levels), 1)
    rp = (C.c_void_p * n)(*[k[0].ctypes.data for k in keep])
    cl = (C.c_void_p * n)(*[k[1].ctypes.data for k in keep])
    vl = (C.c_void_p * n)(*[k[2].ctypes.data for k in keep])
    return dims, keep, rp, cl, vl


def symgs(level, r, z):
    """One colour-ordered symmetric Gauss-Seidel sweep; returns the new z."""
    z = _f64(z).copy()
    nx, ny, nz = level["dims"]
    lib().orc_symgs(nx, ny, nz, _p(_i32(level["rowptr"])), _p(_i32(level["col"])),
                    _p(_f64(level["val"])), _p(_f64(r)), _p(z))
    return z


def mg_apply(levels, r):
    """z = M^{-1} r: one V-cycle over the levels (one level: one sweep)."""
    dims, keep, rp, cl, vl = _level_args(levels)
    z = np.empty(levels[0]["n"])
    lib().orc_mg_apply(len(levels), _p(dims), rp, cl, vl, _p(_f64(r)), _p(z))
    return z


def pcg(levels, b, nlev=None, x0=None, tol=1e-9, max_iters=1000, history=False):
    """PCG on levels[0] with a V-cycle over the first `nlev` levels as the
    preconditioner (nlev = 0: none, the textbook CG)."""
    nlev = len(levels) if nlev is None else nlev
    dims, keep, rp, cl, vl = _level_args(levels)
    n = levels[0]["n"]
    b = _f64(b)
    x = np.zeros(n) if x0 is None else _f64(x0).copy()
    it, rel, trel = C.c_int64(0), C.c_double(0), C.c_double(0)
    hist = np.zeros(max_iters + 1) if history else None
    st = lib().orc_pcg(nlev, _p(dims), rp, cl, vl, _p(b), _p(x), tol, max_iters, C.byref(it),
                       C.byref(rel), C.byref(trel), _p(hist))
    out = {"status": st, "x": x, "iterations": it.value, "rel_residual": rel.value,
           "true_rel_residual": trel.value}
    if history:
        out["history"] = hist[: it.value + 1]
    return out


def ir_mixed(nrows, rowptr, col, val, b, tol=1e-10, inner_tol=1e-5, inner_max=1000,
             max_outer=30):
    """FP32-inner / FP64-outer iterative refinement."""
    b = _f64(b)
    x = np.zeros(nrows)
    outer, inner, trel = C.c_int64(0), C.c_int64(0), C.c_double(0)
    st = lib().orc_ir_mixed_csr(nrows, _p(_i32(rowptr)), _p(_i32(col)), _p(_f64(val)), _p(b),
                                _p(x), tol, inner_tol, inner_max, max_outer, C.byref(outer),
                                C.byref(inner), C.byref(trel))
    return {"status": st, "x": x, "outer": outer.value, "inner_total": inner.value,
            "true_rel_residual": trel.value}


def cg_reliable(nrows, rowptr, col, val, b, tol=1e-10, delta=0.1, max_iters=5000):
    """Mixed precision with reliable updates: FP32 CG whose correction is
    folded into the FP64 solution (with an FP64 residual) whenever the
    recursive residual has dropped by `delta`; the direction is kept."""
    b = _f64(b)
    x = np.zeros(nrows)
    it, folds, trel = C.c_int64(0), C.c_int64(0), C.c_double(0)
    st = lib().orc_cg_reliable_csr(nrows, _p(_i32(rowptr)), _p(_i32(col)), _p(_f64(val)), _p(b),
                                   _p(x), tol, delta, max_iters, C.byref(it), C.byref(folds),
                                   C.byref(trel))
    return {"status": st, "x": x, "iterations": it.value, "folds": folds.value,
            "true_rel_residual": trel.value}
