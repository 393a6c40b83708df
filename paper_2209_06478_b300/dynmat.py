"""Python binding of the dynmat C ABI (include/dynmat.h): argument marshalling only.

Every call goes straight to libdynmat.so (hand-written sm_103a kernels).
There is no fallback: importing this module raises when the library is
missing, and calls raise DynmatError when the library returns an error.

Device arrays are torch CUDA tensors (PyTorch provides device memory and
streams); host arrays are numpy arrays or CPU tensors.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdynmat.so")

COO, CSR, DIA, ELL, HYB = 0, 1, 2, 3, 4
FORMATS = ("coo", "csr", "dia", "ell", "hyb")
F64, F32 = 0, 1
(OK, ERR_INVALID_ARG, ERR_INDEX_RANGE, ERR_DUPLICATE, ERR_OOM, ERR_FORMAT_TOO_LARGE, ERR_CUDA,
 ERR_BREAKDOWN, ERR_NOT_CONVERGED, ERR_TIMEOUT) = range(10)
SELECT_FEATURES, SELECT_PROFILE = 0, 1
CG_FP64, CG_MIXED, CG_MIXED_RELIABLE = 0, 1, 2
ARR_ROW, ARR_COL, ARR_VAL, ARR_ROWPTR, ARR_OFFSETS, ARR_HYB_COL, ARR_HYB_VAL = range(7)


class DynmatError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("dynmat error %d (%s): %s" % (status, status_string(status), message))
        self.status = status


class Info(C.Structure):
    _fields_ = [("format", C.c_int32), ("vdtype", C.c_int32), ("nrows", C.c_int64),
                ("ncols", C.c_int64), ("nnz", C.c_int64), ("ndiag", C.c_int64),
                ("ell_width", C.c_int64), ("hyb_coo_nnz", C.c_int64), ("ld", C.c_int64),
                ("bytes", C.c_int64), ("values_exact_in_f32", C.c_int32),
                ("spmv_variant", C.c_int32)]


class Features(C.Structure):
    _fields_ = [("nrows", C.c_int64), ("ncols", C.c_int64), ("nnz", C.c_int64),
                ("ndiag", C.c_int64), ("maxlen", C.c_int64), ("hyb_k", C.c_int64),
                ("hyb_over", C.c_int64), ("bytes", C.c_int64 * 5), ("choice", C.c_int32),
                ("guard", C.c_int32)]


class CgOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iters", C.c_int32), ("precision", C.c_int32),
                ("inner_tol", C.c_double), ("max_outer", C.c_int32), ("check_every", C.c_int32),
                ("delta", C.c_double)]


class CgResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("iterations", C.c_int32),
                ("outer_iterations", C.c_int32), ("rel_residual", C.c_double),
                ("true_rel_residual", C.c_double)]


class TileShape(C.Structure):
    _fields_ = [("lanes", C.c_int32), ("rows_per_tile", C.c_int32), ("nnz_per_tile", C.c_int32)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libdynmat.so is not built (run paper_2209_06478_b300.build): %s"
                          % LIB_PATH)
    lib = C.CDLL(LIB_PATH)
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    st = C.c_int
    sigs = {
        "dynmat_set_allocator": (st, [vp, vp, vp]),
        "dynmat_set_memory_limit": (st, [i64]),
        "dynmat_memory_in_use": (i64, []),
        "dynmat_set_pad_limit": (st, [dbl]),
        "dynmat_host_alloc": (st, [i64, C.POINTER(vp)]),
        "dynmat_host_free": (st, [vp]),
        "dynmat_create": (st, [C.POINTER(vp), i64, i64, i64, vp, vp, vp, C.c_int, C.c_int, vp]),
        "dynmat_destroy": (st, [vp, vp]),
        "dynmat_create_stencil": (st, [C.POINTER(vp), i64, i64, i64, i32, C.c_int, C.c_int, vp]),
        "dynmat_get_info": (st, [vp, C.POINTER(Info)]),
        "dynmat_copy_out": (st, [vp, C.c_int, vp, i64, C.c_int, vp]),
        "dynmat_convert": (st, [vp, C.c_int, C.c_int, vp]),
        "dynmat_features_get": (st, [vp, i32, C.POINTER(Features), vp]),
        "dynmat_select_format": (st, [vp, C.c_int, C.POINTER(C.c_int), vp]),
        "dynmat_autotune": (st, [vp, C.POINTER(C.c_int), C.POINTER(i32), vp]),
        "dynmat_tune_variant": (st, [vp, C.POINTER(i32), vp]),
        "dynmat_spmv": (st, [vp, vp, vp, C.c_int, vp]),
        "dynmat_spmv_host": (st, [vp, vp, vp, C.c_int, vp]),
        "dynmat_set_variant": (st, [vp, i32]),
        "dynmat_spmv_coo_noalloc": (st, [i64, i64, vp, vp, vp, vp, vp, vp]),
        "dynmat_spmv_acc": (st, [vp, vp, vp, C.c_int, vp]),
        "dynmat_diagonal": (st, [vp, vp, vp]),
        "dynmat_mg_create": (st, [C.POINTER(vp), i64, i64, i64, i32, i32, vp]),
        "dynmat_mg_destroy": (st, [vp, vp]),
        "dynmat_mg_level": (st, [vp, i32, C.POINTER(vp), vp]),
        "dynmat_mg_symgs": (st, [vp, i32, vp, vp, vp]),
        "dynmat_mg_apply": (st, [vp, vp, vp, vp]),
        "pcg_solve": (st, [vp, vp, vp, C.POINTER(CgOpts), C.POINTER(CgResult), vp]),
        "dynmat_set_diagonal": (st, [vp, vp, vp]),
        "dynmat_gather": (st, [vp, vp, i64, vp, C.c_int, vp]),
        "dynmat_split_spmv": (st, [vp, vp, vp, i64, vp, vp, vp, vp, C.c_int, vp]),
        "cg_solve": (st, [vp, vp, vp, C.POINTER(CgOpts), C.POINTER(CgResult), vp]),
        "dynmat_batch_create": (st, [C.POINTER(vp), i32, vp]),
        "dynmat_batch_destroy": (st, [vp, vp]),
        "dynmat_batch_set": (st, [vp, i32, vp, C.POINTER(TileShape), vp, vp, vp]),
        "dynmat_batch_spmv": (st, [vp, vp]),
        "dynmat_batch_autotune": (st, [vp, i32, C.POINTER(C.c_int), C.POINTER(TileShape), vp]),
        "dynmat_batch_tune_matrix": (st, [vp, i32, C.POINTER(C.c_int), C.POINTER(TileShape), vp]),
        "cg_batch_admit": (st, [vp, i32, vp, vp, vp, C.POINTER(CgOpts), C.POINTER(TileShape), vp]),
        "cg_batch_step": (st, [vp, i32, C.POINTER(i32), C.POINTER(i32), vp]),
        "cg_batch_result": (st, [vp, i32, C.POINTER(CgResult), vp]),
        "cg_batch_pause": (st, [vp, i32, i32, vp]),
        "cg_batch_retire": (st, [vp, i32, vp]),
        "dynmat_selftest_wait_timeout": (st, [i32, i64, C.POINTER(i32), vp]),
        "dynmat_last_error": (C.c_char_p, []),
        "dynmat_status_string": (C.c_char_p, [C.c_int]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def status_string(s: int) -> str:
    return lib.dynmat_status_string(s).decode()


def last_error() -> str:
    return (lib.dynmat_last_error() or b"").decode()


def _check(status):
    if status != OK:
        raise DynmatError(status, last_error())


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _ptr(a):
    """Address of a torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return C.c_void_p(a.ctypes.data)
    return C.c_void_p(a.data_ptr())


def _length(a):
    """Entries of a 1-D torch tensor or numpy array; None if unknown."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return int(a.size)
    numel = getattr(a, "numel", None)
    return int(numel()) if callable(numel) else None


def _on_device(a) -> int:
    return 0 if isinstance(a, np.ndarray) or not getattr(a, "is_cuda", False) else 1


def _vdtype(a) -> int:
    name = str(a.dtype)
    if name.endswith("float64"):
        return F64
    if name.endswith("float32"):
        return F32
    raise TypeError("values must be float64 or float32, got %s" % name)


# ---------------------------------------------------------------------------
# ABI calls (same names as include/dynmat.h)
# ---------------------------------------------------------------------------

def dynmat_set_memory_limit(nbytes: int):
    _check(lib.dynmat_set_memory_limit(int(nbytes)))


def dynmat_memory_in_use() -> int:
    return int(lib.dynmat_memory_in_use())


def dynmat_set_pad_limit(ratio: float):
    _check(lib.dynmat_set_pad_limit(float(ratio)))


class _HostBlock:
    """Owner of one dynmat_host_alloc block; numpy views keep it alive."""

    def __init__(self, shape, dtype):
        dt = np.dtype(dtype)
        nbytes = max(1, int(np.prod(shape)) * dt.itemsize)
        p = C.c_void_p()
        _check(lib.dynmat_host_alloc(nbytes, C.byref(p)))
        self.ptr = p.value
        self._free = lib.dynmat_host_free
        self.__array_interface__ = {"shape": tuple(shape), "typestr": dt.str,
                                    "data": (self.ptr, False), "version": 3}

    def __del__(self):
        if self.ptr:
            self._free(C.c_void_p(self.ptr))
            self.ptr = None


def dynmat_host_alloc(shape, dtype=np.float64) -> np.ndarray:
    """A zeroed numpy array in huge-page-backed, CUDA-registered host memory
    (for spmv_host); freed with dynmat_host_free when the array is collected."""
    if isinstance(shape, (int, np.integer)):
        shape = (int(shape),)
    return np.asarray(_HostBlock(shape, dtype))


def dynmat_create(nrows, ncols, row, col, val, stream=None) -> "DynMat":
    """row, col int32 and val float64/float32 — all host (numpy) or all device (torch)."""
    nnz = int(row.shape[0])
    if not (int(col.shape[0]) == nnz and int(val.shape[0]) == nnz):
        raise ValueError("row, col and val must have the same length")
    on_dev = _on_device(row)
    if not (on_dev == _on_device(col) == _on_device(val)):
        raise ValueError("row, col and val must all be on the host or all on the device")
    h = C.c_void_p()
    _check(lib.dynmat_create(C.byref(h), int(nrows), int(ncols), nnz, _ptr(row), _ptr(col),
                             _ptr(val), _vdtype(val), on_dev, _stream(stream)))
    return DynMat(h)


def dynmat_create_stencil(n, points=27, fmt=COO, vdtype=F64, ny=None, nz=None,
                          stream=None) -> "DynMat":
    """HPCG stencil matrix on an n x ny x nz grid, built on the device."""
    if isinstance(fmt, str):
        fmt = FORMATS.index(fmt)
    h = C.c_void_p()
    _check(lib.dynmat_create_stencil(C.byref(h), int(n), int(ny or n), int(nz or n), int(points),
                                     int(fmt), int(vdtype), _stream(stream)))
    return DynMat(h)


def dynmat_destroy(A: "DynMat", stream=None):
    A.destroy(stream)


def dynmat_convert(A: "DynMat", fmt: int, vdtype: int | None = None, stream=None):
    A.convert(fmt, vdtype, stream)


def dynmat_select_format(A: "DynMat", mode: int = SELECT_FEATURES, stream=None) -> int:
    return A.select_format(mode, stream)


def dynmat_spmv(A: "DynMat", x, y, stream=None):
    A.spmv(x, y, stream)


def cg_solve(A: "DynMat", b, x, **kw):
    return A.cg_solve(b, x, **kw)


NOALLOC_MAX_NNZ = 16777216


def dynmat_selftest_wait_timeout(which: int, cycles: int, stream=None) -> bool:
    """Runs a kernel whose bounded wait nothing can satisfy (0: grid barrier,
    1: mbarrier); True when the wait gave up after `cycles` and said so."""
    out = C.c_int32(0)
    _check(lib.dynmat_selftest_wait_timeout(int(which), int(cycles), C.byref(out),
                                            _stream(stream)))
    return bool(out.value)


def dynmat_gather(src, idx, dst, stream=None):
    """dst[k] = src[idx[k]] on the device (idx int32)."""
    _check(lib.dynmat_gather(_ptr(src), _ptr(idx), int(idx.shape[0]), _ptr(dst), _vdtype(src),
                             _stream(stream)))


def dynmat_split_spmv(A_loc, A_rem, halo, x_src, x_loc, x_ext, y, stream=None):
    """y = A_loc x_loc + A_rem x_src[halo] (x_ext: scratch of len(halo))."""
    n_ext = int(halo.shape[0]) if halo is not None else 0
    _check(lib.dynmat_split_spmv(A_loc.h, A_rem.h if A_rem is not None else None, _ptr(halo),
                                 n_ext, _ptr(x_src), _ptr(x_loc), _ptr(x_ext), _ptr(y),
                                 _vdtype(x_loc), _stream(stream)))


def _require_device(name, a, dtype):
    """A contiguous CUDA tensor of the given dtype ("int32" or "float64")."""
    if isinstance(a, np.ndarray) or not getattr(a, "is_cuda", False):
        raise DynmatError(ERR_INVALID_ARG, "%s must be a CUDA tensor" % name)
    if not str(a.dtype).endswith(dtype):
        raise DynmatError(ERR_INVALID_ARG, "%s must be %s, got %s" % (name, dtype, a.dtype))
    contiguous = getattr(a, "is_contiguous", None)
    if callable(contiguous) and not contiguous():
        raise DynmatError(ERR_INVALID_ARG, "%s must be contiguous" % name)


def dynmat_spmv_coo_noalloc(nrows, row, col, val, x, y, stream=None):
    """COO product with no device allocation (canonical FP64 COO on the
    device; see include/dynmat.h for the limits and the shared work array).

    The C call takes raw device pointers and no column count, so this
    wrapper refuses, before anything runs, what would make a kernel read or
    write past an array or misread its type: host arrays, wrong dtypes,
    non-contiguous tensors, col or val not as long as row, y shorter than
    nrows. The column indices themselves must lie within x (the caller's
    contract, as for every canonical COO)."""
    for name, a, dt in (("row", row, "int32"), ("col", col, "int32"), ("val", val, "float64"),
                        ("x", x, "float64"), ("y", y, "float64")):
        _require_device(name, a, dt)
    nnz = _length(row)
    if _length(col) != nnz or _length(val) != nnz:
        raise DynmatError(ERR_INVALID_ARG, "row, col and val must have the same length "
                          "(%d, %d, %d)" % (nnz, _length(col), _length(val)))
    if _length(y) < int(nrows):
        raise DynmatError(ERR_INVALID_ARG, "y has %d entries, nrows is %d" % (_length(y), nrows))
    _check(lib.dynmat_spmv_coo_noalloc(int(nrows), nnz, _ptr(row), _ptr(col), _ptr(val),
                                       _ptr(x), _ptr(y), _stream(stream)))


class DynMat:
    """Owner of a dynmat_t handle (or, with owner set, a borrowed one that
    the owner object frees)."""

    def __init__(self, handle: C.c_void_p, owner=None):
        self.h = handle
        self.owner = owner
        self._shape = None  # (nrows, ncols): fixed for the handle's life

    @property
    def shape(self):
        if self._shape is None:
            i = self.info()
            self._shape = (int(i.nrows), int(i.ncols))
        return self._shape

    def _check_vectors(self, x, y):
        """The C ABI takes raw pointers: refuse vectors shorter than the
        matrix before any kernel can run past their end."""
        n, m = self.shape
        nx, ny = _length(x), _length(y)
        if nx is not None and nx < m:
            raise DynmatError(ERR_INVALID_ARG, "x has %d entries, the matrix %d columns" % (nx, m))
        if ny is not None and ny < n:
            raise DynmatError(ERR_INVALID_ARG, "y has %d entries, the matrix %d rows" % (ny, n))

    def _check_diag(self, d):
        k, nd = min(self.shape), _length(d)
        if nd is not None and nd < k:
            raise DynmatError(ERR_INVALID_ARG, "the diagonal has %d entries, not %d" % (nd, k))

    def __del__(self):
        try:
            if self.h and self.owner is None:
                lib.dynmat_destroy(self.h, None)
                self.h = None
        except Exception:
            pass

    def destroy(self, stream=None):
        if self.owner is not None:
            raise DynmatError(ERR_INVALID_ARG, "a borrowed handle is freed by its owner")
        if self.h:
            _check(lib.dynmat_destroy(self.h, _stream(stream)))
            self.h = None

    def info(self) -> Info:
        o = Info()
        _check(lib.dynmat_get_info(self.h, C.byref(o)))
        return o

    @property
    def format(self) -> int:
        return self.info().format

    def convert(self, fmt: int, vdtype: int | None = None, stream=None):
        if isinstance(fmt, str):
            fmt = FORMATS.index(fmt)
        if vdtype is None:
            vdtype = self.info().vdtype
        _check(lib.dynmat_convert(self.h, int(fmt), int(vdtype), _stream(stream)))
        return self

    def features(self, guard: int = 3, stream=None) -> dict:
        f = Features()
        _check(lib.dynmat_features_get(self.h, int(guard), C.byref(f), _stream(stream)))
        return {"nrows": f.nrows, "ncols": f.ncols, "nnz": f.nnz, "ndiag": f.ndiag,
                "maxlen": f.maxlen, "hyb_k": f.hyb_k, "hyb_over": f.hyb_over,
                "bytes": list(f.bytes), "choice": f.choice}

    def select_format(self, mode: int = SELECT_FEATURES, stream=None) -> int:
        out = C.c_int(-1)
        _check(lib.dynmat_select_format(self.h, int(mode), C.byref(out), _stream(stream)))
        return out.value

    def autotune(self, stream=None):
        f, v = C.c_int(-1), C.c_int32(0)
        _check(lib.dynmat_autotune(self.h, C.byref(f), C.byref(v), _stream(stream)))
        return f.value, v.value

    def tune_variant(self, stream=None) -> int:
        v = C.c_int32(0)
        _check(lib.dynmat_tune_variant(self.h, C.byref(v), _stream(stream)))
        return v.value

    def set_variant(self, variant: int):
        _check(lib.dynmat_set_variant(self.h, int(variant)))

    def spmv(self, x, y, stream=None):
        self._check_vectors(x, y)
        _check(lib.dynmat_spmv(self.h, _ptr(x), _ptr(y), _vdtype(x), _stream(stream)))

    def diagonal(self, d, stream=None):
        """d[i] = a(i, i) (device tensor of the value type, min(nrows, ncols))."""
        self._check_diag(d)
        _check(lib.dynmat_diagonal(self.h, _ptr(d), _stream(stream)))

    def set_diagonal(self, d, stream=None):
        """Every stored (i, i) entry := d[i]."""
        self._check_diag(d)
        _check(lib.dynmat_set_diagonal(self.h, _ptr(d), _stream(stream)))

    def batch_tune(self, effort: int = 0, stream=None):
        """Converts to the format fastest in the batch kernel; returns
        (format, (lanes, rows_per_tile, nnz_per_tile))."""
        f, s = C.c_int(-1), TileShape()
        _check(lib.dynmat_batch_tune_matrix(self.h, int(effort), C.byref(f), C.byref(s),
                                            _stream(stream)))
        return f.value, (s.lanes, s.rows_per_tile, s.nnz_per_tile)

    def spmv_acc(self, x, y, stream=None):
        """y += A x."""
        self._check_vectors(x, y)
        _check(lib.dynmat_spmv_acc(self.h, _ptr(x), _ptr(y), _vdtype(x), _stream(stream)))

    def spmv_host(self, x: np.ndarray, y: np.ndarray, stream=None):
        self._check_vectors(x, y)
        _check(lib.dynmat_spmv_host(self.h, _ptr(x), _ptr(y), _vdtype(x), _stream(stream)))

    def copy_out(self, which: int, count: int, dtype, stream=None) -> np.ndarray:
        out = np.empty(count, dtype=dtype)
        _check(lib.dynmat_copy_out(self.h, int(which), _ptr(out), out.nbytes, 0,
                                   _stream(stream)))
        return out

    def arrays(self, stream=None) -> dict:
        """The active format's arrays copied to the host (numpy), unpadded:
        DIA values as (ndiag, nrows), ELL arrays as (K, nrows)."""
        i = self.info()
        vdt = np.float64 if i.vdtype == F64 else np.float32
        N = i.nrows
        f = FORMATS[i.format]
        if f == "coo":
            return {"row": self.copy_out(ARR_ROW, i.nnz, np.int32, stream),
                    "col": self.copy_out(ARR_COL, i.nnz, np.int32, stream),
                    "val": self.copy_out(ARR_VAL, i.nnz, vdt, stream)}
        if f == "csr":
            return {"rowptr": self.copy_out(ARR_ROWPTR, N + 1, np.int32, stream),
                    "col": self.copy_out(ARR_COL, i.nnz, np.int32, stream),
                    "val": self.copy_out(ARR_VAL, i.nnz, vdt, stream)}
        if f == "dia":
            v = self.copy_out(ARR_VAL, i.ndiag * i.ld, vdt, stream).reshape(i.ndiag, i.ld)
            return {"offsets": self.copy_out(ARR_OFFSETS, i.ndiag, np.int32, stream),
                    "val": np.ascontiguousarray(v[:, :N]), "ld": i.ld}
        K = i.ell_width
        c = self.copy_out(ARR_COL, K * i.ld, np.int32, stream).reshape(K, i.ld)
        v = self.copy_out(ARR_VAL, K * i.ld, vdt, stream).reshape(K, i.ld)
        out = {"col": np.ascontiguousarray(c[:, :N]), "val": np.ascontiguousarray(v[:, :N]),
               "ld": i.ld}
        if f == "hyb":
            m = i.hyb_coo_nnz
            return {"ell_col": out["col"], "ell_val": out["val"], "ld": i.ld,
                    "coo_row": self.copy_out(ARR_ROW, m, np.int32, stream),
                    "coo_col": self.copy_out(ARR_HYB_COL, m, np.int32, stream),
                    "coo_val": self.copy_out(ARR_HYB_VAL, m, vdt, stream)}
        return out

    def cg_solve(self, b, x, tol=1e-9, max_iters=1000, precision=CG_FP64, inner_tol=1e-5,
                 max_outer=30, check_every=25, delta=0.1, stream=None) -> dict:
        self._check_vectors(x, b)  # b: one entry per row, x: one per column
        o = CgOpts(tol, max_iters, precision, inner_tol, max_outer, check_every, delta)
        r = CgResult()
        _check(lib.cg_solve(self.h, _ptr(b), _ptr(x), C.byref(o), C.byref(r), _stream(stream)))
        return {"status": r.status, "iterations": r.iterations,
                "outer_iterations": r.outer_iterations, "rel_residual": r.rel_residual,
                "true_rel_residual": r.true_rel_residual}


class DynMG:
    """Owner of a dynmat_mg_t: HPCG's multigrid hierarchy (stencil levels)."""

    def __init__(self, nx, ny=None, nz=None, points=27, levels=4, stream=None):
        ny = nx if ny is None else ny
        nz = nx if nz is None else nz
        h = C.c_void_p()
        _check(lib.dynmat_mg_create(C.byref(h), int(nx), int(ny), int(nz), int(points),
                                    int(levels), _stream(stream)))
        self.h = h
        self.levels = int(levels)

    def __del__(self):
        try:
            if self.h:
                lib.dynmat_mg_destroy(self.h, None)
                self.h = None
        except Exception:
            pass

    def level(self, l: int):
        """(borrowed DynMat of level l, its grid dims)."""
        a = C.c_void_p()
        dims = (C.c_int64 * 3)()
        _check(lib.dynmat_mg_level(self.h, int(l), C.byref(a), dims))
        return DynMat(a, owner=self), (dims[0], dims[1], dims[2])

    def symgs(self, level: int, r, z, stream=None):
        _check(lib.dynmat_mg_symgs(self.h, int(level), _ptr(r), _ptr(z), _stream(stream)))

    def apply(self, r, z, stream=None):
        """z = M^{-1} r (one V-cycle)."""
        _check(lib.dynmat_mg_apply(self.h, _ptr(r), _ptr(z), _stream(stream)))

    def pcg_solve(self, b, x, tol=1e-9, max_iters=1000, check_every=25, stream=None) -> dict:
        o = CgOpts(tol, max_iters, CG_FP64, 1e-5, 30, check_every, 0.1)
        r = CgResult()
        _check(lib.pcg_solve(self.h, _ptr(b), _ptr(x), C.byref(o), C.byref(r), _stream(stream)))
        return {"status": r.status, "iterations": r.iterations, "rel_residual": r.rel_residual,
                "true_rel_residual": r.true_rel_residual}


class DynBatch:
    """Owner of a dynmat_batch_t: many matrices per persistent launch."""

    def __init__(self, max_slots: int, stream=None):
        h = C.c_void_p()
        _check(lib.dynmat_batch_create(C.byref(h), int(max_slots), _stream(stream)))
        self.h = h
        self.max_slots = int(max_slots)
        self._keep = {}  # slot -> objects the device descriptors point at

    def __del__(self):
        try:
            if self.h:
                lib.dynmat_batch_destroy(self.h, None)
                self.h = None
        except Exception:
            pass

    def destroy(self, stream=None):
        if self.h:
            _check(lib.dynmat_batch_destroy(self.h, _stream(stream)))
            self.h = None

    @staticmethod
    def _shape(shape):
        if shape is None:
            return None
        if isinstance(shape, TileShape):
            return C.byref(shape)
        return C.byref(TileShape(*shape))

    def set(self, slot: int, A, x=None, y=None, shape=None, stream=None):
        _check(lib.dynmat_batch_set(self.h, int(slot), A.h if A is not None else None,
                                    self._shape(shape), _ptr(x), _ptr(y), _stream(stream)))
        self._keep[slot] = (A, x, y)

    def spmv(self, stream=None):
        _check(lib.dynmat_batch_spmv(self.h, _stream(stream)))

    def autotune(self, slot: int, stream=None):
        f, s = C.c_int(-1), TileShape()
        _check(lib.dynmat_batch_autotune(self.h, int(slot), C.byref(f), C.byref(s),
                                         _stream(stream)))
        return f.value, (s.lanes, s.rows_per_tile, s.nnz_per_tile)

    def cg_admit(self, slot: int, A, b, x, tol=1e-10, max_iters=1000, precision=CG_FP64,
                 inner_tol=1e-5, max_outer=30, shape=None, stream=None):
        o = CgOpts(tol, max_iters, precision, inner_tol, max_outer, 0, 0.1)
        _check(lib.cg_batch_admit(self.h, int(slot), A.h, _ptr(b), _ptr(x), C.byref(o),
                                  self._shape(shape), _stream(stream)))
        self._keep[slot] = (A, b, x)

    def cg_step(self, iterations: int = 8, stream=None):
        flags = (C.c_int32 * self.max_slots)()
        active = C.c_int32(0)
        _check(lib.cg_batch_step(self.h, int(iterations), flags, C.byref(active),
                                 _stream(stream)))
        return [k for k in range(self.max_slots) if flags[k]], active.value

    def cg_pause(self, slot: int, paused: bool = True, stream=None):
        """Leaves a running CG slot out of the following cg_step calls, or
        takes it back; its iterates are the same bits, only later."""
        _check(lib.cg_batch_pause(self.h, int(slot), 1 if paused else 0, _stream(stream)))

    def cg_result(self, slot: int, stream=None) -> dict:
        r = CgResult()
        _check(lib.cg_batch_result(self.h, int(slot), C.byref(r), _stream(stream)))
        return {"status": r.status, "iterations": r.iterations,
                "outer_iterations": r.outer_iterations, "rel_residual": r.rel_residual,
                "true_rel_residual": r.true_rel_residual}

    def cg_retire(self, slot: int, stream=None):
        _check(lib.cg_batch_retire(self.h, int(slot), _stream(stream)))
        self._keep.pop(slot, None)
