"""The C-ABI library on a machine without a GPU: it loads, exports every
function that include/dynmat.h declares, and the binding's ctypes structs have
the header's layout. No compute calls are made here."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


@pytest.fixture(scope="module")
def built():
    from paper_2209_06478_b300 import build
    return build.build()


def declared_functions():
    names = []
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        # a declaration: <type> name(<args>);  (typedefs of function pointers excluded)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b([a-z_][a-z0-9_]*)\s*\([^;{]*\)\s*;", text, re.M):
            line = m.group(0)
            if line.lstrip().startswith("typedef"):
                continue
            names.append(m.group(1))
    return sorted(set(names))


def test_header_declares_the_abi():
    names = declared_functions()
    for must in ("dynmat_create", "dynmat_convert", "dynmat_select_format", "dynmat_spmv",
                 "cg_solve", "dynmat_destroy", "dynmat_get_info", "dynmat_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(built):
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True,
                         check=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_library_loads_and_binds(built):
    from paper_2209_06478_b300 import dynmat as dm
    lib = C.CDLL(built)
    for n in declared_functions():
        assert hasattr(lib, n)
    assert dm.status_string(dm.OK) == "ok"
    assert dm.status_string(dm.ERR_DUPLICATE) == "duplicate entry"
    # host-only argument checks
    with pytest.raises(dm.DynmatError) as e:
        dm.dynmat_set_memory_limit(-1)
    assert e.value.status == dm.ERR_INVALID_ARG
    with pytest.raises(dm.DynmatError):
        dm.dynmat_set_pad_limit(0.0)
    dm.dynmat_set_memory_limit(0)
    dm.dynmat_set_pad_limit(16.0)
    assert dm.dynmat_memory_in_use() == 0


def test_host_alloc_argument_checks(built):
    """The host allocator's checks that come before any CUDA call."""
    from paper_2209_06478_b300 import dynmat as dm
    p = C.c_void_p()
    assert dm.lib.dynmat_host_alloc(0, C.byref(p)) == dm.ERR_INVALID_ARG
    assert dm.lib.dynmat_host_alloc(-8, C.byref(p)) == dm.ERR_INVALID_ARG
    assert dm.lib.dynmat_host_alloc(64, None) == dm.ERR_INVALID_ARG
    assert dm.lib.dynmat_host_free(None) == dm.OK
    junk = (C.c_char * 64)()
    assert dm.lib.dynmat_host_free(C.cast(junk, C.c_void_p)) == dm.ERR_INVALID_ARG
    assert "dynmat_host_alloc" in dm.last_error()


def test_binding_refuses_short_vectors(built):
    """The binding checks vector lengths against the matrix shape before the
    call reaches the library (raw pointers carry no size)."""
    from paper_2209_06478_b300 import dynmat as dm

    class Fake(dm.DynMat):
        def __init__(self):
            super().__init__(C.c_void_p(None))
            self._shape = (5, 3)

    A = Fake()
    for x, y in ((np.zeros(2), np.zeros(5)), (np.zeros(3), np.zeros(4))):
        with pytest.raises(dm.DynmatError) as e:
            A.spmv_host(x, y)
        assert e.value.status == dm.ERR_INVALID_ARG
    with pytest.raises(dm.DynmatError):
        A.diagonal(np.zeros(2))     # min(5, 3) = 3 entries needed
    with pytest.raises(dm.DynmatError):
        A.cg_solve(np.zeros(4), np.zeros(3))  # b needs one entry per row
    A.h = None  # nothing to destroy


class _FakeDeviceTensor:
    """Stands in for a CUDA tensor on a machine without a GPU. Its address
    is never taken: a wrapper that got as far as the C call would fail the
    test with AssertionError instead of DynmatError."""

    def __init__(self, n, dtype, cuda=True, contiguous=True):
        self.n, self.dtype, self.is_cuda, self._contig = n, "torch." + dtype, cuda, contiguous

    def numel(self):
        return self.n

    def is_contiguous(self):
        return self._contig

    def data_ptr(self):
        raise AssertionError("the wrapper passed a pointer to the library")


def test_noalloc_binding_refuses_bad_arguments_before_any_call(built):
    """dynmat_spmv_coo_noalloc takes raw pointers and no column count: the
    binding must refuse host arrays, wrong dtypes, non-contiguous tensors,
    col/val lengths that differ from row's and a y shorter than nrows, each
    before the library is called."""
    from paper_2209_06478_b300 import dynmat as dm
    T = _FakeDeviceTensor

    def args(**over):
        a = {"row": T(8, "int32"), "col": T(8, "int32"), "val": T(8, "float64"),
             "x": T(6, "float64"), "y": T(6, "float64")}
        a.update(over)
        return a

    bad = [
        args(row=np.zeros(8, np.int32)),                 # host array
        args(x=T(6, "float64", cuda=False)),             # CPU tensor
        args(row=T(8, "int64")),                         # int64 indices
        args(col=T(8, "int64")),
        args(val=T(8, "float32")),                       # FP32 values
        args(x=T(6, "float32")),
        args(y=T(6, "float32")),
        args(col=T(7, "int32")),                         # col shorter than row
        args(val=T(9, "float64")),                       # val longer than row
        args(y=T(5, "float64")),                         # y shorter than nrows
        args(val=T(8, "float64", contiguous=False)),     # strided view
    ]
    for a in bad:
        with pytest.raises(dm.DynmatError) as e:
            dm.dynmat_spmv_coo_noalloc(6, a["row"], a["col"], a["val"], a["x"], a["y"], stream=0)
        assert e.value.status == dm.ERR_INVALID_ARG
    # the same arguments, all valid, reach the C call (the fake refuses to be addressed)
    a = args()
    with pytest.raises(AssertionError):
        dm.dynmat_spmv_coo_noalloc(6, a["row"], a["col"], a["val"], a["x"], a["y"], stream=0)


def test_struct_layouts_match_header(tmp_path):
    from paper_2209_06478_b300 import dynmat as dm
    src = tmp_path / "layout.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "dynmat.h"
int main(void) {
  printf("%zu %zu %zu %zu\\n", sizeof(dynmat_info), sizeof(dynmat_features), sizeof(cg_opts), sizeof(cg_result));
  printf("%zu %zu %zu\\n", offsetof(dynmat_info, bytes), offsetof(dynmat_features, choice), offsetof(cg_result, true_rel_residual));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    a, b = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")[:2]
    sizes = [int(v) for v in a.split()]
    offs = [int(v) for v in b.split()]
    assert sizes == [C.sizeof(dm.Info), C.sizeof(dm.Features), C.sizeof(dm.CgOpts), C.sizeof(dm.CgResult)]
    assert offs == [dm.Info.bytes.offset, dm.Features.choice.offset, dm.CgResult.true_rel_residual.offset]
