"""Local / remote split on the GPU (§IV-B, §V-E): each rank's
y = A_loc x_loc + A_rem x[halo] through dynmat_split_spmv, with the two parts
in independent formats, equals the oracle's product of the whole (rank-major)
matrix within 1e-13 * sum|a x| per row; y += A x alone; shape checks; and the
paper's observation that the unsplit local system matrix cannot go to DIA
while its local part can."""
import numpy as np
import pytest

import synth
from test_split_cpu import assembled

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2209_06478_b300 import build
    build.build()
    from paper_2209_06478_b300 import dynmat
    return dynmat, torch


def whole_product(orc, n, procs, x):
    gr, gc, gv = assembled(n, procs)
    N = n[0] * n[1] * n[2]
    st, r2, c2, v2 = orc.canonical(N, N, gr.astype(np.int32), gc.astype(np.int32), gv)
    want = orc.spmv("coo", N, N, {"row": r2, "col": c2, "val": v2}, x)
    bound = orc.spmv("coo", N, N, {"row": r2, "col": c2, "val": np.abs(v2)}, np.abs(x))
    return want, bound


@pytest.mark.parametrize("loc_fmt,rem_fmt", [("dia", "coo"), ("dia", "csr"), ("csr", "coo"),
                                             ("csr", "hyb"), ("ell", "csr")])
def test_split_spmv_matches_whole_product(env, orc, loc_fmt, rem_fmt):
    dm, torch = env
    n, procs = (16, 12, 10), (2, 3, 2)
    N = n[0] * n[1] * n[2]
    xh = synth.uniform_pm1(77, N)
    want, bound = whole_product(orc, n, procs, xh)
    x = torch.from_numpy(xh).cuda()
    for r in range(procs[0] * procs[1] * procs[2]):
        part = synth.partition_stencil(n, procs, r)
        nl, off, h = part["nloc"], part["offset"], part["halo"]
        Al = dm.dynmat_create(nl, nl, *part["local"])
        Al.convert(loc_fmt)
        Ar = dm.dynmat_create(nl, h.size, *part["remote"])
        Ar.convert(rem_fmt)
        halo = torch.from_numpy(h).cuda()
        x_ext = torch.empty(h.size, dtype=torch.float64, device="cuda")
        y = torch.full((nl,), float("nan"), dtype=torch.float64, device="cuda")
        dm.dynmat_split_spmv(Al, Ar, halo, x, x[off:off + nl], x_ext, y)
        torch.cuda.synchronize()
        sl = slice(off, off + nl)
        assert np.all(np.abs(y.cpu().numpy() - want[sl]) <= 1e-13 * bound[sl]), r
        assert np.array_equal(x_ext.cpu().numpy(), xh[h])  # the halo exchange


def test_spmv_acc_adds_the_product(env, orc):
    dm, torch = env
    N, r, c, v = synth.powerlaw(5, 3000)
    st, r2, c2, v2 = orc.canonical(N, N, r, c, v)
    xh = synth.uniform_pm1(6, N)
    y0 = synth.uniform_pm1(7, N)
    prod = orc.spmv("coo", N, N, {"row": r2, "col": c2, "val": v2}, xh)
    bound = orc.spmv("coo", N, N, {"row": r2, "col": c2, "val": np.abs(v2)}, np.abs(xh))
    for fmt in ("coo", "csr", "hyb"):
        A = dm.dynmat_create(N, N, r, c, v)
        A.convert(fmt)
        y = torch.from_numpy(y0.copy()).cuda()
        A.spmv_acc(torch.from_numpy(xh).cuda(), y)
        got = y.cpu().numpy()
        assert np.all(np.abs(got - (y0 + prod)) <= 1e-13 * bound + 2.0 ** -52 * np.abs(y0 + prod)), fmt


def test_single_rank_has_no_remote_part(env, orc):
    dm, torch = env
    n, procs = (8, 8, 8), (1, 1, 1)
    part = synth.partition_stencil(n, procs, 0)
    assert part["halo"].size == 0
    nl = part["nloc"]
    xh = synth.uniform_pm1(9, nl)
    want, bound = whole_product(orc, n, procs, xh)
    Al = dm.dynmat_create(nl, nl, *part["local"])
    Al.convert("dia")
    x = torch.from_numpy(xh).cuda()
    y = torch.empty(nl, dtype=torch.float64, device="cuda")
    dm.dynmat_split_spmv(Al, None, None, None, x, None, y)
    assert np.all(np.abs(y.cpu().numpy() - want) <= 1e-13 * bound)


def test_shape_mismatch_is_refused(env):
    dm, torch = env
    part = synth.partition_stencil((8, 8, 8), (2, 1, 1), 0)
    nl, h = part["nloc"], part["halo"]
    Al = dm.dynmat_create(nl, nl, *part["local"])
    Ar = dm.dynmat_create(nl, h.size, *part["remote"])
    x = torch.zeros(2 * nl, dtype=torch.float64, device="cuda")
    y = torch.zeros(nl, dtype=torch.float64, device="cuda")
    halo = torch.from_numpy(h).cuda()
    short = halo[:-1]  # n_ext one less than the remote part's columns
    x_ext = torch.zeros(h.size, dtype=torch.float64, device="cuda")
    with pytest.raises(dm.DynmatError):
        dm.dynmat_split_spmv(Al, Ar, short, x, x[:nl], x_ext, y)
    with pytest.raises(dm.DynmatError):
        dm.dynmat_split_spmv(Ar, None, None, None, x[:nl], None, y)  # not square


def test_unsplit_local_system_matrix_is_too_padded_for_dia(env):
    """§IV-B: with remote columns appended (HPCG's local numbering), the
    local system matrix is rectangular and irregular; DIA would pad it past
    the guard, while the square local part converts."""
    dm, torch = env
    n, procs = (32, 32, 32), (2, 2, 2)
    part = synth.partition_stencil(n, procs, 0)
    nl, h = part["nloc"], part["halo"]
    lr, lc, lv = part["local"]
    rr, rc, rv = part["remote"]
    rows = np.concatenate([lr, rr])
    cols = np.concatenate([lc, rc + nl]).astype(np.int32)
    vals = np.concatenate([lv, rv])
    whole = dm.dynmat_create(nl, nl + h.size, rows, cols, vals)
    with pytest.raises(dm.DynmatError) as e:
        whole.convert("dia")
    assert e.value.status == dm.ERR_FORMAT_TOO_LARGE
    local = dm.dynmat_create(nl, nl, lr, lc, lv)
    local.convert("dia")
    assert local.info().ndiag == 27
