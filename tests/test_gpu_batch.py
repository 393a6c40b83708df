"""Batched persistent launches: results of every slot must equal the
per-matrix path (SpMV within 1e-13 * sum|a x|, the oracle for one slot), the
tuner must keep results correct, and a CG slot's iterates must be
bit-identical alone and in a mixed batch."""
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


def mats():
    out = []
    out.append(("banded", *synth.banded(100, 17110, 33)))
    out.append(("powerlaw", *synth.powerlaw(101, 24384)))
    out.append(("uniform", *synth.uniform(102, 13016)))
    N, r, c, v = synth.stencil27(20)
    out.append(("stencil", N, r, c, v))
    out.append(("banded_odd", *synth.banded(103, 9999, 7)))
    return out


MATS = mats()


def per_matrix(dm, torch, A, x):
    y = torch.empty(A.info().nrows, dtype=x.dtype, device="cuda")
    A.spmv(x, y)
    return y


def test_batch_spmv_matches_per_matrix(env, orc):
    dm, torch = env
    fmts = ["dia", "csr", "csr", "csr", "ell"]
    shapes = [(8, 1024, 4096), (2, 2048, 1024), (8, 2048, 300), (8, 1024, 4096), (4, 3072, 512)]
    B = dm.DynBatch(8)
    keep = []
    for k, ((name, N, r, c, v), f, sh) in enumerate(zip(MATS, fmts, shapes)):
        A = dm.dynmat_create(N, N, r, c, v)
        A.convert(f)
        x = torch.from_numpy(synth.uniform_pm1(10 + k, N)).cuda()
        y = torch.full((N,), float("nan"), dtype=torch.float64, device="cuda")
        B.set(k, A, x, y, shape=sh)
        keep.append((name, A, x, y, r, c, v, N))
    for rep in range(3):  # first call builds, later calls replay the graph
        B.spmv()
        torch.cuda.synchronize()
        for name, A, x, y, r, c, v, N in keep:
            ref = per_matrix(dm, torch, A, x).cpu().numpy()
            st, r2, c2, v2 = orc.canonical(N, N, r, c, v)
            a = orc.to_format("csr", N, N, r2, c2, v2)
            bound = orc.spmv("csr", N, N, {"rowptr": a["rowptr"], "col": c2, "val": np.abs(v2)},
                             np.abs(x.cpu().numpy()))
            got = y.cpu().numpy()
            assert np.all(np.abs(got - ref) <= 1e-13 * bound), (name, rep)
    # oracle check of one slot
    name, A, x, y, r, c, v, N = keep[1]
    st, r2, c2, v2 = orc.canonical(N, N, r, c, v)
    want = orc.spmv("csr", N, N, orc.to_format("csr", N, N, r2, c2, v2), x.cpu().numpy())
    bound = orc.spmv("csr", N, N, {"rowptr": orc.coo_to_csr(N, r2), "col": c2, "val": np.abs(v2)},
                     np.abs(x.cpu().numpy()))
    assert np.all(np.abs(y.cpu().numpy() - want) <= 1e-13 * bound)


def test_batch_spmv_f32_and_slot_changes(env):
    dm, torch = env
    B = dm.DynBatch(4)
    name, N, r, c, v = MATS[0]
    A = dm.dynmat_create(N, N, r, c, v)
    A.convert("dia", dm.F32)
    x = torch.from_numpy(synth.uniform_pm1(3, N).astype(np.float32)).cuda()
    y = torch.empty(N, dtype=torch.float32, device="cuda")
    B.set(2, A, x, y)
    B.spmv()
    ref = per_matrix(dm, torch, A, x)
    torch.cuda.synchronize()
    assert torch.allclose(y, ref, rtol=1e-5, atol=1e-5)
    # add a slot after the graph exists, then remove one
    name2, N2, r2, c2, v2 = MATS[2]
    A2 = dm.dynmat_create(N2, N2, r2, c2, v2)
    A2.convert("csr")
    x2 = torch.from_numpy(synth.uniform_pm1(4, N2)).cuda()
    y2 = torch.empty(N2, dtype=torch.float64, device="cuda")
    B.set(0, A2, x2, y2)
    B.spmv()
    torch.cuda.synchronize()
    assert torch.allclose(y2, per_matrix(dm, torch, A2, x2), rtol=1e-13, atol=1e-13)
    B.set(2, None)
    y2.fill_(0)
    B.spmv()
    torch.cuda.synchronize()
    assert torch.allclose(y2, per_matrix(dm, torch, A2, x2), rtol=1e-13, atol=1e-13)


def test_batch_autotune_keeps_results(env, orc):
    dm, torch = env
    B = dm.DynBatch(3)
    keep = []
    for k, (name, N, r, c, v) in enumerate(MATS[:3]):
        A = dm.dynmat_create(N, N, r, c, v)
        A.convert("csr")
        x = torch.from_numpy(synth.uniform_pm1(20 + k, N)).cuda()
        y = torch.empty(N, dtype=torch.float64, device="cuda")
        B.set(k, A, x, y)
        fmt, shape = B.autotune(k)
        assert fmt in (dm.DIA, dm.ELL, dm.CSR) and A.info().format == fmt
        keep.append((A, x, y, N, r, c, v))
    B.spmv()
    torch.cuda.synchronize()
    for A, x, y, N, r, c, v in keep:
        st, r2, c2, v2 = orc.canonical(N, N, r, c, v)
        want = orc.spmv("csr", N, N, orc.to_format("csr", N, N, r2, c2, v2), x.cpu().numpy())
        bound = orc.spmv("csr", N, N, {"rowptr": orc.coo_to_csr(N, r2), "col": c2,
                                       "val": np.abs(v2)}, np.abs(x.cpu().numpy()))
        assert np.all(np.abs(y.cpu().numpy() - want) <= 1e-13 * bound)


def spd(k):
    kinds = [("banded", 30000, 21), ("powerlaw", 20000, 0), ("uniform", 25000, 0)]
    kind, n, extra = kinds[k % 3]
    return synth.make(kind, 500 + k, n, extra, spd=True)


def run_batch_cg(dm, torch, problems, slots, precision, tol=1e-10):
    B = dm.DynBatch(max(slots) + 1)
    xs = {}
    for s, (A, b) in zip(slots, problems):
        x = torch.zeros_like(b)
        B.cg_admit(s, A, b, x, tol=tol, max_iters=2000, precision=precision)
        xs[s] = x
    for _ in range(2000):
        done, active = B.cg_step(8)
        if active == 0:
            break
    res = {s: B.cg_result(s) for s in slots}
    return res, {s: xs[s].cpu().numpy() for s in slots}


def test_batch_cg_fp64_matches_solo_and_is_mix_invariant(env, orc):
    dm, torch = env
    probs = []
    mats_ = []
    for k in range(4):
        N, r, c, v = spd(k)
        A = dm.dynmat_create(N, N, r, c, v)
        A.convert(["dia", "csr", "csr", "ell"][k])
        b = torch.from_numpy(synth.uniform_pm1(40 + k, N)).cuda()
        probs.append((A, b))
        mats_.append((N, r, c, v))
    res, xs = run_batch_cg(dm, torch, probs, [0, 1, 2, 3], dm.CG_FP64)
    for k, (A, b) in enumerate(probs):
        assert res[k]["status"] == dm.OK, (k, res[k])
        assert res[k]["true_rel_residual"] <= 2e-10
        # the oracle: its FP64 product recomputes the true residual of the
        # returned x, and its CG reaches the same tolerance in about as many
        # iterations with about the same x
        N, r, c, v = mats_[k]
        st, r2, c2, v2 = orc.canonical(N, N, r, c, v)
        a = {"rowptr": orc.coo_to_csr(N, r2), "col": c2, "val": v2}
        b_np = b.cpu().numpy()
        true = np.linalg.norm(b_np - orc.spmv("csr", N, N, a, xs[k])) / np.linalg.norm(b_np)
        assert true <= 2e-10 and abs(true - res[k]["true_rel_residual"]) <= 1e-3 * true + 1e-15
        ref = orc.cg(N, a["rowptr"], c2, v2, b_np, tol=1e-10, max_iters=2000)
        assert abs(ref["iterations"] - res[k]["iterations"]) <= max(2, 0.02 * ref["iterations"])
        assert np.linalg.norm(xs[k] - ref["x"]) <= 1e-7 * np.linalg.norm(ref["x"])
        # solo per-matrix path
        xs_solo = torch.zeros_like(b)
        solo = A.cg_solve(b, xs_solo, tol=1e-10, max_iters=2000)
        assert abs(solo["iterations"] - res[k]["iterations"]) <= 2
        xs_solo = xs_solo.cpu().numpy()
        assert np.linalg.norm(xs[k] - xs_solo) <= 1e-7 * np.linalg.norm(xs_solo)
    # slot 2's problem alone in a batch: bit-identical iterates
    res1, xs1 = run_batch_cg(dm, torch, [probs[2]], [5], dm.CG_FP64)
    assert res1[5]["iterations"] == res[2]["iterations"]
    assert np.array_equal(xs1[5].view(np.uint64), xs[2].view(np.uint64))


@pytest.mark.parametrize("prec", ["mixed", "reliable"])
def test_batch_cg_mixed_reaches_1e10(env, orc, prec):
    dm, torch = env
    precision = dm.CG_MIXED if prec == "mixed" else dm.CG_MIXED_RELIABLE
    probs = []
    refs = []
    for n in (16, 24):
        N, r, c, v = synth.stencil27(n)
        A = dm.dynmat_create(N, N, r, c, v)
        A.convert("dia", dm.F32)
        rp = orc.coo_to_csr(N, r)
        b_np = synth.uniform_pm1(n, N)
        probs.append((A, torch.from_numpy(b_np).cuda()))
        refs.append((N, rp, c, v, b_np))
    N, r, c, v = spd(1)  # power-law SPD: values not exact in FP32 -> use its FP32 rounding
    st, r, c, v = orc.canonical(N, N, r, c, v)
    v32 = v.astype(np.float32).astype(np.float64)
    A = dm.dynmat_create(N, N, r, c, v32)
    A.convert("csr", dm.F32)
    b_np = synth.uniform_pm1(77, N)
    probs.append((A, torch.from_numpy(b_np).cuda()))
    refs.append((N, orc.coo_to_csr(N, r), c, v32, b_np))
    res, xs = run_batch_cg(dm, torch, probs, [0, 1, 2], precision)
    for k, (N, rp, c, v, b_np) in enumerate(refs):
        assert res[k]["status"] == dm.OK, (k, res[k])
        assert res[k]["outer_iterations"] >= 2
        y = orc.spmv("csr", N, N, {"rowptr": rp, "col": c, "val": v}, xs[k])
        assert np.linalg.norm(b_np - y) / np.linalg.norm(b_np) <= 1e-10
        if prec == "reliable":
            ref = orc.cg_reliable(N, rp, c, v, b_np, tol=1e-10)
            # FP32 inner sums in another order round differently: a few
            # iterations either way (2%, at least 3)
            assert abs(res[k]["iterations"] - ref["iterations"]) <= max(3, 0.02 * ref["iterations"])
            assert np.linalg.norm(xs[k] - ref["x"]) / np.linalg.norm(ref["x"]) <= 1e-8
    if prec == "reliable":
        # slot 1 alone in a batch: bit-identical to its run in the mix
        res1, xs1 = run_batch_cg(dm, torch, [probs[1]], [3], precision)
        assert res1[3]["iterations"] == res[1]["iterations"]
        assert np.array_equal(xs1[3].view(np.uint64), xs[1].view(np.uint64))


def test_batch_admission_oom_leaves_batch_running(env):
    dm, torch = env
    N, r, c, v = synth.stencil27(16)
    A = dm.dynmat_create(N, N, r, c, v)
    A.convert("dia")
    b = torch.ones(N, dtype=torch.float64, device="cuda")
    B = dm.DynBatch(2)
    x0 = torch.zeros_like(b)
    B.cg_admit(0, A, b, x0, tol=1e-10)
    dm.dynmat_set_memory_limit(dm.dynmat_memory_in_use() + 4096)
    try:
        x1 = torch.zeros_like(b)
        with pytest.raises(dm.DynmatError) as e:
            B.cg_admit(1, A, b, x1, tol=1e-10)
        assert e.value.status == dm.ERR_OOM
    finally:
        dm.dynmat_set_memory_limit(0)
    for _ in range(200):
        done, active = B.cg_step(8)
        if active == 0:
            break
    assert B.cg_result(0)["status"] == dm.OK


def skewed_rows(seed: int, N: int = 20000):
    """Rows of every awkward length for the segmented CSR tile: empty rows
    (also a trailing run), one-entry rows, rows of 2..41 entries, and rows of
    2500 and 5000 entries that cross chunk and tile boundaries."""
    i = np.arange(N)
    lens = np.where(i % 7 == 3, 0, np.where(i % 5 == 0, 1, 1 + (i * 37) % 41))
    lens[100] = 5000
    lens[9000] = 2500
    lens[N - 10:] = 0
    row = np.repeat(i, lens).astype(np.int32)
    k = np.concatenate([np.arange(n) for n in lens]) if lens.sum() else np.zeros(0, np.int64)
    col = ((row.astype(np.int64) * 131 + k * 997) % N).astype(np.int32)  # distinct per row
    val = synth.uniform_pm1(seed, row.size)
    return N, row, col, val


@pytest.mark.parametrize("E", [256, 777, 4096, 16384])
def test_segmented_csr_tile_matches_oracle(env, orc, E):
    dm, torch = env
    N, r, c, v = skewed_rows(200)
    st, r2, c2, v2 = orc.canonical(N, N, r, c, v)
    a = orc.to_format("csr", N, N, r2, c2, v2)
    x64 = synth.uniform_pm1(201, N)
    want = orc.spmv("csr", N, N, a, x64)
    bound = orc.spmv("csr", N, N, {"rowptr": a["rowptr"], "col": c2, "val": np.abs(v2)},
                     np.abs(x64))
    lens = np.diff(a["rowptr"])
    B = dm.DynBatch(3)
    A = dm.dynmat_create(N, N, r, c, v)
    A.convert("csr")
    x = torch.from_numpy(x64).cuda()
    y = torch.full((N,), float("nan"), dtype=torch.float64, device="cuda")
    B.set(0, A, x, y, shape=(0, 2048, E))
    # an FP32 copy in the same batch (FP32 products and sums)
    A32 = dm.dynmat_create(N, N, r, c, v.astype(np.float32))
    A32.convert("csr")
    x32 = torch.from_numpy(x64.astype(np.float32)).cuda()
    y32 = torch.full((N,), float("nan"), dtype=torch.float32, device="cuda")
    B.set(1, A32, x32, y32, shape=(0, 1024, E))
    # and a stencil in DIA next to them
    Ns, rs, cs, vs = synth.stencil27(12)
    S = dm.dynmat_create(Ns, Ns, rs, cs, vs)
    S.convert("dia")
    xs = torch.ones(Ns, dtype=torch.float64, device="cuda")
    ys = torch.full((Ns,), float("nan"), dtype=torch.float64, device="cuda")
    B.set(2, S, xs, ys)
    B.spmv()
    torch.cuda.synchronize()
    got = y.cpu().numpy()
    assert np.all(np.abs(got - want) <= 1e-13 * bound)
    assert np.all(got[lens == 0] == 0.0)
    # FP32: within (len + 2) u32 of the exact products' sum (FP64 oracle on the
    # FP32-rounded inputs)
    v32 = v2.astype(np.float32).astype(np.float64)
    xr = x64.astype(np.float32).astype(np.float64)
    want32 = orc.spmv("csr", N, N, {"rowptr": a["rowptr"], "col": c2, "val": v32}, xr)
    b32 = orc.spmv("csr", N, N, {"rowptr": a["rowptr"], "col": c2, "val": np.abs(v32)}, np.abs(xr))
    err = np.abs(y32.cpu().numpy().astype(np.float64) - want32)
    assert np.all(err <= (lens + 2) * 2.0 ** -24 * b32)
    # the stencil's rows sum to A 1 exactly (integers)
    sw = orc.spmv("coo", Ns, Ns, {"row": rs, "col": cs, "val": vs}, np.ones(Ns))
    assert np.array_equal(ys.cpu().numpy(), sw)
    # deterministic: a replay gives the same bits
    first = got.copy()
    B.spmv()
    torch.cuda.synchronize()
    assert np.array_equal(y.cpu().numpy(), first)


def tiny_rows(seed: int, N: int = 60000):
    """Rows of 0, 1 and 2 entries (mean 0.9): a 256-entry chunk holds more
    than 32 row starts, and tiles of 4096 or more entries hold more rows than
    the tile's staged row pointers (1023), so the row pointers are read from
    global memory."""
    i = np.arange(N)
    lens = ((i * 2654435761) >> 7) % 3
    lens[(i % 11) == 0] = 0
    row = np.repeat(i, lens).astype(np.int32)
    k = np.concatenate([np.arange(n) for n in lens])
    col = ((row.astype(np.int64) * 7919 + k * 104729) % N).astype(np.int32)
    val = synth.uniform_pm1(seed, row.size)
    return N, row, col, val


@pytest.mark.parametrize("E", [256, 4096, 16384])
def test_segmented_csr_tile_on_tiny_rows(env, orc, E):
    dm, torch = env
    N, r, c, v = tiny_rows(400)
    st, r2, c2, v2 = orc.canonical(N, N, r, c, v)
    a = orc.to_format("csr", N, N, r2, c2, v2)
    x64 = synth.uniform_pm1(401, N)
    want = orc.spmv("csr", N, N, a, x64)
    bound = orc.spmv("csr", N, N, {"rowptr": a["rowptr"], "col": c2, "val": np.abs(v2)},
                     np.abs(x64))
    B = dm.DynBatch(1)
    A = dm.dynmat_create(N, N, r, c, v)
    A.convert("csr")
    x = torch.from_numpy(x64).cuda()
    y = torch.full((N,), float("nan"), dtype=torch.float64, device="cuda")
    B.set(0, A, x, y, shape=(0, 2048, E))
    B.spmv()
    torch.cuda.synchronize()
    got = y.cpu().numpy()
    assert np.all(np.abs(got - want) <= 1e-13 * bound)
    assert np.all(got[np.diff(a["rowptr"]) == 0] == 0.0)


def test_segmented_csr_cg_matches_lanes(env):
    """Batched CG on an SPD matrix with long rows: the segmented tile and the
    lanes tile reach the same tolerance with the same iteration count (+-2)."""
    dm, torch = env
    N, r, c, v = synth.powerlaw(300, 30000, spd=True)
    b = torch.from_numpy(synth.uniform_pm1(301, N)).cuda()
    res = {}
    for lanes in (0, 8):
        B = dm.DynBatch(1)
        A = dm.dynmat_create(N, N, r, c, v)
        A.convert("csr")
        x = torch.zeros(N, dtype=torch.float64, device="cuda")
        B.cg_admit(0, A, b, x, tol=1e-10, max_iters=2000, shape=(lanes, 2048, 1024))
        while True:
            done, n_active = B.cg_step(16)
            if n_active == 0:
                break
        res[lanes] = B.cg_result(0)
    assert res[0]["status"] == 0 and res[8]["status"] == 0
    assert res[0]["true_rel_residual"] <= 1e-9
    assert abs(res[0]["iterations"] - res[8]["iterations"]) <= 2


@pytest.mark.parametrize("prec", ["fp64", "reliable"])
def test_paused_slot_keeps_its_bits(env, prec):
    """A slot paused for some steps (cg_batch_pause) and resumed reaches the
    same iteration count and bit-identical solution as without the pause;
    while paused its solve does not move, and the other slots run on."""
    dm, torch = env
    precision = dm.CG_FP64 if prec == "fp64" else dm.CG_MIXED_RELIABLE
    vdt = dm.F64 if prec == "fp64" else dm.F32
    probs = []
    for k in range(3):
        N, r, c, v = spd(k)
        if prec == "reliable":
            v = v.astype(np.float32).astype(np.float64)
        A = dm.dynmat_create(N, N, r, c, v)
        A.convert(["dia", "csr", "ell"][k], vdt)
        probs.append((A, torch.from_numpy(synth.uniform_pm1(70 + k, N)).cuda()))
    ref, xref = run_batch_cg(dm, torch, probs, [0, 1, 2], precision)
    B = dm.DynBatch(3)
    xs = {}
    for s, (A, b) in enumerate(probs):
        xs[s] = torch.zeros_like(b)
        B.cg_admit(s, A, b, xs[s], tol=1e-10, max_iters=2000, precision=precision)
    B.cg_step(8)
    B.cg_pause(1, True)
    frozen = xs[1].clone()
    for _ in range(3):
        B.cg_step(8)
    torch.cuda.synchronize()
    assert torch.equal(xs[1], frozen)              # nothing moved while paused
    B.cg_pause(1, True)                            # pausing twice is harmless
    B.cg_pause(1, False)
    for _ in range(2000):
        done, active = B.cg_step(8)
        if active == 0:
            break
    for s in range(3):
        got = B.cg_result(s)
        assert got["status"] == dm.OK and got["iterations"] == ref[s]["iterations"], s
        assert np.array_equal(xs[s].cpu().numpy().view(np.uint64), xref[s].view(np.uint64)), s
    assert dm.lib.cg_batch_pause(B.h, 0, 2, None) == dm.ERR_INVALID_ARG  # not 0 or 1
