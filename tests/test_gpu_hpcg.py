"""HPCG's preconditioned CG on the GPU (§II-B): the colour-ordered symmetric
Gauss-Seidel sweep, the multigrid V-cycle and PCG against the oracle's
statement of the same steps. The sweep differs from the oracle only in
rounding (fused multiply-adds), so results are compared within a bound."""
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


# (48, 40, 36) and (33, 17, 9): colour grids of uneven sizes, spread over
# the blocks in uneven runs.
@pytest.mark.parametrize("dims,points", [((8, 6, 4), 27), ((16, 16, 16), 27), ((6, 10, 4), 7),
                                         ((48, 40, 36), 27), ((33, 17, 9), 7)])
def test_symgs_sweep_matches_oracle(env, orc, dims, points):
    dm, torch = env
    M = dm.DynMG(*dims, points=points, levels=1)
    lv = orc.stencil_levels(dims, 1, kind=points)[0]
    n = lv["n"]
    r = synth.uniform_pm1(11, n)
    z0 = synth.uniform_pm1(12, n)
    want = orc.symgs(lv, r, z0)
    z = torch.from_numpy(z0.copy()).cuda()
    M.symgs(0, torch.from_numpy(r).cuda(), z)
    got = z.cpu().numpy()
    assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want))


@pytest.mark.parametrize("nlev", [1, 2, 3])
def test_vcycle_matches_oracle(env, orc, nlev):
    dm, torch = env
    dims = (16, 16, 16)
    M = dm.DynMG(*dims, levels=nlev)
    levels = orc.stencil_levels(dims, nlev)
    r = synth.uniform_pm1(13, levels[0]["n"])
    want = orc.mg_apply(levels, r)
    z = torch.full((levels[0]["n"],), float("nan"), dtype=torch.float64, device="cuda")
    M.apply(torch.from_numpy(r).cuda(), z)
    assert np.max(np.abs(z.cpu().numpy() - want)) <= 1e-12 * np.max(np.abs(want))


def test_vcycle_matches_oracle_on_uneven_levels(env, orc):
    """Three levels on 48 x 40 x 36 (coarsest 12 x 10 x 9, odd in z): the
    coarse cycle's passes on uneven colour grids, and a second V-cycle from
    the barrier counts the first left."""
    dm, torch = env
    dims = (48, 40, 36)
    M = dm.DynMG(*dims, levels=3)
    levels = orc.stencil_levels(dims, 3)
    r = synth.uniform_pm1(17, levels[0]["n"])
    want = orc.mg_apply(levels, r)
    z = torch.full((levels[0]["n"],), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):
        M.apply(torch.from_numpy(r).cuda(), z)
        assert np.max(np.abs(z.cpu().numpy() - want)) <= 1e-12 * np.max(np.abs(want))


@pytest.mark.parametrize("dims,nlev", [((80, 80, 80), 3), ((96, 96, 96), 2)])
def test_vcycle_launch_paths_match_oracle(env, orc, dims, nlev):
    """The smallest levels run on one thread-block cluster when every colour
    of them has at most 256 points per CTA (at most 4096 on 16 CTAs).
    80^3 with 3 levels: level 1 (40^3, colours of 8000 points) is swept on
    the whole grid before level 2 (20^3) goes to the cluster. 96^3 with 2
    levels: the coarsest level (48^3, colours of 13824 points) is too large,
    and the whole coarse cycle runs on the grid. Two V-cycles each."""
    dm, torch = env
    M = dm.DynMG(*dims, levels=nlev)
    levels = orc.stencil_levels(dims, nlev)
    r = synth.uniform_pm1(19, levels[0]["n"])
    want = orc.mg_apply(levels, r)
    z = torch.full((levels[0]["n"],), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):
        M.apply(torch.from_numpy(r).cuda(), z)
        assert np.max(np.abs(z.cpu().numpy() - want)) <= 1e-12 * np.max(np.abs(want))


@pytest.mark.parametrize("dims,nlev", [((16, 16, 16), 3), ((24, 20, 16), 2)])
def test_vcycle_7_point_matches_oracle(env, orc, dims, nlev):
    """The 7-point hierarchy: its zero-start passes (different slot sets),
    its coarse cycle and its residual at the coarse points."""
    dm, torch = env
    M = dm.DynMG(*dims, points=7, levels=nlev)
    levels = orc.stencil_levels(dims, nlev, kind=7)
    r = synth.uniform_pm1(18, levels[0]["n"])
    want = orc.mg_apply(levels, r)
    z = torch.full((levels[0]["n"],), float("nan"), dtype=torch.float64, device="cuda")
    M.apply(torch.from_numpy(r).cuda(), z)
    assert np.max(np.abs(z.cpu().numpy() - want)) <= 1e-12 * np.max(np.abs(want))


def test_gpu_preconditioner_is_symmetric(env):
    dm, torch = env
    M = dm.DynMG(16, 16, 16, levels=3)
    n = 16 ** 3
    u = torch.from_numpy(synth.uniform_pm1(14, n)).cuda()
    w = torch.from_numpy(synth.uniform_pm1(15, n)).cuda()
    Mu, Mw = torch.empty_like(u), torch.empty_like(w)
    M.apply(u, Mu)
    M.apply(w, Mw)
    a, b = torch.dot(w, Mu).item(), torch.dot(u, Mw).item()
    assert abs(a - b) <= 1e-12 * torch.norm(u).item() * torch.norm(Mw).item()
    assert torch.dot(u, Mu).item() > 0


@pytest.mark.parametrize("nlev", [1, 3])
def test_pcg_iterates_match_oracle(env, orc, nlev):
    dm, torch = env
    dims = (16, 16, 16)
    M = dm.DynMG(*dims, levels=nlev)
    levels = orc.stencil_levels(dims, nlev)
    b = synth.uniform_pm1(16, levels[0]["n"])
    want = orc.pcg(levels, b, tol=0.0, max_iters=10)
    x = torch.zeros(levels[0]["n"], dtype=torch.float64, device="cuda")
    res = M.pcg_solve(torch.from_numpy(b).cuda(), x, tol=0.0, max_iters=10, check_every=4)
    assert res["iterations"] == 10 and res["status"] == dm.ERR_NOT_CONVERGED
    got = x.cpu().numpy()
    assert np.linalg.norm(got - want["x"]) <= 1e-10 * np.linalg.norm(want["x"])


def test_pcg_converges_and_beats_cg(env, orc):
    dm, torch = env
    dims = (24, 24, 24)
    M = dm.DynMG(*dims, levels=3)
    A, d = M.level(0)
    assert d == dims
    n = 24 ** 3
    ones = torch.ones(n, dtype=torch.float64, device="cuda")
    b = torch.empty_like(ones)
    A.spmv(ones, b)
    x = torch.zeros_like(ones)
    res = M.pcg_solve(b, x, tol=1e-9, max_iters=300)
    assert res["status"] == 0 and res["true_rel_residual"] <= 1e-8
    assert torch.max(torch.abs(x - 1.0)).item() < 1e-6
    levels = orc.stencil_levels(dims, 3)
    want = orc.pcg(levels, b.cpu().numpy(), tol=1e-9, max_iters=300)
    assert abs(res["iterations"] - want["iterations"]) <= 1
    xc = torch.zeros_like(ones)
    plain = A.cg_solve(b, xc, tol=1e-9, max_iters=300)
    assert res["iterations"] * 1.5 <= plain["iterations"]


def test_hierarchy_errors(env):
    dm, torch = env
    with pytest.raises(dm.DynmatError):
        dm.DynMG(12, 12, 12, levels=4)     # 12 does not divide by 8
    with pytest.raises(dm.DynmatError):
        dm.DynMG(8, points=9, levels=1)
    with pytest.raises(dm.DynmatError):
        dm.DynMG(8, levels=3)              # a 2^3 coarsest grid drops stencil diagonals
    dm.DynMG(8, points=7, levels=3)        # the 7-point stencil keeps them on 2^3
    M = dm.DynMG(8, levels=2)
    with pytest.raises(dm.DynmatError):
        M.level(2)
    A, _ = M.level(1)
    with pytest.raises(dm.DynmatError):
        A.destroy()                        # borrowed: freed by the hierarchy
