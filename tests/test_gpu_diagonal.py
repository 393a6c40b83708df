"""Diagonal extraction and update (§III-D; §IV-B: HPCG's CG test modifies the
diagonal): bit-exact against the oracle in every format, refused when a
diagonal entry is missing, and a CG check in the spirit of that test
(exaggerated diagonal -> a few iterations; restored -> the original matrix,
bit for bit, and its iteration count)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

FORMATS = ["coo", "csr", "dia", "ell", "hyb"]


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2209_06478_b300 import build
    build.build()
    from paper_2209_06478_b300 import dynmat
    return dynmat, torch


def with_full_diagonal(seed, n, m):
    """A random n x m matrix whose every (i, i), i < min(n, m), is stored."""
    r, c, v = synth.random_coo(seed, n, m, 0.2)
    k = min(n, m)
    d = np.arange(k, dtype=np.int32)
    r = np.concatenate([r, d])
    c = np.concatenate([c, d])
    v = np.concatenate([v, synth.uniform_pm1(seed + 7, k) + 3.0])
    key = r.astype(np.int64) * m + c
    _, first = np.unique(key, return_index=True)
    return r[first], c[first], v[first]


@pytest.mark.parametrize("fmt", FORMATS)
@pytest.mark.parametrize("shape", [(300, 300), (200, 260), (260, 200)])
def test_extract_and_update_bit_exact(env, orc, fmt, shape):
    dm, torch = env
    n, m = shape
    r, c, v = with_full_diagonal(50 + n + m, n, m)
    st, r2, c2, v2 = orc.canonical(n, m, r, c, v)
    k = min(n, m)
    want, stored = orc.diagonal(n, m, r2, c2, v2)
    assert stored == k
    A = dm.dynmat_create(n, m, r, c, v)
    A.convert(fmt)
    d = torch.full((k,), float("nan"), dtype=torch.float64, device="cuda")
    A.diagonal(d)
    assert np.array_equal(d.cpu().numpy(), want)
    newd = synth.uniform_pm1(99, k) + 5.0
    A.set_diagonal(torch.from_numpy(newd).cuda())
    v3, cnt = orc.set_diagonal(r2, c2, v2, newd)
    A.convert("coo")
    got_r = A.copy_out(0, A.info().nnz, np.int32)
    got_c = A.copy_out(1, A.info().nnz, np.int32)
    got_v = A.copy_out(2, A.info().nnz, np.float64)
    assert np.array_equal(got_r, r2) and np.array_equal(got_c, c2)
    assert np.array_equal(got_v, v3)


def test_extract_reads_zero_where_not_stored(env, orc):
    dm, torch = env
    r, c, v = synth.random_coo(61, 120, 120, 0.05)
    st, r2, c2, v2 = orc.canonical(120, 120, r, c, v)
    want, stored = orc.diagonal(120, 120, r2, c2, v2)
    assert stored < 120
    for fmt in ("coo", "csr", "ell", "hyb"):
        A = dm.dynmat_create(120, 120, r, c, v)
        A.convert(fmt)
        d = torch.full((120,), float("nan"), dtype=torch.float64, device="cuda")
        A.diagonal(d)
        assert np.array_equal(d.cpu().numpy(), want), fmt
        with pytest.raises(dm.DynmatError):
            A.set_diagonal(torch.ones(120, dtype=torch.float64, device="cuda"))
        # refused: nothing changed
        A.diagonal(d)
        assert np.array_equal(d.cpu().numpy(), want), fmt


def test_f32_values(env, orc):
    dm, torch = env
    r, c, v = with_full_diagonal(71, 150, 150)
    v32 = v.astype(np.float32)
    A = dm.dynmat_create(150, 150, r, c, v32)
    A.convert("csr")
    d = torch.empty(150, dtype=torch.float32, device="cuda")
    A.diagonal(d)
    st, r2, c2, v2 = orc.canonical(150, 150, r, c, v32.astype(np.float64))
    want, _ = orc.diagonal(150, 150, r2, c2, v2)
    assert np.array_equal(d.cpu().numpy().astype(np.float64), want)


def test_exaggerated_diagonal_cg(env):
    dm, torch = env
    N, r, c, v = synth.stencil27(16)
    A = dm.dynmat_create(N, N, r, c, v)
    A.convert("dia")
    orig_vals = A.copy_out(2, A.info().ndiag * A.info().ld, np.float64)
    ones = torch.ones(N, dtype=torch.float64, device="cuda")
    b = torch.empty(N, dtype=torch.float64, device="cuda")
    A.spmv(ones, b)
    x = torch.zeros(N, dtype=torch.float64, device="cuda")
    base = A.cg_solve(b, x, tol=1e-9, max_iters=500)
    d0 = torch.empty(N, dtype=torch.float64, device="cuda")
    A.diagonal(d0)
    assert torch.all(d0 == 26.0)
    # the diagonal grows by 10^6 (differently per row): A is then nearly a
    # scaled identity and CG needs only a few iterations
    scale = torch.from_numpy(1e6 * (1.0 + (np.arange(N) % 7) / 7.0)).cuda()
    A.set_diagonal(d0 * scale)
    b2 = torch.empty_like(b)
    A.spmv(ones, b2)
    x2 = torch.zeros_like(x)
    res = A.cg_solve(b2, x2, tol=1e-9, max_iters=500)
    assert res["status"] == 0 and res["iterations"] <= 12
    assert torch.max(torch.abs(x2 - 1.0)).item() < 1e-6
    # restoring gives back the original matrix and its iteration count
    A.set_diagonal(d0)
    assert np.array_equal(A.copy_out(2, A.info().ndiag * A.info().ld, np.float64), orig_vals)
    x3 = torch.zeros_like(x)
    again = A.cg_solve(b, x3, tol=1e-9, max_iters=500)
    assert again["iterations"] == base["iterations"]
    assert torch.equal(x3, x)
