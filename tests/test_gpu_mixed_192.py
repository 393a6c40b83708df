"""The mixed-precision configuration at full size: the 27-point stencil on a
192^3 grid (7,077,888 rows, 189,119,224 entries), b = A 1, tolerance 1e-10.
Three solves: reliable-update mixed precision (FP32 values and inner CG,
FP64 residual and solution), restarted mixed precision, and plain FP64 CG.
The matrix and b come from the generator and the CPU oracle; the true
relative residual ||b - A x|| / ||b|| of every returned x is recomputed by
the oracle's FP64 product, and x's error against the all-ones solution is
bounded by kappa * tol with the stencil's closed-form condition number."""
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

N3 = 192
# A residual computed in FP64 carries rounding of about 1e-14 ||b||: 1% of
# slack on the 1e-10 target, 1e-3 between the oracle's and the library's value.
SLACK = 1.01


@pytest.fixture(scope="module")
def dm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2209_06478_b300 import build
    build.build()
    from paper_2209_06478_b300 import dynmat
    return dynmat


@pytest.fixture(scope="module")
def system(orc):
    N, r, c, v = synth.stencil27(N3)
    rp = orc.coo_to_csr(N, r)
    a = {"rowptr": rp, "col": c, "val": v}
    b = orc.spmv("csr", N, N, a, np.ones(N), omp=True)
    return N, r, c, v, a, b


def kappa(n):
    t1 = 1 + 2 * math.cos(math.pi / (n + 1))
    tn = 1 + 2 * math.cos(n * math.pi / (n + 1))
    return (27 - t1 * t1 * tn) / (27 - t1 ** 3)


@pytest.mark.parametrize("precision,vdtype,target", [
    ("CG_MIXED_RELIABLE", "F32", 1e-10),
    ("CG_MIXED", "F32", 1e-10),
    ("CG_FP64", "F64", 2e-10),  # stops on the recursive residual; the true one may sit above
])
def test_192_true_residual_checked_by_the_oracle(dm, orc, system, precision, vdtype, target):
    import torch
    N, r, c, v, a, b = system
    A = dm.dynmat_create(N, N, r, c, v)
    A.convert("dia", getattr(dm, vdtype))
    bt = torch.from_numpy(b).cuda()
    xt = torch.zeros_like(bt)
    res = A.cg_solve(bt, xt, tol=1e-10, max_iters=5000, precision=getattr(dm, precision),
                     inner_tol=1e-5, check_every=32)
    A.destroy()
    x = xt.cpu().numpy()
    assert res["status"] == dm.OK, res
    true = float(np.linalg.norm(b - orc.spmv("csr", N, N, a, x, omp=True)) / np.linalg.norm(b))
    print("%s: %d iterations, true relative residual %.3e (library %.3e)"
          % (precision, res["iterations"], true, res["true_rel_residual"]))
    assert true <= SLACK * target
    assert abs(res["true_rel_residual"] - true) <= 1e-3 * true + 1e-15
    assert np.linalg.norm(x - 1) / math.sqrt(N) <= kappa(N3) * SLACK * target
