"""Bounded waits: a wait that nothing can satisfy gives up after its limit,
says so, and leaves the context usable (no GPU fault, no hang). The kernels
use the same wait functions with a limit of about 2 s; the self-test uses
20M cycles (about 10 ms)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2209_06478_b300 import dynmat as dm
    return dm, torch


@pytest.mark.parametrize("which", [0, 1])
def test_unsatisfiable_wait_times_out_and_context_survives(env, which):
    dm, torch = env
    assert dm.dynmat_selftest_wait_timeout(which, 20_000_000) is True
    # the device still works: a product right after matches its reference
    N, r, c, v = synth.stencil27(8)
    A = dm.dynmat_create(N, N, r, c, v)
    A.convert("csr")
    x = torch.ones(N, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    A.spmv(x, y)
    torch.cuda.synchronize()
    vals = set(np.unique(y.cpu().numpy()).tolist())
    assert vals <= {19.0, 15.0, 9.0, 0.0}


def test_selftest_rejects_bad_arguments(env):
    dm, torch = env
    with pytest.raises(dm.DynmatError):
        dm.dynmat_selftest_wait_timeout(2, 1000)
    with pytest.raises(dm.DynmatError):
        dm.dynmat_selftest_wait_timeout(0, 0)
