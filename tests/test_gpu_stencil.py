"""Device-side HPCG problem generation equals the shared seeded generator
(bit for bit) and create + convert of its triplets."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2209_06478_b300 import build
    build.build()
    from paper_2209_06478_b300 import dynmat
    return dynmat


@pytest.mark.parametrize("points", [27, 7])
@pytest.mark.parametrize("dims", [(5, 5, 5), (4, 6, 3), (1, 1, 7), (16, 16, 16)])
def test_device_stencil_equals_generator(dm, points, dims):
    nx, ny, nz = dims
    N, r, c, v = synth.stencil(nx, points, ny=ny, nz=nz)
    A = dm.dynmat_create_stencil(nx, points, dm.COO, dm.F64, ny=ny, nz=nz)
    a = A.arrays()
    assert np.array_equal(a["row"], r) and np.array_equal(a["col"], c)
    assert np.array_equal(a["val"], v)
    for fmt in ("csr", "dia", "ell", "hyb"):
        for vdt in (dm.F64, dm.F32):
            G = dm.dynmat_create_stencil(nx, points, fmt, vdt, ny=ny, nz=nz)
            H = dm.dynmat_create(N, N, r, c, v)
            H.convert(fmt, vdt)
            ga, ha = G.arrays(), H.arrays()
            for k in ha:
                if isinstance(ha[k], np.ndarray):
                    assert np.array_equal(ga[k], ha[k]), (fmt, vdt, k)
