"""The batch configuration at full size, in the launch configuration the
bench times: the 64 FP64 matrices of the batch workload (10k-500k rows; a
third banded with 3-64 diagonals, a third power-law rows, a third uniform
8-32 per row; seeds 100-163), each set in CSR, then given the format and tile
shape the batch tuner picks, and multiplied in one persistent launch replayed
from its CUDA graph. Every row of every product is compared with the oracle's
FP64 CSR product within 1e-13 * sum |a_ij x_j|."""
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


def test_batch_of_64_tuned_matches_oracle(env, orc):
    dm, torch = env
    specs = synth.batch_specs()
    assert len(specs) == 64
    B = dm.DynBatch(len(specs))
    keep = []
    for k, (seed, kind, n, extra) in enumerate(specs):
        N, r, c, v = synth.make(kind, seed, n, extra)
        # the generators emit canonical order (rows, then columns, ascending)
        assert np.all(np.diff(r) >= 0)
        A = dm.dynmat_create(N, N, r, c, v)
        A.convert("csr")
        x = torch.from_numpy(synth.uniform_pm1(seed, N)).cuda()
        y = torch.full((N,), float("nan"), dtype=torch.float64, device="cuda")
        B.set(k, A, x, y)
        keep.append((kind, A, x, y, N, r, c, v))
    formats = {}
    for k in range(len(specs)):
        fmt, _ = B.autotune(k)
        formats.setdefault(keep[k][0], set()).add(dm.FORMATS[fmt])
    # banded matrices go to DIA or, where it times faster, ELL; the irregular
    # ones never to DIA (it would hold one diagonal per distinct column offset)
    assert "dia" in formats["banded"] and formats["banded"] <= {"dia", "ell"}
    assert "dia" not in formats["powerlaw"] | formats["uniform"]
    for rep in range(2):  # the first call captures the graph, the second replays it
        for _, _, _, y, _, _, _, _ in keep:
            y.fill_(float("nan"))
        B.spmv()
        torch.cuda.synchronize()
        for kind, A, x, y, N, r, c, v in keep:
            rp = orc.coo_to_csr(N, r)
            xh = x.cpu().numpy()
            want = orc.spmv("csr", N, N, {"rowptr": rp, "col": c, "val": v}, xh, omp=True)
            bound = orc.spmv("csr", N, N, {"rowptr": rp, "col": c, "val": np.abs(v)}, np.abs(xh),
                             omp=True)
            got = y.cpu().numpy()
            assert np.all(np.abs(got - want) <= 1e-13 * bound), (kind, N, rep)
