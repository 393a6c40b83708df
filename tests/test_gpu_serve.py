"""The continuous-batching server on the GPU: every request converges to the
target, and a request's solution is bit-identical when served alone and when
served in a mix with other requests."""
import numpy as np
import pytest

from paper_2209_06478_b300 import serve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2209_06478_b300 import build
    build.build()
    from paper_2209_06478_b300 import dynmat
    pool = serve.irregular_pool((("banded", 20_000), ("powerlaw", 10_000)))
    return dynmat, torch, pool


def requests():
    return serve.make_requests(14, 300.0, seed=11, stencil_sizes=(12, 16, 24, 32),
                               irregular=(("banded", 20_000), ("powerlaw", 10_000)),
                               irregular_share=0.3)


def test_mixed_batched_server_converges_and_is_mix_invariant(env):
    dm, torch, pool = env
    reqs = requests()
    eng = serve.BatchedEngine(dm, torch, 6, dm.CG_MIXED_RELIABLE, pool, keep_solutions=True)
    sch = serve.Scheduler(eng, 6, 150 * 10**9, iterations_per_tick=8)
    recs = sch.run(reqs)
    for r in recs.values():
        assert r.status == 0 and r.residual <= 1e-10, r
    # the same request alone (a fresh server, nothing else in the batch)
    for pick in (reqs[2], reqs[7]):
        alone = serve.Request(pick.rid, 0.0, pick.kind, pick.size, pick.seed)
        eng1 = serve.BatchedEngine(dm, torch, 6, dm.CG_MIXED_RELIABLE, pool,
                                   keep_solutions=True)
        serve.Scheduler(eng1, 6, 150 * 10**9, iterations_per_tick=8).run([alone])
        a, b = eng1.solutions[pick.rid], eng.solutions[pick.rid]
        assert np.array_equal(a.view(np.uint64), b.view(np.uint64)), pick


def test_fp64_paths_converge(env):
    dm, torch, pool = env
    reqs = requests()[:8]
    for eng in (serve.BatchedEngine(dm, torch, 4, dm.CG_FP64, pool),
                serve.SerialEngine(dm, torch, pool)):
        slots = 4 if isinstance(eng, serve.BatchedEngine) else 1
        recs = serve.Scheduler(eng, slots, 150 * 10**9).run(reqs)
        for r in recs.values():
            assert r.status == 0 and r.residual <= 2e-10, r


def test_budget_limits_admission(env):
    dm, torch, pool = env
    import gc
    reqs = [serve.Request(i, 0.0, "stencil27", 32, 50 + i) for i in range(6)]
    eng = serve.BatchedEngine(dm, torch, 6, dm.CG_MIXED_RELIABLE, pool)
    eng.cache.get(reqs[0])          # the shared matrix is resident from the start
    gc.collect()
    torch.cuda.synchronize()
    per_request = eng.bytes_needed(reqs[0])
    assert per_request > 0 and eng.cache.estimate(reqs[0]) == 0
    # room for about 2.5 requests' vectors and work space at a time
    budget = dm.dynmat_memory_in_use() + eng.vec_bytes + int(2.5 * per_request)
    sch = serve.Scheduler(eng, 6, budget)
    peak = []
    orig_admit = eng.admit

    def admit(slot, req):
        ok = orig_admit(slot, req)
        peak.append(len(eng.vecs))
        return ok

    eng.admit = admit
    recs = sch.run(reqs)
    assert all(r.status == 0 for r in recs.values())
    assert max(peak) <= 3  # the budget never let more than a few in at once


def test_online_tuning_picks_a_batch_format_and_keeps_results(env):
    """The online tuner (a short probe in the batch kernel at first use)
    converts each new matrix to a batch format and hands its tile shape to
    admission; every request still converges to the tolerance."""
    dm, torch, _ = env
    from paper_2209_06478_b300 import serve
    pool = serve.irregular_pool((("banded", 60000), ("powerlaw", 50000)))
    reqs = serve.make_requests(6, 400.0, stencil_sizes=(24,), irregular=tuple(pool),
                               irregular_share=0.6)
    out = serve.serve("mixed_batched", reqs, pool=pool, online_tune=True)
    assert out["converged"] == len(reqs)
    assert out["max_true_rel_residual"] <= 1e-10
    tuned = out["online_tune"]["formats"]
    assert sum(tuned.values()) == len({r.key for r in reqs})
    assert set(tuned) <= {"dia", "ell", "csr"}


def test_batch_tune_matrix_converts_and_returns_a_shape(env):
    dm, torch, _ = env
    import synth
    N, r, c, v = synth.banded(11, 40000, 9)
    A = dm.dynmat_create(N, N, r, c, v)
    fmt, shape = A.batch_tune(effort=0)
    assert dm.FORMATS[fmt] in ("dia", "ell", "csr")
    assert A.info().format == fmt
    assert shape[1] >= 1024 and shape[2] >= 256
    with pytest.raises(dm.DynmatError):
        A.batch_tune(effort=3)
