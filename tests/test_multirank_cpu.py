"""Multi-process paths on CPU: two ranks over torch.distributed's gloo backend.

- The benchmark's whole-job figures: the maximum over ranks of the timed
  region and of the kernel time, work units summed over ranks.
- The partitioned product of §V-E: each rank holds only its slice of x and
  its (local, remote) parts, fetches its halo from the other rank, and
  multiplies with the oracle; the gathered y equals the oracle's product
  of the whole (rank-major permuted) stencil.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

WORLD = 2


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def run_ranks(fn, *args):
    port = free_port()
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    procs = [ctx.Process(target=_entry, args=(r, port, q, fn, args)) for r in range(WORLD)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    out = {}
    while not q.empty():
        r, res = q.get()
        out[r] = res
    for p in procs:
        assert p.exitcode == 0, "rank exited with %s" % p.exitcode
    return [out[r] for r in range(WORLD)]


def _entry(rank, port, q, fn, args):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        q.put((rank, fn(rank, *args)))
    finally:
        dist.destroy_process_group()


def _aggregate(rank):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    # rank 1 is slower and did more work
    total = [10.0, 12.5][rank]
    kernel = [0.20, 0.25][rank]
    units = [1000.0, 3000.0][rank]
    return bench.aggregate_ranks(total, kernel, units, WORLD, None)


def test_bench_aggregates_max_time_and_total_units():
    res = run_ranks(_aggregate)
    for total_ms, kernel_ms, units in res:  # every rank sees the same whole-job figures
        assert total_ms == 12.5 and kernel_ms == 0.25 and units == 4000.0


def _split_product(rank, n, procs):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import oracle
    import synth
    part = synth.partition_stencil(n, procs, rank)
    nl, off, halo = part["nloc"], part["offset"], part["halo"]
    N = int(np.prod(n))
    x_global = synth.uniform_pm1(3, N)          # the same seeded vector on every rank ...
    x_mine = x_global[off:off + nl].copy()      # ... of which this rank keeps only its slice
    # halo exchange: every rank contributes its slice (equal sizes here)
    parts = [torch.zeros(nl, dtype=torch.float64) for _ in range(WORLD)]
    dist.all_gather(parts, torch.from_numpy(x_mine))
    x_all = torch.cat(parts).numpy()
    x_halo = x_all[halo]
    assert np.array_equal(x_all[off:off + nl], x_mine)
    lr, lc, lv = part["local"]
    rr, rc, rv = part["remote"]
    a_loc = oracle.to_format("csr", nl, nl, lr, lc, lv)
    y = oracle.spmv("csr", nl, nl, a_loc, x_mine)
    if rr.size:
        a_rem = oracle.to_format("coo", nl, halo.size, rr, rc, rv)
        y = y + oracle.spmv("coo", nl, halo.size, a_rem, x_halo)
    ys = [torch.zeros(nl, dtype=torch.float64) for _ in range(WORLD)]
    dist.all_gather(ys, torch.from_numpy(y))
    return torch.cat(ys).numpy(), x_global


@pytest.mark.parametrize("n,procs", [((6, 4, 4), (2, 1, 1)), ((4, 6, 4), (1, 2, 1)),
                                     ((4, 4, 6), (1, 1, 2))])
def test_two_rank_split_product_matches_whole(n, procs):
    import oracle
    import synth
    from test_split_cpu import rank_major_perm
    res = run_ranks(_split_product, n, procs)
    y0, x = res[0]
    assert np.array_equal(y0, res[1][0])         # both ranks gathered the same y
    N, r, c, v = synth.stencil(n[0], 27, n[1], n[2])
    perm = rank_major_perm(n, procs)
    pr, pc = perm[r], perm[c]
    whole = oracle.to_format("csr", N, N, *oracle.canonical(N, N, pr, pc, v)[1:])
    y_whole = oracle.spmv("csr", N, N, whole, x)
    bound = oracle.spmv("csr", N, N, {"rowptr": whole["rowptr"], "col": whole["col"],
                                      "val": np.abs(whole["val"])}, np.abs(x))
    # the split sums a row in two parts (local, then remote): rounding only
    assert np.all(np.abs(y0 - y_whole) <= 1e-13 * bound)
