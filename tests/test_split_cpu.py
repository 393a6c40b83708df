"""Local / remote split of a partitioned stencil (§IV-B, §V-E): the partition
generator is pinned to the unpartitioned stencil and to the halo's closed
form, and the oracle's split product to its product of the whole matrix."""
import numpy as np
import pytest

import synth


def rank_major_perm(n, procs):
    """perm[g] = rank-major index of natural point g (x fastest over the grid)."""
    nx, ny, nz = n
    px, py, pz = procs
    lx, ly, lz = nx // px, ny // py, nz // pz
    g = np.arange(nx * ny * nz)
    x, y, z = g % nx, (g // nx) % ny, g // (nx * ny)
    owner = x // lx + px * (y // ly + py * (z // lz))
    loc = x % lx + lx * (y % ly + ly * (z % lz))
    return owner * (lx * ly * lz) + loc


def assembled(n, procs, kind=27):
    """All ranks' parts mapped back to rank-major global (row, col, val)."""
    P = procs[0] * procs[1] * procs[2]
    rows, cols, vals = [], [], []
    for r in range(P):
        part = synth.partition_stencil(n, procs, r, kind)
        off = part["offset"]
        lr, lc, lv = part["local"]
        rr, rc, rv = part["remote"]
        rows += [lr.astype(np.int64) + off, rr.astype(np.int64) + off]
        cols += [lc.astype(np.int64) + off, part["halo"][rc].astype(np.int64)]
        vals += [lv, rv]
    return np.concatenate(rows), np.concatenate(cols), np.concatenate(vals)


@pytest.mark.parametrize("n,procs,kind", [((6, 6, 6), (2, 1, 3), 27), ((8, 4, 6), (2, 2, 2), 27),
                                          ((6, 6, 6), (3, 3, 1), 7), ((4, 4, 4), (1, 1, 1), 27)])
def test_parts_reassemble_the_permuted_stencil(n, procs, kind):
    N, r, c, v = synth.stencil(n[0], kind, n[1], n[2])
    perm = rank_major_perm(n, procs)
    want = sorted(zip(perm[r].tolist(), perm[c].tolist(), v.tolist()))
    gr, gc, gv = assembled(n, procs, kind)
    got = sorted(zip(gr.tolist(), gc.tolist(), gv.tolist()))
    assert got == want  # every entry exactly once, with its value


def test_interior_halo_closed_form():
    # the middle rank of a 3x3x3 grid of 3x4x5 subgrids touches no boundary
    n, procs = (9, 12, 15), (3, 3, 3)
    part = synth.partition_stencil(n, procs, 13)
    a, b, c = 3, 4, 5
    assert part["nloc"] == a * b * c
    assert part["halo"].size == (a + 2) * (b + 2) * (c + 2) - a * b * c
    # 7-point: only the six faces
    part7 = synth.partition_stencil(n, procs, 13, kind=7)
    assert part7["halo"].size == 2 * (a * b + b * c + a * c)
    # a corner rank of the same grid: three faces, three edges, one corner
    corner = synth.partition_stencil(n, procs, 0)
    assert corner["halo"].size == (a + 1) * (b + 1) * (c + 1) - a * b * c


def test_halo_is_sorted_and_owned_elsewhere():
    n, procs = (8, 8, 8), (2, 2, 2)
    for r in range(8):
        part = synth.partition_stencil(n, procs, r)
        h = part["halo"]
        assert np.all(np.diff(h) > 0)
        assert not np.any((h >= part["offset"]) & (h < part["offset"] + part["nloc"]))
        rr, rc, rv = part["remote"]
        assert rc.min() >= 0 and rc.max() < h.size and np.all(rv == -1.0)


def test_oracle_split_product_equals_whole_product(orc):
    n, procs = (8, 6, 4), (2, 3, 2)
    gr, gc, gv = assembled(n, procs)
    N = n[0] * n[1] * n[2]
    x = synth.uniform_pm1(41, N)
    st, r2, c2, v2 = orc.canonical(N, N, gr.astype(np.int32), gc.astype(np.int32), gv)
    whole = orc.spmv("coo", N, N, {"row": r2, "col": c2, "val": v2}, x)
    bound = orc.spmv("coo", N, N, {"row": r2, "col": c2, "val": np.abs(v2)}, np.abs(x))
    for r in range(procs[0] * procs[1] * procs[2]):
        part = synth.partition_stencil(n, procs, r)
        nl, off, h = part["nloc"], part["offset"], part["halo"]
        lr, lc, lv = part["local"]
        rr, rc, rv = part["remote"]
        st, a, b, c = orc.canonical(nl, nl, lr, lc, lv)
        y = orc.spmv("coo", nl, nl, {"row": a, "col": b, "val": c}, x[off:off + nl])
        st, a, b, c = orc.canonical(nl, h.size, rr, rc, rv)
        y += orc.spmv("coo", nl, h.size, {"row": a, "col": b, "val": c}, x[h])
        sl = slice(off, off + nl)
        assert np.all(np.abs(y - whole[sl]) <= 1e-13 * bound[sl])
