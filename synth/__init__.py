"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module only *generates* inputs: COO triplets of the matrices the method
is run on and dense vectors. It holds none of the method's arithmetic (no
format conversion, no SpMV, no solver step), so both sides of every parity
test can consume its output without sharing code.

Randomness comes from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used as a counter-based
generator: draw k of stream `seed` is mix64(seed + (k + 1) * GAMMA) mod 2^64.
A uniform double in [-1, 1) is 2 * (z >> 11) * 2^-53 - 1, which is exact.

Workloads (§II-B: HPCG solves a Poisson problem on a regular 3-D grid
discretised by a 27-point stencil):

* ``stencil27(n)`` — a(i, i) = 26, a(i, j) = -1 for every in-grid neighbour j
  of i in the 3x3x3 box; row index i = ix + n*(iy + n*iz) (x fastest).
* ``stencil7(n)`` — a(i, i) = 6, a(i, j) = -1 for the six face neighbours.
* ``banded``, ``powerlaw``, ``uniform`` — the irregular matrices of the
  batched and served workloads; ``spd=True`` symmetrises S + S^T and sets the
  diagonal to sum|off-diagonal| + 1 so the matrix is SPD.

Every generator returns COO sorted by (row, col) with no duplicates.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
MASK64 = (1 << 64) - 1


def splitmix64(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Draws start .. start+n-1 of the SplitMix64 stream `seed` (uint64)."""
    k = np.arange(start + 1, start + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + k * GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int, start: int = 0) -> np.ndarray:
    """U[0, 1) doubles from the top 53 bits of each draw (exact)."""
    return (splitmix64(seed, n, start) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_pm1(seed: int, n: int, start: int = 0) -> np.ndarray:
    """U[-1, 1) doubles: 2*u - 1 with u from ``uniform01`` (exact)."""
    return 2.0 * uniform01(seed, n, start) - 1.0


def randint(seed: int, n: int, lo: int, hi: int, start: int = 0) -> np.ndarray:
    """Integers in [lo, hi) as floor(u * (hi - lo)) + lo (int64)."""
    u = uniform01(seed, n, start)
    return (np.floor(u * (hi - lo)).astype(np.int64) + lo).clip(lo, hi - 1)


# ---------------------------------------------------------------------------
# Structured grids (HPCG problem generation)
# ---------------------------------------------------------------------------

def _box_offsets(kind: int):
    """(dz, dy, dx) neighbour offsets in ascending linear-offset order."""
    if kind == 27:
        offs = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    elif kind == 7:
        offs = [(-1, 0, 0), (0, -1, 0), (0, 0, -1), (0, 0, 0), (0, 0, 1), (0, 1, 0), (1, 0, 0)]
    else:
        raise ValueError(kind)
    return offs


def stencil(n: int, kind: int = 27, ny: int | None = None, nz: int | None = None,
            chunk_rows: int = 1 << 20):
    """COO triplets of the `kind`-point stencil on an n x ny x nz grid.

    Diagonal = kind - 1, off-diagonal = -1. Rows are emitted in order and,
    within a row, neighbours in ascending column order (the offsets
    dz*n*ny + dy*n + dx are ascending in (dz, dy, dx) lexicographic order).
    Returns (nrows, row int32, col int32, val float64).
    """
    nx = n
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    N = nx * ny * nz
    offs = _box_offsets(kind)
    diag = float(kind - 1)
    rows_out, cols_out, vals_out = [], [], []
    for r0 in range(0, N, chunk_rows):
        r1 = min(N, r0 + chunk_rows)
        i = np.arange(r0, r1, dtype=np.int64)
        ix = i % nx
        iy = (i // nx) % ny
        iz = i // (nx * ny)
        cols = np.empty((r1 - r0, len(offs)), dtype=np.int64)
        ok = np.empty((r1 - r0, len(offs)), dtype=bool)
        vals = np.empty((r1 - r0, len(offs)), dtype=np.float64)
        for k, (dz, dy, dx) in enumerate(offs):
            jx, jy, jz = ix + dx, iy + dy, iz + dz
            ok[:, k] = (jx >= 0) & (jx < nx) & (jy >= 0) & (jy < ny) & (jz >= 0) & (jz < nz)
            cols[:, k] = i + dz * nx * ny + dy * nx + dx
            vals[:, k] = diag if (dz, dy, dx) == (0, 0, 0) else -1.0
        rr = np.broadcast_to(i[:, None], cols.shape)
        rows_out.append(rr[ok].astype(np.int32))
        cols_out.append(cols[ok].astype(np.int32))
        vals_out.append(vals[ok])
    return (N, np.concatenate(rows_out), np.concatenate(cols_out), np.concatenate(vals_out))


def stencil27(n: int):
    return stencil(n, 27)


def stencil7(n: int):
    return stencil(n, 7)


def partition_stencil(n, procs, rank: int, kind: int = 27):
    """One process's part of the `kind`-point stencil on an n^3 grid (n an int
    or (nx, ny, nz)) split over a px x py x pz process grid, as HPCG
    distributes it. Rank r = ipx + px*(ipy + py*ipz) owns the subgrid of
    (nx/px) x (ny/py) x (nz/pz) points; the global vector is numbered rank by
    rank, each rank's points x-fastest within its subgrid.

    Returns a dict:
      nloc: the rank's rows; offset: its first row in the global numbering;
      local: (row, col, val) of the square part, columns in local numbering;
      remote: (row, col, val) of the rectangular part, columns indexing halo;
      halo: int32 global indices (ascending) of the columns owned elsewhere.
    Rows ascend; within a row entries follow the stencil offsets (dz, dy, dx)
    in lexicographic order.
    """
    nx, ny, nz = (n, n, n) if isinstance(n, int) else tuple(n)
    px, py, pz = procs
    if nx % px or ny % py or nz % pz:
        raise ValueError("grid must divide evenly")
    lx, ly, lz = nx // px, ny // py, nz // pz
    nloc = lx * ly * lz
    ipx, ipy, ipz = rank % px, (rank // px) % py, rank // (px * py)
    i = np.arange(nloc, dtype=np.int64)
    ax, ay, az = i % lx, (i // lx) % ly, i // (lx * ly)
    gx, gy, gz = ipx * lx + ax, ipy * ly + ay, ipz * lz + az
    offs = _box_offsets(kind)
    diag = float(kind - 1)
    cols = np.empty((nloc, len(offs)), dtype=np.int64)   # global column (rank-major)
    ok = np.empty((nloc, len(offs)), dtype=bool)
    mine = np.empty((nloc, len(offs)), dtype=bool)
    lcol = np.empty((nloc, len(offs)), dtype=np.int64)
    vals = np.empty((nloc, len(offs)), dtype=np.float64)
    for k, (dz, dy, dx) in enumerate(offs):
        jx, jy, jz = gx + dx, gy + dy, gz + dz
        ok[:, k] = (jx >= 0) & (jx < nx) & (jy >= 0) & (jy < ny) & (jz >= 0) & (jz < nz)
        jxc, jyc, jzc = np.clip(jx, 0, nx - 1), np.clip(jy, 0, ny - 1), np.clip(jz, 0, nz - 1)
        owner = (jxc // lx) + px * ((jyc // ly) + py * (jzc // lz))
        loc = (jxc % lx) + lx * ((jyc % ly) + ly * (jzc % lz))
        cols[:, k] = owner * nloc + loc
        mine[:, k] = owner == rank
        lcol[:, k] = loc
        vals[:, k] = diag if (dz, dy, dx) == (0, 0, 0) else -1.0
    rows = np.broadcast_to(i[:, None], cols.shape)
    lsel = ok & mine
    rsel = ok & ~mine
    halo = np.unique(cols[rsel])
    rcol = np.searchsorted(halo, cols[rsel])
    return {
        "nloc": nloc, "offset": rank * nloc,
        "local": (rows[lsel].astype(np.int32), lcol[lsel].astype(np.int32), vals[lsel]),
        "remote": (rows[rsel].astype(np.int32), rcol.astype(np.int32), vals[rsel]),
        "halo": halo.astype(np.int32),
    }


def stencil_nnz(n: int, kind: int = 27) -> int:
    """Stored entries of the stencil on an n^3 grid: (3n-2)^3 for 27 points,
    n^3 + 6 n^2 (n-1) for 7 points (each axis contributes 2 n^2 (n-1) links)."""
    if kind == 27:
        return (3 * n - 2) ** 3
    return n ** 3 + 6 * n * n * (n - 1)


# ---------------------------------------------------------------------------
# Irregular matrices (batched / served workloads)
# ---------------------------------------------------------------------------

def _sorted_unique(nrows, ncols, row, col, val):
    key = row.astype(np.int64) * ncols + col.astype(np.int64)
    order = np.argsort(key, kind="stable")
    key = key[order]
    keep = np.ones(key.shape[0], dtype=bool)
    keep[1:] = key[1:] != key[:-1]
    order = order[keep]
    return row[order].astype(np.int32), col[order].astype(np.int32), val[order]


def _spd_from(nrows, row, col, val):
    """S + S^T with the diagonal replaced by sum_j |a_ij| (j != i) + 1."""
    off = row != col
    r = np.concatenate([row[off], col[off]]).astype(np.int64)
    c = np.concatenate([col[off], row[off]]).astype(np.int64)
    v = np.concatenate([val[off], val[off]])
    key = r * nrows + c
    order = np.argsort(key, kind="stable")
    key, v = key[order], v[order]
    first = np.ones(key.size, dtype=bool)
    first[1:] = key[1:] != key[:-1]
    start = np.nonzero(first)[0]
    uniq = key[start]
    vs = np.add.reduceat(v, start) if key.size else v
    r = (uniq // nrows).astype(np.int64)
    c = (uniq % nrows).astype(np.int64)
    d = np.ones(nrows, dtype=np.float64)
    np.add.at(d, r, np.abs(vs))
    r = np.concatenate([r, np.arange(nrows)])
    c = np.concatenate([c, np.arange(nrows)])
    v = np.concatenate([vs, d])
    return _sorted_unique(nrows, nrows, r, c, v)


def banded(seed: int, nrows: int, ndiag: int, spread: float = 0.01, spd: bool = False):
    """Square matrix with the main diagonal plus (ndiag-1)//2 symmetric pairs of
    off-diagonals at distinct offsets drawn from [1, max(1, spread*nrows)]."""
    half = max(0, (ndiag - 1) // 2)
    span = max(half, int(spread * nrows), 1)
    offs = set()
    k = 0
    while len(offs) < half:
        o = int(randint(seed, 1, 1, span + 1, start=k)[0])
        k += 1
        offs.add(o)
    offsets = sorted([-o for o in offs] + [0] + list(offs))
    rows, cols = [], []
    for o in offsets:
        i = np.arange(max(0, -o), min(nrows, nrows - o), dtype=np.int64)
        rows.append(i)
        cols.append(i + o)
    row = np.concatenate(rows)
    col = np.concatenate(cols)
    val = uniform_pm1(seed ^ 0x5BD1E995, row.size)
    row, col, val = _sorted_unique(nrows, nrows, row, col, val)
    if spd:
        return (nrows,) + _spd_from(nrows, row, col, val)
    return nrows, row, col, val


ZIPF_S = 1.6956
ZIPF_MAX = 5000


def zipf_lengths(seed: int, nrows: int, s: float = ZIPF_S, lmax: int = ZIPF_MAX) -> np.ndarray:
    """Row lengths L in [1, lmax] with P(L = l) proportional to l^-s."""
    l = np.arange(1, lmax + 1, dtype=np.float64)
    p = l ** (-s)
    cdf = np.cumsum(p) / p.sum()
    u = uniform01(seed, nrows)
    return np.minimum(np.searchsorted(cdf, u, side="right") + 1, lmax).astype(np.int64)


def _sorted_distinct(a: np.ndarray) -> np.ndarray:
    a = np.sort(a)
    if a.size == 0:
        return a
    keep = np.ones(a.size, dtype=bool)
    keep[1:] = a[1:] != a[:-1]
    return a[keep]


def _rows_with_lengths(seed: int, nrows: int, ncols: int, lengths: np.ndarray):
    """Distinct uniform columns per row, `lengths[i]` of them (capped at ncols)."""
    lengths = np.minimum(lengths, ncols)
    total = int(lengths.sum())
    row = np.repeat(np.arange(nrows, dtype=np.int64), lengths)
    col = randint(seed, total, 0, ncols)
    key = _sorted_distinct(row * ncols + col)
    got = np.bincount((key // ncols).astype(np.int64), minlength=nrows)
    # Refill the rows that lost entries to collisions (few; long rows mostly).
    short = np.nonzero(got < lengths)[0]
    extra = []
    draw = total
    lo_idx = np.searchsorted(key, short * ncols, side="left")
    hi_idx = np.searchsorted(key, (short + 1) * ncols, side="left")
    for i, a, b in zip(short.tolist(), lo_idx.tolist(), hi_idx.tolist()):
        have = set((key[a:b] - i * ncols).tolist())
        need = int(lengths[i]) - len(have)
        while need > 0:
            cands = randint(seed, 4 * need + 8, 0, ncols, start=draw)
            draw += cands.size
            for c in cands.tolist():
                if c not in have:
                    have.add(c)
                    extra.append(i * ncols + c)
                    need -= 1
                    if need == 0:
                        break
    if extra:
        key = _sorted_distinct(np.concatenate([key, np.array(extra, dtype=np.int64)]))
    return (key // ncols).astype(np.int64), (key % ncols).astype(np.int64)


def powerlaw(seed: int, nrows: int, spd: bool = False):
    """Zipf row lengths (mean ~20, max 5000), uniform distinct columns."""
    lengths = zipf_lengths(seed, nrows)
    row, col = _rows_with_lengths(seed ^ 0x27D4EB2F, nrows, nrows, lengths)
    val = uniform_pm1(seed ^ 0x165667B1, row.size)
    if spd:
        return (nrows,) + _spd_from(nrows, row, col, val)
    return nrows, row.astype(np.int32), col.astype(np.int32), val


def uniform(seed: int, nrows: int, lo: int = 8, hi: int = 32, spd: bool = False):
    """Uniform row lengths in [lo, hi], uniform distinct columns."""
    lengths = randint(seed, nrows, lo, hi + 1)
    row, col = _rows_with_lengths(seed ^ 0x27D4EB2F, nrows, nrows, lengths)
    val = uniform_pm1(seed ^ 0x165667B1, row.size)
    if spd:
        return (nrows,) + _spd_from(nrows, row, col, val)
    return nrows, row.astype(np.int32), col.astype(np.int32), val


def random_coo(seed: int, nrows: int, ncols: int, density: float, empty_rows: bool = True,
               shuffle: bool = False, int_values: bool = False):
    """Small random matrix for unit tests. Some rows are left empty on purpose;
    `shuffle` returns the triplets in a scrambled (non-canonical) order;
    `int_values` draws small integers so that sums are exact."""
    m = int(round(density * nrows * ncols))
    m = max(0, min(m, nrows * ncols))
    if m == 0:
        e = np.zeros(0, dtype=np.int32)
        return e, e.copy(), np.zeros(0, dtype=np.float64)
    cells = _sorted_distinct(randint(seed, 3 * m + 8, 0, nrows * ncols))[:m]
    perm = np.argsort(uniform01(seed ^ 0xABCDEF, cells.size), kind="stable")
    cells = np.sort(cells[perm][:m])
    row = (cells // ncols).astype(np.int32)
    col = (cells % ncols).astype(np.int32)
    if empty_rows and nrows > 2:
        keep = (row % 5) != 3
        row, col = row[keep], col[keep]
    if int_values:
        val = randint(seed ^ 0x1234, row.size, -4, 5).astype(np.float64)
        val[val == 0] = 5.0
    else:
        val = uniform_pm1(seed ^ 0x1234, row.size)
        val[val == 0] = 0.5
    if shuffle and row.size:
        p = np.argsort(uniform01(seed ^ 0x777, row.size), kind="stable")
        row, col, val = row[p], col[p], val[p]
    return row, col, val


def batch_specs(first_seed: int = 100, count: int = 64, lo: int = 10_000, hi: int = 500_000):
    """The heterogeneous batch: per matrix (seed, kind, nrows, extra).

    Rows are log-uniform in [lo, hi]; kinds cycle banded / powerlaw / uniform;
    banded matrices draw 3..64 diagonals."""
    specs = []
    for k in range(count):
        seed = first_seed + k
        u = float(uniform01(seed, 1)[0])
        nrows = int(round(np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))))
        kind = ("banded", "powerlaw", "uniform")[k % 3]
        extra = int(randint(seed ^ 0x9E37, 1, 3, 65)[0]) if kind == "banded" else 0
        specs.append((seed, kind, nrows, extra))
    return specs


def make(kind: str, seed: int, nrows: int, extra: int = 0, spd: bool = False):
    if kind == "banded":
        return banded(seed, nrows, extra, spd=spd)
    if kind == "powerlaw":
        return powerlaw(seed, nrows, spd=spd)
    if kind == "uniform":
        return uniform(seed, nrows, spd=spd)
    raise ValueError(kind)
