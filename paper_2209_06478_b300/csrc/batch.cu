// Batched execution over many matrices (the batch and serving workloads):
// one persistent launch per phase covers the row tiles of every matrix in
// the batch, each matrix in its own format (DIA, ELL or CSR) and tile shape.
//
//  - A slot holds one matrix (a dynmat handle, not owned) and its shape.
//  - Tiles: DIA / ELL row ranges; CSR row blocks of about `nnz_per_tile`
//    entries, summed either by the segmented tile (lanes = 0: a fixed run of
//    8 entries per lane, rows completed by scans) or with `lanes` lanes
//    per row, in which case every CSR row longer than `nnz_per_tile` gets a
//    tile of its own reduced by the whole block.
//  - A persistent grid (resident blocks x 148 SMs) takes tiles from an
//    atomic counter; per-tile work is fixed, so results do not depend on
//    which block runs which tile.
//  - Tile lists and tile counts live in device memory: a graph captured once
//    stays valid while slots are admitted and retired.
//  - CG over the batch (serving): per-slot device state; each phase's dot
//    products are reduced per slot by the slot's last tile, in tile order,
//    so a slot's iterates are bit-identical whatever else shares the batch.
#include <algorithm>
#include <memory>
#include <vector>

#include "device.cuh"
#include "internal.cuh"

namespace dm {

namespace {

constexpr int BT = 256;

enum TileKind : int32_t { TK_DIA = 0, TK_ELL = 1, TK_CSR = 2, TK_CSR_LONG = 3, TK_VEC = 4 };

// Device descriptor of one slot.
struct SlotDesc {
  int32_t active;     // 1 while the slot takes part in launches
  int32_t fmt;        // DYNMAT_DIA / ELL / CSR
  int32_t vdt;        // matrix value type
  int32_t xdt;        // vector type
  int32_t lanes;      // CSR lanes per row
  int32_t ndiag;
  int32_t off_min, off_max;
  int64_t N, M, ld, K;
  int64_t nnz_per_tile;
  const void* val;
  const int32_t* col;
  const int32_t* rowptr;
  const int32_t* offs;
  void* x;            // SpMV input / CG x
  void* y;            // SpMV output
  void* r;            // CG vectors (type xdt)
  void* p;
  void* q;
  double* part_a;     // per-tile partials, SpMV phase
  double* part_b;     // per-tile partials, vector phase
  int32_t ntiles_a, ntiles_b;
  CgState st;         // st.counter: SpMV-phase ticket
  uint32_t counter_b; // vector-phase ticket
  int32_t mode;       // 0 plain SpMV, 1 CG
  int32_t reliable;   // CG with reliable updates: x/r/p/q are the FP32 CG, folds go to x64
  double* x64;        // reliable: FP64 solution
  const double* b64;  // reliable: right-hand side
  double* q64;        // reliable: A x64 after a fold
};

struct Tile {
  int32_t slot;
  int32_t kind;
  int32_t idx;        // tile index within its slot (partials)
  int32_t pad;
  int64_t r0, r1;     // row range (CSR long: r0 = the row)
};

template <class V> struct BVec;
template <> struct BVec<double> { using T = double2; static constexpr int R = 2; };
template <> struct BVec<float> { using T = float4; static constexpr int R = 4; };

__device__ __forceinline__ void unpack2(const double2& v, double* o) { o[0] = v.x; o[1] = v.y; }
__device__ __forceinline__ void unpack2(const float4& v, float* o) {
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}

template <class X>
__device__ __forceinline__ X bfma(X a, X b, X c) { return fma(a, b, c); }

// ---- per-kind tile bodies; each returns the thread's share of y.x ----------
// (DOT: the CG product phase; otherwise the share is 0 and x is not re-read)

__device__ __forceinline__ void unpack_col(const int2& c, int32_t* o) { o[0] = c.x; o[1] = c.y; }
__device__ __forceinline__ void unpack_col(const int4& c, int32_t* o) {
  o[0] = c.x; o[1] = c.y; o[2] = c.z; o[3] = c.w;
}
template <int R> struct CVec;
template <> struct CVec<2> { using T = int2; };
template <> struct CVec<4> { using T = int4; };

// DIA rows [r0, r1): R consecutive rows per thread (one 16-byte load of each
// diagonal), diagonals in ascending order, U diagonals' loads in flight.
// Tile bodies are out of line so that each is register-allocated on its own
// within the persistent kernel's budget.
template <class V, class X, bool DOT>
__device__ __noinline__ double tile_dia(const SlotDesc& sd, int64_t r0, int64_t r1, const X* __restrict__ x,
                           X* __restrict__ y) {
  using VT = typename BVec<V>::T;
  constexpr int R = BVec<V>::R;
  constexpr int U = R == 2 ? 4 : 2;
  const V* __restrict__ dval = (const V*)sd.val;
  const int32_t* __restrict__ offs = sd.offs;
  const int64_t N = sd.N, M = sd.M, ld = sd.ld;
  const int nd = sd.ndiag;
  const bool interior = (r0 + sd.off_min >= 0) && (r1 - 1 + sd.off_max < M);
  double part = 0.0;
  for (int64_t i = r0 + (int64_t)threadIdx.x * R; i < r1; i += (int64_t)BT * R) {
    X acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = X(0);
    if (interior && i + R <= r1) {
      int d = 0;
      for (; d + U <= nd; d += U) {
        V v[U][R];
        X xv[U][R];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int64_t j = i + __ldg(offs + d + u);
          unpack2(__ldcs(reinterpret_cast<const VT*>(dval + (int64_t)(d + u) * ld + i)), v[u]);
#pragma unroll
          for (int r = 0; r < R; ++r) xv[u][r] = __ldg(x + j + r);
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int r = 0; r < R; ++r) acc[r] = bfma(X(v[u][r]), xv[u][r], acc[r]);
      }
      for (; d < nd; ++d) {
        const int64_t j = i + __ldg(offs + d);
        V v[R];
        unpack2(__ldcs(reinterpret_cast<const VT*>(dval + (int64_t)d * ld + i)), v);
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = bfma(X(v[r]), __ldg(x + j + r), acc[r]);
      }
    } else {
      for (int d = 0; d < nd; ++d) {
        const int64_t j = i + __ldg(offs + d);
        V v[R];
        unpack2(__ldcs(reinterpret_cast<const VT*>(dval + (int64_t)d * ld + i)), v);
#pragma unroll
        for (int r = 0; r < R; ++r)
          if (j + r >= 0 && j + r < M && i + r < r1) acc[r] = bfma(X(v[r]), __ldg(x + j + r), acc[r]);
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (i + r < r1 && i + r < N) {
        y[i + r] = acc[r];
        if (DOT) part = fma((double)acc[r], (double)x[i + r], part);
      }
  }
  return part;
}

// ELL rows [r0, r1): R consecutive rows per thread, slots in order, U
// slots' loads in flight; padding (col -1) is skipped. Rows in [N, ld) are
// padding, so the vector loads past the last row stay inside the arrays.
template <class V, class X, bool DOT>
__device__ __noinline__ double tile_ell(const SlotDesc& sd, int64_t r0, int64_t r1, const X* __restrict__ x,
                           X* __restrict__ y) {
  using VT = typename BVec<V>::T;
  constexpr int R = BVec<V>::R;
  using CT = typename CVec<R>::T;
  constexpr int U = R == 2 ? 4 : 2;
  const V* __restrict__ evl = (const V*)sd.val;
  const int32_t* __restrict__ ecol = sd.col;
  const int64_t ld = sd.ld, K = sd.K;
  double part = 0.0;
  for (int64_t i = r0 + (int64_t)threadIdx.x * R; i < r1; i += (int64_t)BT * R) {
    X acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = X(0);
    int64_t k = 0;
    for (; k + U <= K; k += U) {
      V v[U][R];
      int32_t c[U][R];
      X xv[U][R];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        unpack2(__ldcs(reinterpret_cast<const VT*>(evl + (k + u) * ld + i)), v[u]);
        unpack_col(__ldcs(reinterpret_cast<const CT*>(ecol + (k + u) * ld + i)), c[u]);
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int r = 0; r < R; ++r) xv[u][r] = c[u][r] >= 0 ? __ldg(x + c[u][r]) : X(0);
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int r = 0; r < R; ++r)
          if (c[u][r] >= 0) acc[r] = bfma(X(v[u][r]), xv[u][r], acc[r]);
    }
    for (; k < K; ++k) {
      V v[R];
      int32_t c[R];
      unpack2(__ldcs(reinterpret_cast<const VT*>(evl + k * ld + i)), v);
      unpack_col(__ldcs(reinterpret_cast<const CT*>(ecol + k * ld + i)), c);
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (c[r] >= 0) acc[r] = bfma(X(v[r]), __ldg(x + c[r]), acc[r]);
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (i + r < r1) {
        y[i + r] = acc[r];
        if (DOT) part = fma((double)acc[r], (double)x[i + r], part);
      }
  }
  return part;
}

// Short CSR rows of [r0, r1): groups of L lanes per row; rows longer than
// nnz_per_tile belong to their own long-row tile and are skipped here.
template <class V, class X, int L, bool DOT>
__device__ __noinline__ double tile_csr(const SlotDesc& sd, int64_t r0, int64_t r1, const X* __restrict__ x,
                           X* __restrict__ y) {
  constexpr int G = BT / L;
  const V* __restrict__ val = (const V*)sd.val;
  const int g = threadIdx.x / L, k = threadIdx.x % L;
  double part = 0.0;
  for (int64_t base = r0; base < r1; base += G) {
    const int64_t i = base + g;
    const bool active = i < r1;
    int32_t a = active ? __ldg(sd.rowptr + i) : 0, b = active ? __ldg(sd.rowptr + i + 1) : 0;
    const bool longrow = (int64_t)(b - a) > sd.nnz_per_tile;
    if (longrow) b = a;
    X acc = X(0);
    // four entries per lane per step: their columns and values are loaded
    // together, then the four gathers, then the multiply-adds in entry order
    int32_t e = a + k;
    for (; e + 3 * L < b; e += 4 * L) {
      int32_t cc[4];
      V vv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        cc[u] = __ldcs(sd.col + e + u * L);
        vv[u] = __ldcs(val + e + u * L);
      }
      X xv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) xv[u] = __ldg(x + cc[u]);
#pragma unroll
      for (int u = 0; u < 4; ++u) acc = bfma(X(vv[u]), xv[u], acc);
    }
    for (; e < b; e += L) acc = bfma(X(__ldcs(val + e)), __ldg(x + __ldcs(sd.col + e)), acc);
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, L);
    if (k == 0 && active && !longrow) {
      y[i] = acc;
      if (DOT) part = fma((double)acc, (double)x[i], part);
    }
  }
  return part;
}

// One long CSR row: the block strides its entries, then a fixed-tree sum.
template <class V, class X, bool DOT>
__device__ __noinline__ double tile_csr_long(const SlotDesc& sd, int64_t row, const X* __restrict__ x,
                                X* __restrict__ y, double* scratch) {
  const V* __restrict__ val = (const V*)sd.val;
  const int32_t a = __ldg(sd.rowptr + row), b = __ldg(sd.rowptr + row + 1);
  X acc = X(0);
  for (int32_t e = a + threadIdx.x; e < b; e += BT)
    acc = bfma(X(__ldcs(val + e)), __ldg(x + __ldcs(sd.col + e)), acc);
  const double s = block_sum((double)acc, scratch);
  // The row sum is formed in double from the per-thread partials; for FP32
  // vectors it is rounded to float once at the end.
  double part = 0.0;
  if (threadIdx.x == 0) {
    const X v = X(s);
    y[row] = v;
    if (DOT) part = (double)v * (double)x[row];
  }
  return part;
}

// ---- segmented CSR tile (lanes = 0) -------------------------------------------
// The tile's entries [E0, E1) are cut into runs of SEG_VPT entries on a grid
// aligned to SEG_VPT, so that each run's values and column indices are whole
// 16-byte words. Each warp takes a contiguous range of runs and walks it in
// chunks of 32 runs, lane l taking run l of the chunk:
//  - the lane loads its run's values and columns with vector loads and issues
//    all its x gathers before the first multiply-add;
//  - the warp finds the rows that start inside the chunk from the row
//    pointers (32 rows per step) and marks each start in a per-warp table of
//    the chunk's positions;
//  - the lane sums its entries in order, writing every row that starts and
//    ends inside its run; its first and last pieces are combined with the
//    other lanes' by a segmented scan over the lanes, with as many steps as
//    the longest row spans lanes, and the open row at the chunk's end is
//    carried into the next chunk;
//  - rows that cross the warps' ranges are closed after one block barrier, in
//    warp order.
// Every row is written once, in an order fixed by the tile: deterministic, and
// balanced whatever the row lengths. Empty rows are written 0 in a pass over
// the tile's row pointers, which also stages them in shared memory.
constexpr int SEG_VPT = 8;
constexpr int SEG_W = BT / 32;
constexpr int SEG_CHUNK = 32 * SEG_VPT;
constexpr int SEG_RCAP = 1023;

struct SegShared {
  alignas(16) int32_t rowid[SEG_W][SEG_CHUNK];  // per warp: row starting at each chunk position, or -1
  int32_t rp[SEG_RCAP + 1];                     // the tile's row pointers when it has at most SEG_RCAP rows
  double hf[SEG_W];                             // per warp: its first row's sum, when closed inside the warp
  double tl[SEG_W];                             // per warp: the sum of its open row at its end
  int32_t f[SEG_W], t[SEG_W];                   // per warp: first and last row (tile-relative)
  int32_t closed[SEG_W], nonempty[SEG_W];
};

// One run (8 entries starting at a multiple of 8, so 32-byte aligned) as
// 32-byte loads: every load takes whole 32-byte sectors, so no sector is
// fetched twice whatever L1 keeps between a lane's loads.
__device__ __forceinline__ void load_run(const double* p, double* o) {
#pragma unroll
  for (int i = 0; i < SEG_VPT / 4; ++i)
    asm("ld.global.nc.v4.f64 {%0,%1,%2,%3}, [%4];"
                 : "=d"(o[4 * i]), "=d"(o[4 * i + 1]), "=d"(o[4 * i + 2]), "=d"(o[4 * i + 3])
                 : "l"(p + 4 * i));
}
__device__ __forceinline__ void load_run(const float* p, float* o) {
  asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=f"(o[0]), "=f"(o[1]), "=f"(o[2]), "=f"(o[3]), "=f"(o[4]), "=f"(o[5]), "=f"(o[6]),
                 "=f"(o[7])
               : "l"(p));
}
__device__ __forceinline__ void load_run(const int32_t* p, int32_t* o) {
  asm("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(o[0]), "=r"(o[1]), "=r"(o[2]), "=r"(o[3]), "=r"(o[4]), "=r"(o[5]), "=r"(o[6]),
                 "=r"(o[7])
               : "l"(p));
}

template <class V, class X, bool DOT>
__device__ __noinline__ double tile_csr_seg(const SlotDesc& sd, int64_t r0, int64_t r1, const X* __restrict__ x,
                                            X* __restrict__ y, SegShared& sm) {
  constexpr unsigned FULL = 0xffffffffu;
  const V* __restrict__ val = (const V*)sd.val;
  const int32_t* __restrict__ col = sd.col;
  const int32_t* __restrict__ rowptr = sd.rowptr + r0;
  X* __restrict__ yt = y + r0;
  const X* __restrict__ xt = x + r0;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int32_t nrows = (int32_t)(r1 - r0);
  const bool rp_shared = nrows <= SEG_RCAP;
  double part = 0.0;
  // empty rows, and the row pointers to shared memory
  for (int32_t i = tid; i <= nrows; i += BT) {
    const int32_t s = __ldg(rowptr + i);
    if (rp_shared) sm.rp[i] = s;
    if (i < nrows && s == __ldg(rowptr + i + 1)) yt[i] = X(0);
  }
  __syncthreads();
  auto RP = [&](int32_t i) -> int32_t { return rp_shared ? sm.rp[i] : __ldg(rowptr + i); };
  const int32_t E0 = RP(0), E1 = RP(nrows);
  if (E0 == E1) return part;
  const int32_t a = E0 & ~(SEG_VPT - 1);
  const int32_t nruns = (E1 - a + SEG_VPT - 1) / SEG_VPT;
  // whole chunks of 32 runs per warp: the first nch % SEG_W warps take one
  // more, so that warps left without a chunk come last
  const int32_t nch = (nruns + 31) >> 5;
  const int32_t cb = nch / SEG_W, cx = nch % SEG_W;
  const int32_t wc0 = w * cb + min(w, cx);
  const int32_t wr0 = min(nruns, 32 * wc0);
  const int32_t wr1 = min(nruns, 32 * (wc0 + cb + (w < cx ? 1 : 0)));
  if (wr0 < wr1) {
    const int32_t wlo = max(E0, a + wr0 * SEG_VPT), whi = min(E1, a + wr1 * SEG_VPT);
    // the row holding wlo: the last row starting at or before it (32 probes a step)
    int32_t lo = 0, hi = nrows;
    while (hi - lo > 1) {
      const int32_t step = (hi - lo + 31) >> 5;
      const int32_t m = lo + lane * step;
      const unsigned b = __ballot_sync(FULL, m < hi && RP(m) <= wlo);
      lo += (31 - __clz(b)) * step;
      hi = min(hi, lo + step);
    }
    int32_t rc = lo;  // the open row at the chunk's start
    int32_t rend = RP(lo + 1);  // its end
    const int32_t first_row = lo;
    bool first_open = true;  // the warp's first row not yet closed inside the warp
    X carry = X(0);
    // Chunks that lie inside the open row (no row starts in them) skip the
    // scan: each lane keeps its own running sum, folded into the carry by a
    // butterfly sum when the row ends (the same bits in every lane).
    X pend = X(0);
    bool pending = false;
    auto fold = [&]() {
      X t = pend;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t = t + __shfl_xor_sync(FULL, t, o);
      carry = carry + t;
      pend = X(0);
      pending = false;
    };
    int32_t* rid_w = sm.rowid[w];
    for (int32_t cr = wr0; cr < wr1; cr += 32) {
      const int32_t pbase = a + cr * SEG_VPT;
      const int32_t eb = pbase + lane * SEG_VPT;
      const int32_t cend = min(whi, pbase + SEG_CHUNK);
      // valid entries of the run: [wlo, whi) (only the tile's and the warp's
      // first and last runs are partial)
      const bool full = eb >= wlo && eb + SEG_VPT <= whi;
      V v[SEG_VPT];
      int32_t c[SEG_VPT];
      X xg[SEG_VPT];
      if (full) {
        load_run(val + eb, v);
        load_run(col + eb, c);
#pragma unroll
        for (int k = 0; k < SEG_VPT; ++k) xg[k] = __ldg(x + c[k]);
      } else {
#pragma unroll
        for (int k = 0; k < SEG_VPT; ++k) {
          const bool in = eb + k >= wlo && eb + k < whi;
          v[k] = in ? __ldg(val + eb + k) : V(0);
          xg[k] = in ? __ldg(x + __ldg(col + eb + k)) : X(0);
        }
      }
      if (rend >= cend) {  // the open row covers the chunk
#pragma unroll
        for (int k = 0; k < SEG_VPT; ++k) pend = bfma(X(v[k]), xg[k], pend);
        pending = true;
        continue;
      }
      if (pending) fold();
      // rows starting in the chunk: rows after rc whose first entry is before cend
      reinterpret_cast<int4*>(rid_w)[2 * lane] = make_int4(-1, -1, -1, -1);
      reinterpret_cast<int4*>(rid_w)[2 * lane + 1] = make_int4(-1, -1, -1, -1);
      __syncwarp();
      for (int32_t rr = rc + 1 + lane;; rr += 32) {
        const bool in = rr < nrows;
        const int32_t s = in ? RP(rr) : E1;
        const int32_t s1 = in ? RP(rr + 1) : E1;
        if (in && s1 > s && s < cend) rid_w[s - pbase] = rr;
        if (!__shfl_sync(FULL, in && s1 < cend, 31)) break;
      }
      __syncwarp();
      int32_t rid[SEG_VPT];
      {
        const int4 p0 = reinterpret_cast<const int4*>(rid_w)[2 * lane];
        const int4 p1 = reinterpret_cast<const int4*>(rid_w)[2 * lane + 1];
        rid[0] = p0.x; rid[1] = p0.y; rid[2] = p0.z; rid[3] = p0.w;
        rid[4] = p1.x; rid[5] = p1.y; rid[6] = p1.z; rid[7] = p1.w;
      }
      // the run's entries in order (invalid entries add 0 x 0); rows inside
      // the run are written here
      X acc = X(0), head = X(0);
      int32_t lastrow = -1;
      bool seen = false;
#pragma unroll
      for (int k = 0; k < SEG_VPT; ++k) {
        if (rid[k] >= 0) {
          if (!seen) {
            head = acc;
            seen = true;
          } else {
            yt[lastrow] = acc;
            if (DOT) part = fma((double)acc, (double)xt[lastrow], part);
          }
          acc = X(0);
          lastrow = rid[k];
        }
        acc = bfma(X(v[k]), xg[k], acc);
      }
      // segmented scan over the lanes: a lane's last piece belongs to the row
      // started by the nearest lane at or before it that saw a row start, or
      // to the carried row (key -1) when there is none
      const unsigned bs = __ballot_sync(FULL, seen);
      const unsigned le = bs & (FULL >> (31 - lane));
      const int j = le ? 31 - __clz(le) : -1;
      const int32_t kj = __shfl_sync(FULL, lastrow, j < 0 ? 0 : j);
      const int32_t key = j < 0 ? -1 : kj;
      const int span = lane - (j < 0 ? 0 : j);
      const int maxspan = __reduce_max_sync(FULL, (unsigned)span);
      X s = acc;
      if (lane == 0 && !seen) s = carry + s;
      for (int o = 1; o <= maxspan; o <<= 1) {
        const X s2 = __shfl_up_sync(FULL, s, o);
        if (span >= o) s = s2 + s;
      }
      // a lane that saw a row start closes the row before it
      const X sp = __shfl_up_sync(FULL, s, 1);
      const int32_t kp = __shfl_up_sync(FULL, key, 1);
      if (seen) {
        const bool carried = lane == 0 || kp < 0;
        const X tot = (lane == 0 ? carry : sp) + head;
        if (carried && first_open) {
          sm.hf[w] = (double)tot;
        } else {
          const int32_t row = carried ? rc : kp;
          yt[row] = tot;
          if (DOT) part = fma((double)tot, (double)xt[row], part);
        }
      }
      const int32_t k31 = __shfl_sync(FULL, key, 31);
      carry = __shfl_sync(FULL, s, 31);
      if (k31 >= 0) {
        rc = k31;
        rend = RP(rc + 1);
        first_open = false;
      }
    }
    if (pending) fold();
    if (lane == 0) {
      sm.f[w] = first_row;
      sm.t[w] = rc;
      sm.tl[w] = (double)carry;
      sm.closed[w] = first_open ? 0 : 1;
      sm.nonempty[w] = 1;
    }
  } else if (lane == 0) {
    sm.nonempty[w] = 0;
  }
  __syncthreads();
  // rows crossing the warps' ranges, in warp order (empty warps come last)
  if (tid < SEG_W && sm.nonempty[tid]) {
    auto close = [&](int32_t row, X v, bool chain) {
      if (chain)
        for (int u = tid - 1; u >= 0 && sm.t[u] == row; --u) {
          v = X(sm.tl[u]) + v;
          if (sm.closed[u]) break;
        }
      yt[row] = v;
      if (DOT) part = fma((double)v, (double)xt[row], part);
    };
    const bool closed = sm.closed[tid] != 0;
    if (closed) close(sm.f[tid], X(sm.hf[tid]), true);
    const bool last = tid == SEG_W - 1 || !sm.nonempty[tid + 1];
    if (last || sm.f[tid + 1] != sm.t[tid]) close(sm.t[tid], X(sm.tl[tid]), !closed);
  }
  return part;
}

template <class V, class X, bool DOT>
__device__ double run_tile(const SlotDesc& sd, const Tile& t, const X* x, X* y, double* scratch,
                           SegShared& sm) {
  switch (t.kind) {
    case TK_DIA: return tile_dia<V, X, DOT>(sd, t.r0, t.r1, x, y);
    case TK_ELL: return tile_ell<V, X, DOT>(sd, t.r0, t.r1, x, y);
    case TK_CSR:
      switch (sd.lanes) {
        case 0: return tile_csr_seg<V, X, DOT>(sd, t.r0, t.r1, x, y, sm);
        case 2: return tile_csr<V, X, 2, DOT>(sd, t.r0, t.r1, x, y);
        case 4: return tile_csr<V, X, 4, DOT>(sd, t.r0, t.r1, x, y);
        case 8: return tile_csr<V, X, 8, DOT>(sd, t.r0, t.r1, x, y);
        case 16: return tile_csr<V, X, 16, DOT>(sd, t.r0, t.r1, x, y);
        default: return tile_csr<V, X, 32, DOT>(sd, t.r0, t.r1, x, y);
      }
    default: return tile_csr_long<V, X, DOT>(sd, t.r0, x, y, scratch);
  }
}

// The slot's last tile to finish sums the slot's partials in tile order and
// applies `op` to the slot's CG state.
__device__ void slot_finish(SlotDesc* sd, double* partials, int ntiles, uint32_t* counter, int op,
                            double* scratch) {
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned t = atomicAdd(counter, 1u);
    last = (t == (unsigned)ntiles - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s = 0.0;
  const volatile double* pp = partials;
  for (int i = threadIdx.x; i < ntiles; i += BT) s += pp[i];
  s = block_sum(s, scratch);
  if (threadIdx.x == 0) {
    cg_apply(&sd->st, op, s);
    *counter = 0;
    __threadfence();
  }
  __syncthreads();
}

__device__ __forceinline__ bool take_tile(unsigned* next, int64_t total, int64_t* t) {
  __shared__ int64_t tk;
  __syncthreads();
  if (threadIdx.x == 0) tk = (int64_t)atomicAdd(next, 1u);
  __syncthreads();
  *t = tk;
  return tk < total;
}

// SpMV phase over every active slot. mode 0: y = A x. mode 1 (CG): q = A p
// with p.q reduced per slot (alpha, or breakdown). mode 2: for reliable-update
// slots with a fold due, q64 = A x64 (FP32 values, FP64 vectors and sums).
constexpr int SPMV_BLOCKS_PER_SM = 4;

__global__ void __launch_bounds__(BT, SPMV_BLOCKS_PER_SM)
batch_spmv_kernel(SlotDesc* __restrict__ slots, const Tile* __restrict__ tiles,
                  const int64_t* __restrict__ ntiles, unsigned* __restrict__ next, int mode) {
  __shared__ double scratch[BT];
  __shared__ SegShared seg;
  const int64_t total = *ntiles;
  int64_t ti;
  while (take_tile(next, total, &ti)) {
    const Tile t = tiles[ti];
    SlotDesc* sd = slots + t.slot;
    if (!sd->active || (mode >= 1 && sd->st.done)) continue;
    if (mode == 2) {
      if (!sd->reliable || sd->st.skip_fold) continue;
      run_tile<float, double, false>(*sd, t, sd->x64, sd->q64, scratch, seg);
      continue;
    }
    if (mode == 0) {
      if (sd->vdt == DYNMAT_F64)
        run_tile<double, double, false>(*sd, t, (const double*)sd->x, (double*)sd->y, scratch, seg);
      else if (sd->xdt == DYNMAT_F32)
        run_tile<float, float, false>(*sd, t, (const float*)sd->x, (float*)sd->y, scratch, seg);
      else
        run_tile<float, double, false>(*sd, t, (const double*)sd->x, (double*)sd->y, scratch, seg);
      continue;
    }
    double part;
    if (sd->vdt == DYNMAT_F64)
      part = run_tile<double, double, true>(*sd, t, (const double*)sd->p, (double*)sd->q, scratch, seg);
    else if (sd->xdt == DYNMAT_F32)
      part = run_tile<float, float, true>(*sd, t, (const float*)sd->p, (float*)sd->q, scratch, seg);
    else
      part = run_tile<float, double, true>(*sd, t, (const double*)sd->p, (double*)sd->q, scratch, seg);
    {
      const double s = t.kind == TK_CSR_LONG ? part : block_sum(part, scratch);
      if (threadIdx.x == 0) sd->part_a[t.idx] = s;
      slot_finish(sd, sd->part_a, sd->ntiles_a, &sd->st.counter, DOT_CG_PQ, scratch);
    }
  }
}

// CG vector phase: x += alpha p, r -= alpha q, r.r per slot (-> beta, test).
template <class X>
__device__ double update_rows(SlotDesc* sd, int64_t r0, int64_t r1) {
  X* __restrict__ x = (X*)sd->x;
  X* __restrict__ r = (X*)sd->r;
  const X* __restrict__ p = (const X*)sd->p;
  const X* __restrict__ q = (const X*)sd->q;
  const X a = (X)sd->st.alpha;
  double part = 0.0;
  for (int64_t i = r0 + threadIdx.x; i < r1; i += BT) {
    x[i] = fma(a, p[i], x[i]);
    const X ri = fma(-a, q[i], r[i]);
    r[i] = ri;
    part = fma((double)ri, (double)ri, part);
  }
  return part;
}

__global__ void __launch_bounds__(BT)
batch_update_kernel(SlotDesc* __restrict__ slots, const Tile* __restrict__ tiles,
                    const int64_t* __restrict__ ntiles, unsigned* __restrict__ next) {
  __shared__ double scratch[BT];
  const int64_t total = *ntiles;
  int64_t ti;
  while (take_tile(next, total, &ti)) {
    const Tile t = tiles[ti];
    SlotDesc* sd = slots + t.slot;
    if (!sd->active || sd->st.done) continue;
    const double part = sd->xdt == DYNMAT_F64 ? update_rows<double>(sd, t.r0, t.r1)
                                              : update_rows<float>(sd, t.r0, t.r1);
    const double s = block_sum(part, scratch);
    if (threadIdx.x == 0) sd->part_b[t.idx] = s;
    slot_finish(sd, sd->part_b, sd->ntiles_b, &sd->counter_b,
                sd->reliable ? DOT_RU_RR : DOT_CG_RR, scratch);
  }
}

// Reliable updates, fold (slots with a fold due): x64 += (double) d; d = 0.
__global__ void __launch_bounds__(BT)
batch_fold_kernel(SlotDesc* __restrict__ slots, const Tile* __restrict__ tiles,
                  const int64_t* __restrict__ ntiles, unsigned* __restrict__ next) {
  const int64_t total = *ntiles;
  int64_t ti;
  while (take_tile(next, total, &ti)) {
    const Tile t = tiles[ti];
    SlotDesc* sd = slots + t.slot;
    if (!sd->active || !sd->reliable || sd->st.done || sd->st.skip_fold) continue;
    double* __restrict__ x = sd->x64;
    float* __restrict__ d = (float*)sd->x;
    for (int64_t i = t.r0 + threadIdx.x; i < t.r1; i += BT) {
      x[i] = x[i] + (double)d[i];
      d[i] = 0.0f;
    }
  }
}

// After the fold's product: r = b - q64 (FP64), r32 = (float) r, r.r in
// FP64 reduced per slot (test against tol, beta).
__global__ void __launch_bounds__(BT)
batch_fold_residual_kernel(SlotDesc* __restrict__ slots, const Tile* __restrict__ tiles,
                           const int64_t* __restrict__ ntiles, unsigned* __restrict__ next) {
  __shared__ double scratch[BT];
  const int64_t total = *ntiles;
  int64_t ti;
  while (take_tile(next, total, &ti)) {
    const Tile t = tiles[ti];
    SlotDesc* sd = slots + t.slot;
    if (!sd->active || !sd->reliable || sd->st.done || sd->st.skip_fold) continue;
    const double* __restrict__ b = sd->b64;
    const double* __restrict__ q = sd->q64;
    float* __restrict__ r32 = (float*)sd->r;
    double part = 0.0;
    for (int64_t i = t.r0 + threadIdx.x; i < t.r1; i += BT) {
      const double ri = b[i] - q[i];
      r32[i] = (float)ri;
      part = fma(ri, ri, part);
    }
    const double s = block_sum(part, scratch);
    if (threadIdx.x == 0) sd->part_b[t.idx] = s;
    slot_finish(sd, sd->part_b, sd->ntiles_b, &sd->counter_b, DOT_RU_FOLD, scratch);
  }
}

template <class X>
__device__ void direction_rows(SlotDesc* sd, int64_t r0, int64_t r1) {
  X* __restrict__ p = (X*)sd->p;
  const X* __restrict__ r = (const X*)sd->r;
  const X b = (X)sd->st.beta;
  for (int64_t i = r0 + threadIdx.x; i < r1; i += BT) p[i] = fma(b, p[i], r[i]);
}

__global__ void __launch_bounds__(BT)
batch_direction_kernel(SlotDesc* __restrict__ slots, const Tile* __restrict__ tiles,
                       const int64_t* __restrict__ ntiles, unsigned* __restrict__ next) {
  const int64_t total = *ntiles;
  int64_t ti;
  while (take_tile(next, total, &ti)) {
    const Tile t = tiles[ti];
    SlotDesc* sd = slots + t.slot;
    if (!sd->active || sd->st.done) continue;
    if (sd->xdt == DYNMAT_F64) direction_rows<double>(sd, t.r0, t.r1);
    else direction_rows<float>(sd, t.r0, t.r1);
  }
}

// CSR tiles of one slot: row blocks by entry count, plus one tile per long row.
__global__ void csr_tiles_kernel(const int32_t* __restrict__ rowptr, int64_t N, int64_t nnz,
                                 int64_t E, int32_t slot, int64_t nblocks, Tile* __restrict__ out) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nblocks) return;
  auto lower = [&](int64_t e) {  // first row r with rowptr[r] >= e (r in [0, N])
    int64_t lo = 0, hi = N;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (rowptr[mid] < e) lo = mid + 1; else hi = mid;
    }
    return lo;
  };
  const int64_t r0 = b == 0 ? 0 : lower(b * E);
  const int64_t r1 = b == nblocks - 1 ? N : lower((b + 1) * E);
  Tile t;
  t.slot = slot;
  t.kind = TK_CSR;
  t.idx = (int32_t)b;
  t.pad = 0;
  t.r0 = r0;
  t.r1 = max(r0, r1);
  out[b] = t;
}

__global__ void long_rows_kernel(const int32_t* __restrict__ rowptr, int64_t N, int64_t E,
                                 int32_t slot, int32_t idx0, unsigned* __restrict__ count,
                                 Tile* __restrict__ out, int64_t cap) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  if ((int64_t)(rowptr[i + 1] - rowptr[i]) > E) {
    const unsigned k = atomicAdd(count, 1u);
    if ((int64_t)k < cap) {
      Tile t;
      t.slot = slot;
      t.kind = TK_CSR_LONG;
      t.idx = -1;  // set in order by long_rows_order_kernel
      t.pad = 0;
      t.r0 = i;
      t.r1 = i + 1;
      out[k] = t;
    }
  }
}

// Long-row tiles were appended in arbitrary order: give them their partial
// index by row order so the per-slot reduction order is fixed.
__global__ void long_rows_order_kernel(Tile* __restrict__ t, int64_t n, int32_t idx0) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t rank = 0;
  for (int64_t j = 0; j < n; ++j) rank += t[j].r0 < t[i].r0;
  t[i].idx = idx0 + (int32_t)rank;
}

__global__ void long_rows_count_kernel(const int32_t* __restrict__ rowptr, int64_t N, int64_t E,
                                       unsigned* __restrict__ count) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N && (int64_t)(rowptr[i + 1] - rowptr[i]) > E) atomicAdd(count, 1u);
}

int resident(const void* fn) {
  int b = 0;
  DM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, BT, 0));
  return std::max(1, b) * device().sms;
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct BatchSlot {
  dynmat_s* A = nullptr;
  dynmat_tile_shape shape{};
  int mode = 0;            // 0 SpMV, 1 CG
  int precision = CG_FP64;
  // CG work (owned): r, p, q in the vector type; partials; for mixed the
  // FP32 inner vectors and the FP64 residual.
  DBuf work;
  double* part_a = nullptr;
  double* part_b = nullptr;
  int64_t ntiles_a = 0, ntiles_b = 0;
  void* cx = nullptr;      // CG iterate (FP64 user x, or FP32 inner correction)
  void* r = nullptr;
  void* p = nullptr;
  void* q = nullptr;
  const double* b = nullptr;  // user right-hand side
  double* x64 = nullptr;      // user solution vector
  double* r64 = nullptr;      // mixed: FP64 residual
  double* q64 = nullptr;      // mixed: FP64 A x
  double bnorm = 0;
  cg_opts opts{};
  int outer = 0, inner_total = 0, fp64_iters = 0;
  int status = DYNMAT_OK;
  bool finished = false;
  bool paused = false;     // CG slot left out of cg_batch_step (cg_batch_pause)
  double rel = 0;
  // SpMV mode vectors
  const void* sx = nullptr;
  void* sy = nullptr;
};

}  // namespace dm

struct dynmat_batch_s {
  int32_t max_slots = 0;
  std::vector<dm::BatchSlot> slots;
  dm::DBuf d_slots;      // SlotDesc[max_slots]
  dm::DBuf d_tiles_a;    // Tile[]
  dm::DBuf d_tiles_b;
  dm::DBuf d_meta;       // int64 ntiles_a, ntiles_b; unsigned counters[4]
  int64_t cap_a = 0, cap_b = 0;
  bool dirty = true;
  int grid_spmv = 0, grid_upd = 0, grid_dir = 0;
  bool has_reliable = false;  // some slot runs reliable updates: graphs carry fold phases
  // graphs: SpMV (mode 0) and one CG iteration x k
  cudaGraphExec_t g_spmv = nullptr;
  cudaGraphExec_t g_cg = nullptr;
  int g_cg_iters = 0;
  cudaStream_t s = nullptr;
};

namespace dm {
namespace {

constexpr int64_t VEC_TILE_ROWS = 4096;

int64_t* meta_counts(dynmat_batch_s* B) { return B->d_meta.as<int64_t>(); }
unsigned* meta_next(dynmat_batch_s* B) { return (unsigned*)(B->d_meta.as<int64_t>() + 2); }

void check_slot(dynmat_batch_s* B, int32_t slot) {
  DM_REQUIRE(B, DYNMAT_ERR_INVALID_ARG, "null batch");
  DM_REQUIRE(slot >= 0 && slot < B->max_slots, DYNMAT_ERR_INVALID_ARG, "slot %d out of range",
             slot);
}

// Shape defaults: DIA/ELL 2048-row tiles; CSR row blocks of about 4096
// entries summed by the segmented tile (any row-length mix).
dynmat_tile_shape default_shape(const dynmat_s*) {
  dynmat_tile_shape s{};
  s.rows_per_tile = 2048;
  s.nnz_per_tile = 16384;
  s.lanes = 0;
  return s;
}

void validate_shape(const dynmat_tile_shape& s) {
  DM_REQUIRE(s.lanes == 0 || s.lanes == 2 || s.lanes == 4 || s.lanes == 8 || s.lanes == 16 ||
                 s.lanes == 32,
             DYNMAT_ERR_INVALID_ARG, "lanes must be 0, 2, 4, 8, 16 or 32");
  DM_REQUIRE(s.rows_per_tile >= 1024 && s.rows_per_tile % 1024 == 0, DYNMAT_ERR_INVALID_ARG,
             "rows_per_tile must be a positive multiple of 1024");
  DM_REQUIRE(s.nnz_per_tile >= 256, DYNMAT_ERR_INVALID_ARG, "nnz_per_tile must be >= 256");
}

SlotDesc make_desc(const BatchSlot& S) {
  SlotDesc d{};
  const dynmat_s* A = S.A;
  d.active = (A && !S.paused) ? 1 : 0;
  if (!A) return d;
  d.fmt = A->fmt;
  d.vdt = A->vdt;
  d.N = A->nrows;
  d.M = A->ncols;
  d.lanes = S.shape.lanes;
  d.nnz_per_tile = S.shape.nnz_per_tile;
  switch (A->fmt) {
    case DYNMAT_DIA:
      d.val = A->dia.val.p;
      d.offs = A->dia.offsets.as<int32_t>();
      d.ndiag = (int32_t)A->dia.ndiag;
      d.off_min = A->dia.off_min;
      d.off_max = A->dia.off_max;
      d.ld = A->dia.ld;
      break;
    case DYNMAT_ELL:
      d.val = A->ell.val.p;
      d.col = A->ell.col.as<int32_t>();
      d.ld = A->ell.ld;
      d.K = A->ell.K;
      break;
    default:
      d.val = A->csr.val.p;
      d.col = A->csr.col.as<int32_t>();
      d.rowptr = A->csr.rowptr.as<int32_t>();
      break;
  }
  d.mode = S.mode;
  if (S.mode == 0) {
    d.xdt = A->vdt;
    d.x = const_cast<void*>(S.sx);
    d.y = S.sy;
  } else {
    d.xdt = S.precision == CG_FP64 ? DYNMAT_F64 : DYNMAT_F32;
    d.x = S.cx;
    d.r = S.r;
    d.p = S.p;
    d.q = S.q;
    if (S.precision == CG_MIXED_RELIABLE) {
      d.reliable = 1;
      d.x64 = S.x64;
      d.b64 = S.b;
      d.q64 = S.q64;
    }
  }
  d.part_a = S.part_a;
  d.part_b = S.part_b;
  d.ntiles_a = (int32_t)S.ntiles_a;
  d.ntiles_b = (int32_t)S.ntiles_b;
  return d;
}

// Number of SpMV tiles of a slot (CSR: row blocks, plus one tile per long
// row unless the segmented tile takes every row; blocking).
int64_t count_tiles_a(const BatchSlot& S, int64_t* nlong, cudaStream_t s) {
  const dynmat_s* A = S.A;
  *nlong = 0;
  if (A->nrows == 0) return 0;
  if (A->fmt != DYNMAT_CSR) return cdiv(A->nrows, S.shape.rows_per_tile);
  const int64_t E = S.shape.nnz_per_tile;
  if (S.shape.lanes == 0) return std::max<int64_t>(1, cdiv(A->csr.nnz, E));
  DBuf cnt(4, s);
  DM_CUDA(cudaMemsetAsync(cnt.p, 0, 4, s));
  long_rows_count_kernel<<<(unsigned)cdiv(A->nrows, BT), BT, 0, s>>>(
      A->csr.rowptr.as<int32_t>(), A->nrows, E, cnt.as<unsigned>());
  DM_CHECK_LAUNCH();
  unsigned h = 0;
  DM_CUDA(cudaMemcpyAsync(&h, cnt.p, 4, cudaMemcpyDeviceToHost, s));
  DM_CUDA(cudaStreamSynchronize(s));
  *nlong = h;
  return std::max<int64_t>(1, cdiv(A->csr.nnz, E)) + h;
}

void drop_graphs(dynmat_batch_s* B);

// Rebuilds descriptors and tile lists of all slots (blocking). The tile
// arrays may move, so every captured graph (whose kernels hold their
// addresses) is dropped first; the next launch captures again.
void rebuild(dynmat_batch_s* B, cudaStream_t s) {
  DM_CUDA(cudaStreamSynchronize(s));
  drop_graphs(B);
  std::vector<Tile> host_a, host_b;
  std::vector<int64_t> csr_off(B->max_slots, -1), csr_blocks(B->max_slots, 0),
      csr_long(B->max_slots, 0);
  for (int k = 0; k < B->max_slots; ++k) {
    BatchSlot& S = B->slots[k];
    if (!S.A || S.finished) continue;
    const dynmat_s* A = S.A;
    int64_t nlong = 0;
    const int64_t na = count_tiles_a(S, &nlong, s);
    DM_REQUIRE(na == S.ntiles_a || S.mode == 0, DYNMAT_ERR_INVALID_ARG, "tile count changed");
    if (A->fmt == DYNMAT_CSR) {
      csr_off[k] = (int64_t)host_a.size();
      csr_blocks[k] = na - nlong;
      csr_long[k] = nlong;
      host_a.resize(host_a.size() + na);  // filled on the device
    } else {
      for (int64_t t = 0; t < na; ++t) {
        Tile ti{};
        ti.slot = k;
        ti.kind = A->fmt == DYNMAT_DIA ? TK_DIA : TK_ELL;
        ti.idx = (int32_t)t;
        ti.r0 = t * S.shape.rows_per_tile;
        ti.r1 = std::min<int64_t>(A->nrows, ti.r0 + S.shape.rows_per_tile);
        host_a.push_back(ti);
      }
    }
    if (S.mode == 1) {
      for (int64_t t = 0; t < S.ntiles_b; ++t) {
        Tile ti{};
        ti.slot = k;
        ti.kind = TK_VEC;
        ti.idx = (int32_t)t;
        ti.r0 = t * VEC_TILE_ROWS;
        ti.r1 = std::min<int64_t>(A->nrows, ti.r0 + VEC_TILE_ROWS);
        host_b.push_back(ti);
      }
    }
  }
  const int64_t na = (int64_t)host_a.size(), nb = (int64_t)host_b.size();
  if (na > B->cap_a) {
    B->d_tiles_a.alloc(std::max<int64_t>(na, 1) * sizeof(Tile), s);
    B->cap_a = na;
  }
  if (nb > B->cap_b) {
    B->d_tiles_b.alloc(std::max<int64_t>(nb, 1) * sizeof(Tile), s);
    B->cap_b = nb;
  }
  if (na) DM_CUDA(cudaMemcpyAsync(B->d_tiles_a.p, host_a.data(), na * sizeof(Tile),
                                  cudaMemcpyHostToDevice, s));
  if (nb) DM_CUDA(cudaMemcpyAsync(B->d_tiles_b.p, host_b.data(), nb * sizeof(Tile),
                                  cudaMemcpyHostToDevice, s));
  // CSR tiles computed on the device from the row pointers.
  for (int k = 0; k < B->max_slots; ++k) {
    if (csr_off[k] < 0) continue;
    BatchSlot& S = B->slots[k];
    const dynmat_s* A = S.A;
    Tile* base = B->d_tiles_a.as<Tile>() + csr_off[k];
    const int64_t nbk = csr_blocks[k];
    csr_tiles_kernel<<<(unsigned)cdiv(nbk, BT), BT, 0, s>>>(
        A->csr.rowptr.as<int32_t>(), A->nrows, A->csr.nnz, S.shape.nnz_per_tile, k, nbk, base);
    DM_CHECK_LAUNCH();
    if (csr_long[k]) {
      DBuf cnt(4, s);
      DM_CUDA(cudaMemsetAsync(cnt.p, 0, 4, s));
      long_rows_kernel<<<(unsigned)cdiv(A->nrows, BT), BT, 0, s>>>(
          A->csr.rowptr.as<int32_t>(), A->nrows, S.shape.nnz_per_tile, k, (int32_t)nbk,
          cnt.as<unsigned>(), base + nbk, csr_long[k]);
      DM_CHECK_LAUNCH();
      long_rows_order_kernel<<<(unsigned)cdiv(csr_long[k], BT), BT, 0, s>>>(base + nbk,
                                                                          csr_long[k], (int32_t)nbk);
      DM_CHECK_LAUNCH();
    }
  }
  // Running CG slots keep their device-side state (scalars, tickets).
  std::vector<SlotDesc> old(B->max_slots), descs(B->max_slots);
  DM_CUDA(cudaMemcpyAsync(old.data(), B->d_slots.p, old.size() * sizeof(SlotDesc),
                          cudaMemcpyDeviceToHost, s));
  DM_CUDA(cudaStreamSynchronize(s));
  B->has_reliable = false;
  for (int k = 0; k < B->max_slots; ++k) {
    BatchSlot& S = B->slots[k];
    descs[k] = S.finished ? SlotDesc{} : make_desc(S);
    if (S.A && S.mode == 1 && !S.finished) {
      descs[k].st = old[k].st;
      descs[k].counter_b = old[k].counter_b;
      if (S.precision == CG_MIXED_RELIABLE) B->has_reliable = true;
    }
  }
  DM_CUDA(cudaMemcpyAsync(B->d_slots.p, descs.data(), descs.size() * sizeof(SlotDesc),
                          cudaMemcpyHostToDevice, s));
  int64_t counts[2] = {na, nb};
  DM_CUDA(cudaMemcpyAsync(meta_counts(B), counts, sizeof counts, cudaMemcpyHostToDevice, s));
  DM_CUDA(cudaMemsetAsync(meta_next(B), 0, 4 * sizeof(unsigned), s));
  DM_CUDA(cudaStreamSynchronize(s));
  B->dirty = false;
}

// Kernels reading the current lists; counters reset by memset nodes.
void enqueue_spmv(dynmat_batch_s* B, int mode, cudaStream_t s) {
  DM_CUDA(cudaMemsetAsync(meta_next(B), 0, sizeof(unsigned), s));
  batch_spmv_kernel<<<B->grid_spmv, BT, 0, s>>>(B->d_slots.as<SlotDesc>(),
                                                B->d_tiles_a.as<Tile>(), meta_counts(B),
                                                meta_next(B), mode);
  DM_CHECK_LAUNCH();
}

void enqueue_cg_iteration(dynmat_batch_s* B, cudaStream_t s) {
  enqueue_spmv(B, 1, s);
  DM_CUDA(cudaMemsetAsync(meta_next(B) + 1, 0, sizeof(unsigned), s));
  batch_update_kernel<<<B->grid_upd, BT, 0, s>>>(B->d_slots.as<SlotDesc>(), B->d_tiles_b.as<Tile>(),
                                                 meta_counts(B) + 1, meta_next(B) + 1);
  DM_CHECK_LAUNCH();
  if (B->has_reliable) {
    // folds of reliable-update slots that asked for one (others skip)
    DM_CUDA(cudaMemsetAsync(meta_next(B) + 2, 0, sizeof(unsigned), s));
    batch_fold_kernel<<<B->grid_dir, BT, 0, s>>>(B->d_slots.as<SlotDesc>(),
                                                 B->d_tiles_b.as<Tile>(), meta_counts(B) + 1,
                                                 meta_next(B) + 2);
    DM_CHECK_LAUNCH();
    enqueue_spmv(B, 2, s);
    DM_CUDA(cudaMemsetAsync(meta_next(B) + 1, 0, sizeof(unsigned), s));
    batch_fold_residual_kernel<<<B->grid_upd, BT, 0, s>>>(
        B->d_slots.as<SlotDesc>(), B->d_tiles_b.as<Tile>(), meta_counts(B) + 1, meta_next(B) + 1);
    DM_CHECK_LAUNCH();
  }
  DM_CUDA(cudaMemsetAsync(meta_next(B) + 2, 0, sizeof(unsigned), s));
  batch_direction_kernel<<<B->grid_dir, BT, 0, s>>>(B->d_slots.as<SlotDesc>(),
                                                    B->d_tiles_b.as<Tile>(), meta_counts(B) + 1,
                                                    meta_next(B) + 2);
  DM_CHECK_LAUNCH();
}

cudaGraphExec_t capture(dynmat_batch_s* B, int what, int iters, cudaStream_t s) {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  DM_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  try {
    if (what == 0) enqueue_spmv(B, 0, s);
    else for (int k = 0; k < iters; ++k) enqueue_cg_iteration(B, s);
  } catch (...) {
    cudaStreamEndCapture(s, &g);
    if (g) cudaGraphDestroy(g);
    throw;
  }
  DM_CUDA(cudaStreamEndCapture(s, &g));
  const cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphDestroy(g);
  DM_CUDA(e);
  return ge;
}

// The batch's own stream (capture needs a non-default stream), ordered with
// the caller's stream by events on entry and exit.
struct Ordered {
  cudaStream_t user, own;
  cudaEvent_t ev;
  Ordered(dynmat_batch_s* B, cudaStream_t u) : user(u), own(B->s) {
    DM_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    DM_CUDA(cudaEventRecord(ev, user));
    DM_CUDA(cudaStreamWaitEvent(own, ev, 0));
  }
  ~Ordered() {
    cudaEventRecord(ev, own);
    cudaStreamWaitEvent(user, ev, 0);
    cudaEventDestroy(ev);
  }
};

void drop_graphs(dynmat_batch_s* B) {
  if (B->g_spmv) cudaGraphExecDestroy(B->g_spmv);
  if (B->g_cg) cudaGraphExecDestroy(B->g_cg);
  B->g_spmv = B->g_cg = nullptr;
  B->g_cg_iters = 0;
}

// ---- CG slots ----------------------------------------------------------------

struct StateHost {
  CgState st;
};

CgState read_slot_state(dynmat_batch_s* B, int slot, cudaStream_t s) {
  static thread_local CgState* h = nullptr;
  if (!h) DM_CUDA(cudaMallocHost((void**)&h, sizeof(CgState)));
  const SlotDesc* d = B->d_slots.as<SlotDesc>() + slot;
  DM_CUDA(cudaMemcpyAsync(h, (const char*)d + offsetof(SlotDesc, st), sizeof(CgState),
                          cudaMemcpyDeviceToHost, s));
  DM_CUDA(cudaStreamSynchronize(s));
  return *h;
}

void write_slot_state(dynmat_batch_s* B, int slot, const CgState& st, cudaStream_t s) {
  SlotDesc* d = B->d_slots.as<SlotDesc>() + slot;
  DM_CUDA(cudaMemcpyAsync((char*)d + offsetof(SlotDesc, st), &st, sizeof(CgState),
                          cudaMemcpyHostToDevice, s));
  DM_CUDA(cudaStreamSynchronize(s));
}

void set_slot_active(dynmat_batch_s* B, int slot, int active, cudaStream_t s) {
  SlotDesc* d = B->d_slots.as<SlotDesc>() + slot;
  DM_CUDA(cudaMemcpyAsync((char*)d + offsetof(SlotDesc, active), &active, 4,
                          cudaMemcpyHostToDevice, s));
}

}  // namespace

// Per-matrix helpers shared with cg.cu (defined there). `part` holds one
// double per tile of A's plan, `aux_state` one CgState; both blocking.
// Partial sums that A's reducing kernels can write: one per block, and no
// grid exceeds the plan's tile count or 8 blocks per SM.
inline int64_t dot_parts(const dynmat_s* A) {
  return std::max<int64_t>(A->plan.ntiles, 8 * (int64_t)device().sms);
}
double batch_residual(const dynmat_s* A, const double* b, const double* x, double* r,
                      double* q, float* r32, float* d32, float* p32, double* part,
                      CgState* aux_state, bool inner_init, cudaStream_t s);
double batch_dot(const dynmat_s* A, const double* a, const double* b, double* part,
                 CgState* aux_state, cudaStream_t s);
void batch_add_correction(int64_t N, double* x, const float* d, cudaStream_t s);
double batch_ru_init(const dynmat_s* A, const double* b, float* r32, float* p32, float* d32,
                     double* part, CgState* aux_state, cudaStream_t s);

}  // namespace dm

using namespace dm;

extern "C" {

dynmat_status dynmat_batch_create(dynmat_batch_t* out, int32_t max_slots, dynmat_stream_t stream) {
  return dm::guard([&] {
    DM_REQUIRE(out && max_slots > 0 && max_slots <= 65536, DYNMAT_ERR_INVALID_ARG,
               "bad batch size");
    cudaStream_t s = (cudaStream_t)stream;
    device();
    auto B = std::make_unique<dynmat_batch_s>();
    B->max_slots = max_slots;
    B->slots.resize(max_slots);
    B->d_slots.alloc(max_slots * sizeof(SlotDesc), s);
    DM_CUDA(cudaMemsetAsync(B->d_slots.p, 0, max_slots * sizeof(SlotDesc), s));
    B->d_meta.alloc(64, s);
    DM_CUDA(cudaMemsetAsync(B->d_meta.p, 0, 64, s));
    DM_CUDA(cudaStreamCreateWithFlags(&B->s, cudaStreamNonBlocking));
    // The x gathers live on L1: ask for the smallest shared-memory carveout
    // that still holds the resident blocks (and their 1 KB reserve each).
    {
      cudaFuncAttributes fa;
      DM_CUDA(cudaFuncGetAttributes(&fa, (const void*)batch_spmv_kernel));
      int smem_sm = 0;
      DM_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor,
                                     device().id));
      const size_t need = (size_t)SPMV_BLOCKS_PER_SM * (fa.sharedSizeBytes + 1024);
      const int pct = (int)std::min<size_t>(100, (100 * need + smem_sm - 1) / std::max(smem_sm, 1));
      DM_CUDA(cudaFuncSetAttribute((const void*)batch_spmv_kernel,
                                   cudaFuncAttributePreferredSharedMemoryCarveout, pct));
    }
    B->grid_spmv = resident((const void*)batch_spmv_kernel);
    B->grid_upd = resident((const void*)batch_update_kernel);
    B->grid_dir = resident((const void*)batch_direction_kernel);
    DM_CUDA(cudaStreamSynchronize(s));
    *out = B.release();
  });
}

dynmat_status dynmat_batch_destroy(dynmat_batch_t B, dynmat_stream_t stream) {
  return dm::guard([&] {
    if (!B) return;
    cudaStream_t s = (cudaStream_t)stream;
    DM_CUDA(cudaStreamSynchronize(B->s));
    drop_graphs(B);
    for (auto& S : B->slots) {
      S.work.s = s;
      S.work.release();
    }
    B->d_slots.s = B->d_tiles_a.s = B->d_tiles_b.s = B->d_meta.s = s;
    cudaStreamDestroy(B->s);
    delete B;
  });
}

dynmat_status dynmat_batch_set(dynmat_batch_t B, int32_t slot, dynmat_t A,
                               const dynmat_tile_shape* shape, const void* x, void* y,
                               dynmat_stream_t stream) {
  return dm::guard([&] {
    check_slot(B, slot);
    BatchSlot& S = B->slots[slot];
    DM_REQUIRE(S.mode == 0 || !S.A, DYNMAT_ERR_INVALID_ARG, "slot %d holds a CG solve", slot);
    if (!A) {
      S = BatchSlot{};
      B->dirty = true;
      return;
    }
    DM_REQUIRE(A->fmt == DYNMAT_DIA || A->fmt == DYNMAT_ELL || A->fmt == DYNMAT_CSR,
               DYNMAT_ERR_INVALID_ARG, "batched formats are DIA, ELL and CSR");
    // the segmented CSR tile indexes its 8-entry runs in 32 bits, up to 7
    // entries past the last one
    DM_REQUIRE(A->fmt != DYNMAT_CSR || A->csr.nnz <= INT32_MAX - 64, DYNMAT_ERR_INVALID_ARG,
               "a batched CSR matrix holds at most 2^31 - 65 entries");
    DM_REQUIRE(A->nrows == 0 || (x && y), DYNMAT_ERR_INVALID_ARG, "null vector");
    dynmat_tile_shape sh = shape ? *shape : default_shape(A);
    validate_shape(sh);
    S.A = A;
    S.shape = sh;
    S.mode = 0;
    S.sx = x;
    S.sy = y;
    S.finished = false;
    B->dirty = true;
  });
}

dynmat_status dynmat_batch_spmv(dynmat_batch_t B, dynmat_stream_t stream) {
  return dm::guard([&] {
    DM_REQUIRE(B, DYNMAT_ERR_INVALID_ARG, "null batch");
    cudaStream_t s = (cudaStream_t)stream;
    Ordered o(B, s);
    if (B->dirty) {
      rebuild(B, B->s);
      drop_graphs(B);
    }
    if (!B->g_spmv) B->g_spmv = capture(B, 0, 1, B->s);
    DM_CUDA(cudaGraphLaunch(B->g_spmv, B->s));
  });
}

// A copy of A's active-format arrays (DIA, ELL or CSR) and its plan, so that
// tuner copies do not read one another's data from L2.
std::unique_ptr<dynmat_s> clone_active(const dynmat_s* A, cudaStream_t s) {
  auto C = std::make_unique<dynmat_s>();
  C->nrows = A->nrows;
  C->ncols = A->ncols;
  C->nnz = A->nnz;
  C->fmt = A->fmt;
  C->vdt = A->vdt;
  C->plan = A->plan;
  auto dup = [&](DBuf& d, const DBuf& src) {
    if (!src.p) return;
    d.alloc(src.bytes, s);
    DM_CUDA(cudaMemcpyAsync(d.p, src.p, src.bytes, cudaMemcpyDeviceToDevice, s));
  };
  switch (A->fmt) {
    case DYNMAT_DIA:
      C->dia.ndiag = A->dia.ndiag;
      C->dia.ld = A->dia.ld;
      C->dia.off_min = A->dia.off_min;
      C->dia.off_max = A->dia.off_max;
      dup(C->dia.offsets, A->dia.offsets);
      dup(C->dia.val, A->dia.val);
      break;
    case DYNMAT_ELL:
      C->ell.K = A->ell.K;
      C->ell.ld = A->ell.ld;
      dup(C->ell.col, A->ell.col);
      dup(C->ell.val, A->ell.val);
      break;
    default:
      C->csr.nnz = A->csr.nnz;
      C->csr.maxlen = A->csr.maxlen;
      dup(C->csr.rowptr, A->csr.rowptr);
      dup(C->csr.col, A->csr.col);
      dup(C->csr.val, A->csr.val);
      break;
  }
  return C;
}

size_t active_bytes(const dynmat_s* A) {
  switch (A->fmt) {
    case DYNMAT_DIA: return A->dia.val.bytes + A->dia.offsets.bytes;
    case DYNMAT_ELL: return A->ell.val.bytes + A->ell.col.bytes;
    default: return A->csr.val.bytes + A->csr.col.bytes + A->csr.rowptr.bytes;
  }
}

}  // extern "C"

namespace dm {
// The batch tuner (§V-E's profiling tuner, run online for the batch): times
// A in the persistent batch kernel for every candidate (format among DIA,
// ELL, CSR within the padding guard; tile shape) and converts A to the
// fastest, returning its shape. A lone small matrix cannot fill the GPU, and
// the shape that is fastest alone (many small tiles) is not the one that is
// fastest inside a full batch; so A is timed as `copies` slots, about
// `target_rows` rows in all, each with its own x, y and (up to 2 GB of clones)
// matrix arrays, as distinct matrices of a batch have. effort 0 (short
// probe): the format only, each in its default tile shape (smaller tiles can
// win a plain product yet lose in CG, where every tile adds a dot partial),
// copies of 1M rows; effort 1 (full): every shape, 4M rows. Each candidate:
// 3 timed runs after 2 warm-ups.
void tune_for_batch(dynmat_s* A, const void* x_in, int effort, dynmat_format* fmt_out,
                    dynmat_tile_shape* shape_out, cudaStream_t s) {
  dynmat_features f;
  compute_features(A, 3, &f, s);
  const int64_t target_rows = effort ? 4000000 : 1000000;
  const int copies = (int)std::min<int64_t>(
      64, std::max<int64_t>(1, cdiv(target_rows, std::max<int64_t>(A->nrows, 1))));
  DBuf ycopies((size_t)copies * std::max<int64_t>(A->nrows, 1) * vsize(A->vdt), s);
  // each copy multiplies its own x (as distinct matrices of a batch do)
  const size_t xbytes = (size_t)std::max<int64_t>(A->ncols, 1) * vsize(A->vdt);
  DBuf xcopies((size_t)copies * xbytes, s);
  if (x_in) {
    for (int k = 0; k < copies; ++k)
      DM_CUDA(cudaMemcpyAsync((char*)xcopies.p + k * xbytes, x_in, A->ncols * vsize(A->vdt),
                              cudaMemcpyDeviceToDevice, s));
  } else {
    DM_CUDA(cudaMemsetAsync(xcopies.p, 0, (size_t)copies * xbytes, s));
  }
  dynmat_batch_t T = nullptr;
  if (dynmat_batch_create(&T, copies, s) != DYNMAT_OK) throw Fail{DYNMAT_ERR_CUDA};
  std::unique_ptr<dynmat_batch_s, void (*)(dynmat_batch_s*)> guardT(
      T, [](dynmat_batch_s* b) { dynmat_batch_destroy(b, nullptr); });
  cudaEvent_t e0, e1;
  DM_CUDA(cudaEventCreate(&e0));
  DM_CUDA(cudaEventCreate(&e1));
  double best = 1e30;
  dynmat_format bf = A->fmt;
  dynmat_tile_shape bs = default_shape(A);
  const dynmat_format cands[3] = {DYNMAT_DIA, DYNMAT_ELL, DYNMAT_CSR};
  for (dynmat_format fm : cands) {
    if ((fm == DYNMAT_DIA || fm == DYNMAT_ELL) && f.bytes[fm] > 3 * f.bytes[DYNMAT_CSR]) continue;
    try {
      convert_impl(A, fm, A->vdt, s);
    } catch (const Fail&) {
      clear_error();
      continue;
    }
    std::vector<std::unique_ptr<dynmat_s>> clones;
    const size_t mb = std::max<size_t>(active_bytes(A), 1);
    const int nclones = (int)std::min<size_t>(copies - 1, (size_t)(2ull << 30) / mb);
    for (int k = 0; k < nclones; ++k) clones.push_back(clone_active(A, s));
    auto copy_of = [&](int k) -> dynmat_s* {
      return k == 0 || clones.empty() ? A : clones[(k - 1) % clones.size()].get();
    };
    std::vector<dynmat_tile_shape> shapes;
    if (fm == DYNMAT_CSR) {
      if (effort) {
        for (int E : {2048, 4096, 8192, 16384}) shapes.push_back(dynmat_tile_shape{0, 2048, E});
        for (int L : {2, 4, 8, 16, 32}) shapes.push_back(dynmat_tile_shape{L, 2048, 4096});
      } else {
        shapes.push_back(default_shape(A));
      }
    } else if (effort) {
      // 1024-row tiles only. Timed alone, as copies of one matrix, larger
      // tiles could look as fast, but inside a batch they leave a long tail:
      // the 22 banded matrices of the 64-matrix batch (DIA) took 100, 151,
      // 287 and 552 us with 1024-, 2048-, 4096- and 8192-row tiles, the 21
      // uniform ones (ELL) 264, 304, 391 and 415 us.
      shapes.push_back(dynmat_tile_shape{8, 1024, 4096});
    } else {
      shapes.push_back(default_shape(A));
    }
    for (const auto& sh : shapes) {
      for (int k = 0; k < copies; ++k) {
        void* yk = (char*)ycopies.p + (size_t)k * A->nrows * vsize(A->vdt);
        const void* xk = (const char*)xcopies.p + k * xbytes;
        if (dynmat_batch_set(T, k, copy_of(k), &sh, xk, yk, s) != DYNMAT_OK)
          throw Fail{DYNMAT_ERR_CUDA};
      }
      std::vector<float> ts;
      for (int rep = 0; rep < 5; ++rep) {
        DM_CUDA(cudaEventRecord(e0, s));
        if (dynmat_batch_spmv(T, s) != DYNMAT_OK) throw Fail{DYNMAT_ERR_CUDA};
        DM_CUDA(cudaEventRecord(e1, s));
        DM_CUDA(cudaEventSynchronize(e1));
        float ms = 0;
        DM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (rep >= 2) ts.push_back(ms);
      }
      std::sort(ts.begin(), ts.end());
      // Another format must be 3% faster than the best so far (the formats
      // go DIA, ELL, CSR: fewest bytes first); shapes of one format compete
      // on the plain minimum. Without the margin, near-ties flipped with
      // timing noise: a banded matrix of the 64-matrix batch took ELL in one
      // run out of two, and the batch went from 639 to 661 us.
      const double t = ts[ts.size() / 2];
      if (t < (fm != bf && best < 1e30 ? 0.97 : 1.0) * best) {
        best = t;
        bf = fm;
        bs = sh;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  convert_impl(A, bf, A->vdt, s);
  if (fmt_out) *fmt_out = bf;
  if (shape_out) *shape_out = bs;
}
}  // namespace dm

extern "C" {

// The per-slot tuner of a batch (full effort, with the slot's own x).
dynmat_status dynmat_batch_autotune(dynmat_batch_t B, int32_t slot, dynmat_format* fmt_out,
                                    dynmat_tile_shape* shape_out, dynmat_stream_t stream) {
  return dm::guard([&] {
    check_slot(B, slot);
    BatchSlot& S = B->slots[slot];
    DM_REQUIRE(S.A && S.mode == 0, DYNMAT_ERR_INVALID_ARG, "slot %d has no SpMV matrix", slot);
    dynmat_format bf;
    dynmat_tile_shape bs;
    tune_for_batch(S.A, S.sx, 1, &bf, &bs, (cudaStream_t)stream);
    S.shape = bs;
    B->dirty = true;
    if (fmt_out) *fmt_out = bf;
    if (shape_out) *shape_out = bs;
  });
}

dynmat_status dynmat_batch_tune_matrix(dynmat_t A, int32_t effort, dynmat_format* fmt_out,
                                       dynmat_tile_shape* shape_out, dynmat_stream_t stream) {
  return dm::guard([&] {
    DM_REQUIRE(A, DYNMAT_ERR_INVALID_ARG, "null handle");
    DM_REQUIRE(effort == 0 || effort == 1, DYNMAT_ERR_INVALID_ARG, "effort must be 0 or 1");
    DM_REQUIRE(A->nrows > 0, DYNMAT_ERR_INVALID_ARG, "empty matrix");
    tune_for_batch(A, nullptr, effort, fmt_out, shape_out, (cudaStream_t)stream);
  });
}

// ---- CG over the batch ----------------------------------------------------

dynmat_status cg_batch_admit(dynmat_batch_t B, int32_t slot, dynmat_t A, const double* b,
                             double* x, const cg_opts* opts, const dynmat_tile_shape* shape,
                             dynmat_stream_t stream) {
  return dm::guard([&] {
    check_slot(B, slot);
    DM_REQUIRE(A && b && x && opts, DYNMAT_ERR_INVALID_ARG, "null argument");
    DM_REQUIRE(A->nrows == A->ncols && A->nrows > 0, DYNMAT_ERR_INVALID_ARG,
               "CG needs a non-empty square matrix");
    DM_REQUIRE(A->fmt == DYNMAT_DIA || A->fmt == DYNMAT_ELL || A->fmt == DYNMAT_CSR,
               DYNMAT_ERR_INVALID_ARG, "batched formats are DIA, ELL and CSR");
    // the segmented CSR tile indexes its 8-entry runs in 32 bits, up to 7
    // entries past the last one
    DM_REQUIRE(A->fmt != DYNMAT_CSR || A->csr.nnz <= INT32_MAX - 64, DYNMAT_ERR_INVALID_ARG,
               "a batched CSR matrix holds at most 2^31 - 65 entries");
    DM_REQUIRE(opts->precision == CG_FP64 || opts->precision == CG_MIXED ||
                   opts->precision == CG_MIXED_RELIABLE,
               DYNMAT_ERR_INVALID_ARG, "bad precision");
    DM_REQUIRE(opts->precision == CG_FP64 || A->vdt == DYNMAT_F32, DYNMAT_ERR_INVALID_ARG,
               "batched mixed precision needs a matrix with F32 values");
    DM_REQUIRE(opts->precision == CG_MIXED || A->vdt == DYNMAT_F64 || A->vdt == DYNMAT_F32,
               DYNMAT_ERR_INVALID_ARG, "bad value type");
    BatchSlot& S = B->slots[slot];
    DM_REQUIRE(!S.A, DYNMAT_ERR_INVALID_ARG, "slot %d is occupied", slot);
    cudaStream_t s = (cudaStream_t)stream;
    Ordered o(B, s);
    cudaStream_t bs = B->s;
    BatchSlot T;
    T.A = A;
    T.shape = shape ? *shape : default_shape(A);
    validate_shape(T.shape);
    T.mode = 1;
    T.precision = opts->precision;
    T.opts = *opts;
    T.b = b;
    T.x64 = x;
    const int64_t N = A->nrows;
    int64_t nlong = 0;
    T.ntiles_a = count_tiles_a(T, &nlong, bs);
    T.ntiles_b = cdiv(N, VEC_TILE_ROWS);
    const bool mixed = opts->precision != CG_FP64;  // FP32 CG vectors
    auto al = [](int64_t v) { return round_up(std::max<int64_t>(v, 16), 256); };
    const int64_t vb = mixed ? 4 : 8;
    int64_t need = al(T.ntiles_a * 8) + al(T.ntiles_b * 8) + 3 * al(N * vb) +
                   (mixed ? 2 * al(N * 8) + al(N * 4) + al(sizeof(CgState)) : 0);
    T.work.alloc(need, bs);  // OOM leaves the batch untouched
    char* p = (char*)T.work.p;
    T.part_a = (double*)p; p += al(T.ntiles_a * 8);
    T.part_b = (double*)p; p += al(T.ntiles_b * 8);
    T.r = p; p += al(N * vb);
    T.p = p; p += al(N * vb);
    T.q = p; p += al(N * vb);
    CgState st{};
    if (!mixed) {
      // FP64: CG from the caller's x (x0), initial r = b - A x0, p = r.
      T.cx = x;
      DBuf tmp(al(sizeof(CgState)) + al(dot_parts(A) * 8), bs);
      CgState* stp = tmp.as<CgState>();
      const double rr = batch_residual(A, b, x, (double*)T.r, (double*)T.q, nullptr, nullptr,
                                       nullptr, (double*)((char*)tmp.p + al(sizeof(CgState))),
                                       stp, false, bs);
      DM_CUDA(cudaMemcpyAsync(T.p, T.r, N * 8, cudaMemcpyDeviceToDevice, bs));
      st.tol = opts->tol;
      st.max_iters = opts->max_iters;
      st.rho = rr;
      st.r0 = std::sqrt(rr);
      st.rel = 1.0;
      if (st.r0 == 0.0) { st.done = 1; st.status = DYNMAT_OK; st.rel = 0.0; }
      else if (st.max_iters <= 0) { st.done = 1; st.status = DYNMAT_ERR_NOT_CONVERGED; }
    } else if (opts->precision == CG_MIXED_RELIABLE) {
      // Reliable updates: x = 0; r32 = p32 = (float) b, d = 0; rho = b.b.
      T.r64 = (double*)p; p += al(N * 8);  // unused
      T.q64 = (double*)p; p += al(N * 8);
      T.cx = p; p += al(N * 4);  // FP32 correction d
      CgState* aux = (CgState*)p;
      DM_CUDA(cudaMemsetAsync(x, 0, N * 8, bs));
      DBuf tmp(al(dot_parts(A) * 8), bs);
      const double bb = batch_ru_init(A, b, (float*)T.r, (float*)T.p, (float*)T.cx,
                                      tmp.as<double>(), aux, bs);
      st.tol = opts->tol;
      st.max_iters = opts->max_iters;
      st.delta = opts->delta > 0 ? opts->delta : 0.1;
      st.rho = bb;
      st.bnorm = st.rmax = st.r0 = std::sqrt(bb);
      st.rel = 1.0;
      st.skip_fold = 1;
      T.bnorm = st.bnorm;
      if (st.bnorm == 0.0) {
        st.done = 1;
        st.status = DYNMAT_OK;
        st.rel = 0.0;
      } else if (st.max_iters <= 0) {
        st.done = 1;
        st.status = DYNMAT_ERR_NOT_CONVERGED;
      }
    } else {
      // Mixed: x = 0; outer residual in FP64 and the first inner start.
      T.r64 = (double*)p; p += al(N * 8);
      T.q64 = (double*)p; p += al(N * 8);
      T.cx = p; p += al(N * 4);  // FP32 correction d
      CgState* aux = (CgState*)p;
      DM_CUDA(cudaMemsetAsync(x, 0, N * 8, bs));
      DBuf tmp(al(dot_parts(A) * 8), bs);
      T.bnorm = std::sqrt(batch_dot(A, b, b, tmp.as<double>(), aux, bs));
      const double rho0 = batch_residual(A, b, x, T.r64, T.q64, (float*)T.r, (float*)T.cx,
                                         (float*)T.p, tmp.as<double>(), aux, true, bs);
      T.rel = 1.0;
      st.tol = opts->inner_tol;
      st.max_iters = opts->max_iters;
      st.rho = rho0;
      st.r0 = std::sqrt(rho0);
      st.rel = 1.0;
      T.outer = 1;
      if (T.bnorm == 0.0) {
        st.done = 1;
        st.status = DYNMAT_OK;
        T.finished = true;
        T.status = DYNMAT_OK;
        T.rel = 0.0;
      } else if (st.r0 == 0.0) {
        st.done = 1;
      }
    }
    S = std::move(T);
    rebuild(B, bs);  // descriptors now include the slot
    write_slot_state(B, slot, st, bs);
  });
}

// Advances every active CG slot by `iterations` iterations (one graph
// launch), then completes outer refinement steps of mixed slots whose inner
// solve finished. done_flags (host, max_slots entries, may be NULL) receive 1
// for slots whose solve is over. *n_active receives the slots still running.
dynmat_status cg_batch_step(dynmat_batch_t B, int32_t iterations, int32_t* done_flags,
                            int32_t* n_active, dynmat_stream_t stream) {
  return dm::guard([&] {
    DM_REQUIRE(B && iterations > 0, DYNMAT_ERR_INVALID_ARG, "bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    Ordered o(B, s);
    cudaStream_t bs = B->s;
    if (B->dirty) {
      rebuild(B, bs);
      drop_graphs(B);
    }
    if (!B->g_cg || B->g_cg_iters != iterations) {
      if (B->g_cg) cudaGraphExecDestroy(B->g_cg);
      B->g_cg = nullptr;
      B->g_cg = capture(B, 1, iterations, bs);
      B->g_cg_iters = iterations;
    }
    DM_CUDA(cudaGraphLaunch(B->g_cg, bs));
    // Read back every slot's state in one copy.
    static thread_local std::vector<SlotDesc> hd;
    hd.resize(B->max_slots);
    DM_CUDA(cudaMemcpyAsync(hd.data(), B->d_slots.p, B->max_slots * sizeof(SlotDesc),
                            cudaMemcpyDeviceToHost, bs));
    DM_CUDA(cudaStreamSynchronize(bs));
    int active = 0;
    for (int k = 0; k < B->max_slots; ++k) {
      BatchSlot& S = B->slots[k];
      if (done_flags) done_flags[k] = 0;
      if (!S.A || S.mode != 1) continue;
      if (S.finished) {
        if (done_flags) done_flags[k] = 1;
        continue;
      }
      const CgState& st = hd[k].st;
      if (!st.done) {
        ++active;
        continue;
      }
      if (S.precision == CG_FP64 || S.precision == CG_MIXED_RELIABLE) {
        S.finished = true;
        S.status = st.status;
        S.fp64_iters = st.iter;
        S.outer = st.folds;
        S.rel = st.rel;
      } else {
        // inner solve over: x += d, new FP64 residual, next inner start
        S.inner_total += st.iter;
        const int64_t N = S.A->nrows;
        batch_add_correction(N, S.x64, (const float*)S.cx, bs);
        DBuf tmp(round_up(dot_parts(S.A) * 8, 256) + 256, bs);
        CgState* aux = tmp.as<CgState>();
        double* part = (double*)((char*)tmp.p + 256);
        const double rr = batch_residual(S.A, S.b, S.x64, S.r64, S.q64, nullptr, nullptr,
                                         nullptr, part, aux, false, bs);
        S.rel = S.bnorm > 0 ? std::sqrt(rr) / S.bnorm : std::sqrt(rr);
        if (S.rel <= S.opts.tol) {
          S.finished = true;
          S.status = DYNMAT_OK;
        } else if (S.outer >= S.opts.max_outer || st.status == DYNMAT_ERR_BREAKDOWN) {
          S.finished = true;
          S.status = st.status == DYNMAT_ERR_BREAKDOWN ? DYNMAT_ERR_BREAKDOWN
                                                       : DYNMAT_ERR_NOT_CONVERGED;
        } else {
          const double rho0 = batch_residual(S.A, S.b, S.x64, S.r64, S.q64, (float*)S.r,
                                             (float*)S.cx, (float*)S.p, part, aux, true, bs);
          CgState ns{};
          ns.tol = S.opts.inner_tol;
          ns.max_iters = S.opts.max_iters;
          ns.rho = rho0;
          ns.r0 = std::sqrt(rho0);
          ns.rel = 1.0;
          if (ns.r0 == 0.0) ns.done = 1;
          ++S.outer;
          write_slot_state(B, k, ns, bs);
          ++active;
          continue;
        }
      }
      if (S.finished) {
        if (done_flags) done_flags[k] = 1;
        set_slot_active(B, k, 0, bs);
      }
    }
    DM_CUDA(cudaStreamSynchronize(bs));
    if (n_active) *n_active = active;
  });
}

dynmat_status cg_batch_result(dynmat_batch_t B, int32_t slot, cg_result* res,
                              dynmat_stream_t stream) {
  return dm::guard([&] {
    check_slot(B, slot);
    DM_REQUIRE(res, DYNMAT_ERR_INVALID_ARG, "null result");
    BatchSlot& S = B->slots[slot];
    DM_REQUIRE(S.A && S.mode == 1, DYNMAT_ERR_INVALID_ARG, "slot %d holds no CG solve", slot);
    memset(res, 0, sizeof *res);
    cudaStream_t s = (cudaStream_t)stream;
    Ordered o(B, s);
    if (!S.finished) {
      const CgState st = read_slot_state(B, slot, B->s);
      res->status = -1;  // still running
      res->iterations = S.precision == CG_MIXED ? S.inner_total + st.iter : st.iter;
      res->rel_residual = S.precision == CG_MIXED ? S.rel : st.rel;
      return;
    }
    res->status = S.status;
    res->iterations = S.precision == CG_MIXED ? S.inner_total : S.fp64_iters;
    res->outer_iterations = S.precision == CG_FP64 ? 0 : S.outer;
    res->rel_residual = S.rel;
    // true residual ||b - A x|| / ||b|| in FP64
    const int64_t N = S.A->nrows;
    const int64_t pb = round_up(dot_parts(S.A) * 8, 256);
    DBuf tmp(256 + pb + 2 * round_up(N * 8, 256), B->s);
    CgState* aux = tmp.as<CgState>();
    double* part = (double*)((char*)tmp.p + 256);
    double* r = (double*)((char*)tmp.p + 256 + pb);
    double* q = r + round_up(N * 8, 256) / 8;
    const double rr = batch_residual(S.A, S.b, S.x64, r, q, nullptr, nullptr, nullptr, part, aux,
                                     false, B->s);
    const double bb = batch_dot(S.A, S.b, S.b, part, aux, B->s);
    res->true_rel_residual = bb > 0 ? std::sqrt(rr) / std::sqrt(bb) : std::sqrt(rr);
  });
}

// Leaves a running CG slot out of the following steps (paused = 1), or takes
// it back (0). Every phase kernel skips an inactive slot, so its state does
// not move while it is paused and its iterates are the same bits, only
// later. The descriptor's flag is written on the batch's stream, before
// the next step's graph launch.
dynmat_status cg_batch_pause(dynmat_batch_t B, int32_t slot, int32_t paused,
                             dynmat_stream_t stream) {
  return dm::guard([&] {
    check_slot(B, slot);
    DM_REQUIRE(paused == 0 || paused == 1, DYNMAT_ERR_INVALID_ARG, "paused must be 0 or 1");
    BatchSlot& S = B->slots[slot];
    DM_REQUIRE(S.A && S.mode == 1, DYNMAT_ERR_INVALID_ARG, "slot %d holds no CG solve", slot);
    if (S.finished || S.paused == (paused != 0)) return;
    Ordered o(B, (cudaStream_t)stream);
    S.paused = paused != 0;
    set_slot_active(B, slot, paused ? 0 : 1, B->s);
  });
}

dynmat_status cg_batch_retire(dynmat_batch_t B, int32_t slot, dynmat_stream_t stream) {
  return dm::guard([&] {
    check_slot(B, slot);
    cudaStream_t s = (cudaStream_t)stream;
    Ordered o(B, s);
    BatchSlot& S = B->slots[slot];
    if (!S.A) return;
    set_slot_active(B, slot, 0, B->s);
    DM_CUDA(cudaStreamSynchronize(B->s));
    S.work.s = B->s;
    S = BatchSlot{};
    B->dirty = true;
  });
}

}  // extern "C"
