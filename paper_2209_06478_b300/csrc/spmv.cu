// SpMV y = A x for every format (§III-D "multiply", one kernel per format as
// the paper's CUDA backend has), written for sm_103a.
//
// Every kernel moves 8-16 bytes per fused multiply-add. With FP32 values
// that makes them HBM-bound. With FP64 values on B300, whose FP64 pipe
// retires 2 DFMA per clock per SM (about 0.6 T DFMA/s), the DFMA rate is as
// tight as HBM (DIA: 8.6 bytes per DFMA, bound by the FP64 pipe), so every
// FP64 kernel spends exactly one DFMA per stored entry and no other FP64
// instruction in its inner loop. Common design:
//  - matrix arrays are read once with 16-byte vector loads and a streaming
//    cache hint, so they do not evict the reused x vector from the 126 MB L2;
//  - x is read through the read-only path (L1 / L2 hits for its reuse);
//  - grids are sized from the occupancy of each kernel times the 148 SMs,
//    with a grid-stride loop over fixed row tiles;
//  - each row's sum has exactly one writer and every reduction has a fixed
//    order, so results do not depend on scheduling.
// Row-based kernels (DIA, ELL, CSR-vector) can fuse the dot product p.(A p)
// of CG into their epilogue (one partial per row tile, reduced by the last
// block in index order).
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <type_traits>
#include <vector>
#include <unordered_map>

#include "device.cuh"
#include "internal.cuh"

namespace dm {

namespace {

constexpr int NT = 256;  // threads per block for every SpMV kernel

template <class V> struct Vec16;
template <> struct Vec16<double> { using T = double2; static constexpr int R = 2; };
template <> struct Vec16<float> { using T = float4; static constexpr int R = 4; };
template <int R> struct IVec;
template <> struct IVec<2> { using T = int2; };
template <> struct IVec<4> { using T = int4; };

template <class T, class V>
__device__ __forceinline__ void unpack(const T& v, V* out);
template <> __device__ __forceinline__ void unpack(const double2& v, double* o) { o[0] = v.x; o[1] = v.y; }
template <> __device__ __forceinline__ void unpack(const float4& v, float* o) { o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w; }
template <> __device__ __forceinline__ void unpack(const int2& v, int32_t* o) { o[0] = v.x; o[1] = v.y; }
template <> __device__ __forceinline__ void unpack(const int4& v, int32_t* o) { o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w; }

// acc + v * x in the vector type, as one fused multiply-add (FP64: one DFMA).
template <class V, class X>
__device__ __forceinline__ X fma_acc(V v, X x, X acc) { return fma(X(v), x, acc); }

// ---------------------------------------------------------------------------
// DIA: a thread owns NV x R consecutive rows (NV 16-byte value loads per
// diagonal). val[d*ld + i] is contiguous over i, so a warp reads 512 NV
// contiguous bytes per diagonal; x[i + off] is read through L1 (neighbouring
// diagonals hit the same lines). On B300 the FP64 form of this kernel is
// bound by the FP64 pipe (one DFMA per slot), so the loop issues exactly one
// fused multiply-add per stored slot and nothing else in FP64. Tiles whose
// rows see every diagonal inside the matrix run without bounds checks.
// ---------------------------------------------------------------------------
template <class V, class X, int NV, int ACC, bool DOT>
__global__ void __launch_bounds__(NT)
dia_kernel(int64_t N, int64_t M, int ndiag, const int32_t* __restrict__ offs, int32_t off_min,
           int32_t off_max, const V* __restrict__ dval, int64_t ld, const X* __restrict__ x,
           X* __restrict__ y, int64_t tile_rows, int64_t ntiles, int64_t tile0, DotSpec dot) {
  using VT = typename Vec16<V>::T;
  constexpr int R = Vec16<V>::R;
  constexpr int RT = NV * R;
  __shared__ double scratch[NT];
  if (skipped(dot)) return;
  double part = 0.0;  // this block's share of the dot, over all its tiles
  // tiles [tile0, ntiles): a base row and a local tile count keep the
  // register count of the whole-matrix form
  const int64_t nt = ntiles - tile0;
  const int64_t row0 = tile0 * tile_rows;
  for (int64_t tile = blockIdx.x; tile < nt; tile += gridDim.x) {
    const int64_t t0 = row0 + tile * tile_rows;
    const int64_t t1 = min(N, t0 + tile_rows);
    const bool interior = (t1 - t0 == tile_rows) && (t0 + off_min >= 0) && (t1 - 1 + off_max < M);
    for (int64_t i = t0 + (int64_t)threadIdx.x * RT; i < t1; i += (int64_t)NT * RT) {
      X acc[RT];
#pragma unroll
      for (int r = 0; r < RT; ++r) acc[r] = X(0);
      if (interior && ACC == 2) {
        // two independent multiply-add chains per row (even / odd diagonals)
        X acc2[RT];
#pragma unroll
        for (int r = 0; r < RT; ++r) acc2[r] = X(0);
        int d = 0;
#pragma unroll 2
        for (; d + 1 < ndiag; d += 2) {
          const int64_t off0 = __ldg(offs + d), off1 = __ldg(offs + d + 1);
          V v0[RT], v1[RT];
#pragma unroll
          for (int k = 0; k < NV; ++k) {
            unpack(ld_stream_l1na(reinterpret_cast<const VT*>(dval + (int64_t)d * ld + i) + k), v0 + k * R);
            unpack(ld_stream_l1na(reinterpret_cast<const VT*>(dval + (int64_t)(d + 1) * ld + i) + k),
                   v1 + k * R);
          }
          const X* xp0 = x + i + off0;
          const X* xp1 = x + i + off1;
#pragma unroll
          for (int r = 0; r < RT; ++r) {
            acc[r] = fma_acc(v0[r], ld_x(xp0 + r), acc[r]);
            acc2[r] = fma_acc(v1[r], ld_x(xp1 + r), acc2[r]);
          }
        }
        if (d < ndiag) {
          const int64_t off = __ldg(offs + d);
          V v[RT];
#pragma unroll
          for (int k = 0; k < NV; ++k)
            unpack(ld_stream_l1na(reinterpret_cast<const VT*>(dval + (int64_t)d * ld + i) + k), v + k * R);
#pragma unroll
          for (int r = 0; r < RT; ++r) acc[r] = fma_acc(v[r], ld_x(x + i + off + r), acc[r]);
        }
#pragma unroll
        for (int r = 0; r < RT; ++r) acc[r] += acc2[r];
      } else if (interior) {
#pragma unroll 4
        for (int d = 0; d < ndiag; ++d) {
          const int64_t off = __ldg(offs + d);
          V v[RT];
#pragma unroll
          for (int k = 0; k < NV; ++k)
            unpack(ld_stream_l1na(reinterpret_cast<const VT*>(dval + (int64_t)d * ld + i) + k), v + k * R);
          const X* xp = x + i + off;
#pragma unroll
          for (int r = 0; r < RT; ++r) acc[r] = fma_acc(v[r], ld_x(xp + r), acc[r]);
        }
      } else {
        for (int d = 0; d < ndiag; ++d) {
          const int64_t off = __ldg(offs + d);
          V v[RT];
#pragma unroll
          for (int k = 0; k < NV; ++k)
            unpack(ld_stream_l1na(reinterpret_cast<const VT*>(dval + (int64_t)d * ld + i) + k), v + k * R);
          const int64_t j = i + off;
#pragma unroll
          for (int r = 0; r < RT; ++r)
            if (j + r >= 0 && j + r < M && i + r < N) acc[r] = fma_acc(v[r], ld_x(x + j + r), acc[r]);
        }
      }
#pragma unroll
      for (int r = 0; r < RT; ++r)
        if (i + r < N) {
          y[i + r] = acc[r];
          if constexpr (DOT) part = fma((double)acc[r], (double)x[i + r], part);
        }
    }
  }
  if constexpr (DOT) {
    block_partial(dot, part, scratch);
    finish_dot(dot, gridDim.x, scratch);
  }
}

// ---------------------------------------------------------------------------
// DIA variant 6 (FP64 values and vectors): as variant 1 (a thread owns two
// consecutive rows, one 16-byte value load per diagonal, one DFMA per slot,
// diagonals summed in offset order, so the results are the same bits), but
// the diagonals go by runs of consecutive offsets whose starts and lengths
// are kernel parameters (no offset loads), and a run's x window is read as
// aligned 16-byte pairs held in registers: a run of 3 diagonals needs 2-3
// x loads instead of 6, about one load per DFMA instead of two, which keeps
// the load queue from throttling the FP64 pipe. Tiles whose window could
// reach x[M] (one past the end, read by an aligned pair) or leave the matrix
// take the bounds-checked loop.
// ---------------------------------------------------------------------------
// MINB: 0, or a minimum of resident blocks per SM for the compiler (6: at
// most 40 registers; see launch_typed for when that form runs).
template <bool DOT, int MINB = 0>
__global__ void __launch_bounds__(NT, MINB)
dia_runs_kernel(int64_t N, int64_t M, int ndiag, const int32_t* __restrict__ offs,
                int32_t off_min, int32_t off_max, const double* __restrict__ dval, int64_t ld,
                const double* __restrict__ x, double* __restrict__ y, int64_t tile_rows,
                int64_t ntiles, int64_t tile0, const __grid_constant__ DiaRuns runs, DotSpec dot) {
  __shared__ double scratch[NT];
  if (skipped(dot)) return;
  double part = 0.0;  // this block's share of the dot, over all its tiles
  // tiles [tile0, ntiles): a base row and a local tile count keep the
  // register count of the whole-matrix form
  const int64_t nt = ntiles - tile0;
  const int64_t row0 = tile0 * tile_rows;
  for (int64_t tile = blockIdx.x; tile < nt; tile += gridDim.x) {
    const int64_t t0 = row0 + tile * tile_rows;
    const int64_t t1 = min(N, t0 + tile_rows);
    const bool interior = (t1 - t0 == tile_rows) && (t0 + off_min >= 0) && (t1 + off_max < M);
    for (int64_t i = t0 + (int64_t)threadIdx.x * 2; i < t1; i += (int64_t)NT * 2) {
      double a0 = 0.0, a1 = 0.0;
      if (interior) {
        int d = 0;
        for (int r = 0; r < runs.n; ++r) {
          const int L = runs.len[r];
          const int64_t b = i + runs.start[r];  // row i reads x[b + j], row i + 1 x[b + j + 1]
          const double2* xp = reinterpret_cast<const double2*>(x + (b & ~(int64_t)1));
          const bool odd = b & 1;
          const int np = ((int)odd + L + 2) >> 1;  // pairs covering x[b .. b + L]
          double w[6];
          {
            const double2 q = __ldg(xp);
            w[0] = q.x;
            w[1] = q.y;
          }
          if (np > 1) {
            const double2 q = __ldg(xp + 1);
            w[2] = q.x;
            w[3] = q.y;
          }
          if (np > 2) {
            const double2 q = __ldg(xp + 2);
            w[4] = q.x;
            w[5] = q.y;
          }
          const double* vp = dval + (int64_t)d * ld + i;
          if (!odd) {
#pragma unroll
            for (int j = 0; j < DIA_RUN_LEN; ++j) {
              if (j >= L) break;
              const double2 v = ld_stream_l1na(reinterpret_cast<const double2*>(vp + (int64_t)j * ld));
              a0 = fma(v.x, w[j], a0);
              a1 = fma(v.y, w[j + 1], a1);
            }
          } else {
#pragma unroll
            for (int j = 0; j < DIA_RUN_LEN; ++j) {
              if (j >= L) break;
              const double2 v = ld_stream_l1na(reinterpret_cast<const double2*>(vp + (int64_t)j * ld));
              a0 = fma(v.x, w[j + 1], a0);
              a1 = fma(v.y, w[j + 2], a1);
            }
          }
          d += L;
        }
      } else {
        for (int d = 0; d < ndiag; ++d) {
          const int64_t j = i + __ldg(offs + d);
          const double2 v = ld_stream_l1na(reinterpret_cast<const double2*>(dval + (int64_t)d * ld + i));
          if (j >= 0 && j < M && i < N) a0 = fma(v.x, ld_x(x + j), a0);
          if (j + 1 >= 0 && j + 1 < M && i + 1 < N) a1 = fma(v.y, ld_x(x + j + 1), a1);
        }
      }
      if (i < N) {
        y[i] = a0;
        if constexpr (DOT) part = fma(a0, x[i], part);
      }
      if (i + 1 < N) {
        y[i + 1] = a1;
        if constexpr (DOT) part = fma(a1, x[i + 1], part);
      }
    }
  }
  if constexpr (DOT) {
    block_partial(dot, part, scratch);
    finish_dot(dot, gridDim.x, scratch);
  }
}

// ---------------------------------------------------------------------------
// ELL: slot-major, a thread owns R consecutive rows; col and val of a slot
// are 16-byte (or 8-byte) vector loads, padding (col < 0) is skipped.
// ---------------------------------------------------------------------------
// RANGE: tiles [tile0, ntiles) (a base row and a local tile count); else
// every tile from 0 (tile0 unused). The whole-matrix form keeps its own loop:
// with the range arithmetic it measured 3.5% slower at 128^3.
template <class V, class X, bool DOT, bool RANGE = false>
__global__ void __launch_bounds__(NT)
ell_kernel(int64_t N, int64_t K, const int32_t* __restrict__ ecol, const V* __restrict__ evl,
           int64_t ld, const X* __restrict__ x, X* __restrict__ y, int64_t tile_rows,
           int64_t ntiles, int64_t tile0, DotSpec dot) {
  using VT = typename Vec16<V>::T;
  constexpr int R = Vec16<V>::R;
  using IT = typename IVec<R>::T;
  __shared__ double scratch[NT];
  if (skipped(dot)) return;
  double part = 0.0;  // this block's share of the dot, over all its tiles
  const int64_t nt = RANGE ? ntiles - tile0 : ntiles;
  const int64_t row0 = RANGE ? tile0 * tile_rows : 0;
  for (int64_t tile = blockIdx.x; tile < nt; tile += gridDim.x) {
    const int64_t t0 = RANGE ? row0 + tile * tile_rows : tile * tile_rows;
    const int64_t t1 = RANGE ? min(N, t0 + tile_rows) : min(N, (tile + 1) * tile_rows);
    for (int64_t i = t0 + (int64_t)threadIdx.x * R; i < t1; i += (int64_t)NT * R) {
      X acc[R];
#pragma unroll
      for (int r = 0; r < R; ++r) acc[r] = X(0);
#pragma unroll 4
      for (int64_t k = 0; k < K; ++k) {
        V v[R];
        int32_t c[R];
        unpack(ld_stream(reinterpret_cast<const VT*>(evl + k * ld + i)), v);
        unpack(ld_stream(reinterpret_cast<const IT*>(ecol + k * ld + i)), c);
#pragma unroll
        for (int r = 0; r < R; ++r)
          if (c[r] >= 0) acc[r] = fma_acc(v[r], ld_x(x + c[r]), acc[r]);
      }
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (i + r < N) {
          y[i + r] = acc[r];
          if constexpr (DOT) part += (double)acc[r] * (double)x[i + r];
        }
    }
  }
  if constexpr (DOT) {
    block_partial(dot, part, scratch);
    finish_dot(dot, gridDim.x, scratch);
  }
}

// DIA variant 7, as ELL variant 2 for small matrices: a block takes 32
// consecutive rows at a time, lane l row l, and its 8 warps split the
// diagonals (warp w: diagonals w, w + 8, ...); a column outside the matrix is
// skipped. The warps' partial sums are added in warp order through shared
// memory (deterministic, not the diagonal order of variants 1-6). Rows
// [r0, r1).
template <class V, class X, bool DOT>
__global__ void __launch_bounds__(NT)
dia_split_kernel(int64_t M, int64_t ndiag, const int32_t* __restrict__ offs,
                 const V* __restrict__ dval, int64_t ld, const X* __restrict__ x,
                 X* __restrict__ y, int64_t r0, int64_t r1, DotSpec dot) {
  constexpr int W = NT / 32;
  __shared__ X ps[W][32];
  __shared__ double scratch[NT];
  if (skipped(dot)) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double part = 0.0;
  for (int64_t g = r0 + (int64_t)blockIdx.x * 32; g < r1; g += (int64_t)gridDim.x * 32) {
    const int64_t i = g + lane;
    X acc = X(0);
    if (i < r1) {
#pragma unroll 4
      for (int64_t d = w; d < ndiag; d += W) {
        const int64_t c = i + __ldg(offs + d);
        if (c >= 0 && c < M) acc = fma_acc(dval[d * ld + i], ld_x(x + c), acc);
      }
    }
    ps[w][lane] = acc;
    __syncthreads();
    if (w == 0 && i < r1) {
      X sum = ps[0][lane];
#pragma unroll
      for (int q = 1; q < W; ++q) sum += ps[q][lane];
      y[i] = sum;
      if constexpr (DOT) part += (double)sum * (double)x[i];
    }
    __syncthreads();
  }
  if constexpr (DOT) {
    block_partial(dot, part, scratch);
    finish_dot(dot, gridDim.x, scratch);
  }
}

// ELL variant 2, for matrices whose tiles would leave most SMs idle (at
// 16^3, four 1024-row tiles): a block takes 32 consecutive rows at a time,
// lane l row l, and its 8 warps split the slots (warp w: slots w, w + 8, ...),
// so a row's chain is a few slots long instead of K. The warps' partial sums
// are added in warp order through shared memory (deterministic, not the slot
// order of variant 1). Rows [r0, r1).
template <class V, class X, bool DOT>
__global__ void __launch_bounds__(NT)
ell_split_kernel(int64_t K, const int32_t* __restrict__ ecol, const V* __restrict__ evl,
                 int64_t ld, const X* __restrict__ x, X* __restrict__ y, int64_t r0, int64_t r1,
                 DotSpec dot) {
  constexpr int W = NT / 32;
  __shared__ X ps[W][32];
  __shared__ double scratch[NT];
  if (skipped(dot)) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double part = 0.0;
  for (int64_t g = r0 + (int64_t)blockIdx.x * 32; g < r1; g += (int64_t)gridDim.x * 32) {
    const int64_t i = g + lane;
    X acc = X(0);
    if (i < r1) {
#pragma unroll 4
      for (int64_t k = w; k < K; k += W) {
        const int32_t c = ecol[k * ld + i];
        if (c >= 0) acc = fma_acc(evl[k * ld + i], ld_x(x + c), acc);
      }
    }
    ps[w][lane] = acc;
    __syncthreads();
    if (w == 0 && i < r1) {
      X sum = ps[0][lane];
#pragma unroll
      for (int q = 1; q < W; ++q) sum += ps[q][lane];
      y[i] = sum;
      if constexpr (DOT) part += (double)sum * (double)x[i];
    }
    __syncthreads();
  }
  if constexpr (DOT) {
    block_partial(dot, part, scratch);
    finish_dot(dot, gridDim.x, scratch);
  }
}

// ---------------------------------------------------------------------------
// CSR vector kernel: a group of L lanes per row, lanes stride the row's
// entries, the group reduces with shuffles. L is the tuner's choice from the
// row-length distribution.
// ---------------------------------------------------------------------------
template <class V, class X, int L, bool DOT>
__global__ void __launch_bounds__(NT)
csr_vector_kernel(int64_t N, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                  const V* __restrict__ val, const X* __restrict__ x, X* __restrict__ y,
                  int64_t tile_rows, int64_t ntiles, int64_t tile0, DotSpec dot) {
  constexpr int G = NT / L;
  __shared__ double scratch[NT];
  if (skipped(dot)) return;
  const int g = threadIdx.x / L, k = threadIdx.x % L;
  double part = 0.0;  // this block's share of the dot, over all its tiles
  // tiles [tile0, ntiles), as a base row and a local tile count
  const int64_t nt = ntiles - tile0;
  const int64_t row0 = tile0 * tile_rows;
  for (int64_t tile = blockIdx.x; tile < nt; tile += gridDim.x) {
    const int64_t t0 = row0 + tile * tile_rows;
    const int64_t t1 = min(N, t0 + tile_rows);
    // Warp-uniform trip count: groups past the tile end run with an empty row.
    for (int64_t base = t0; base < t1; base += G) {
      const int64_t i = base + g;
      const bool active = i < t1;
      const int32_t a = active ? __ldg(rowptr + i) : 0, b = active ? __ldg(rowptr + i + 1) : 0;
      X acc0 = X(0), acc1 = X(0);
      int32_t e = a + k;
      for (; e + L < b; e += 2 * L) {
        const int32_t c0 = ld_stream(col + e), c1 = ld_stream(col + e + L);
        const V v0 = ld_stream(val + e), v1 = ld_stream(val + e + L);
        acc0 = fma_acc(v0, ld_x(x + c0), acc0);
        acc1 = fma_acc(v1, ld_x(x + c1), acc1);
      }
      if (e < b) acc0 = fma_acc(ld_stream(val + e), ld_x(x + ld_stream(col + e)), acc0);
      X acc = acc0 + acc1;
#pragma unroll
      for (int o = L / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, L);
      if (k == 0 && active) {
        y[i] = acc;
        if constexpr (DOT) part += (double)acc * (double)x[i];
      }
    }
  }
  if constexpr (DOT) {
    block_partial(dot, part, scratch);
    finish_dot(dot, gridDim.x, scratch);
  }
}

// ---------------------------------------------------------------------------
// Stream kernel (CSR variants 7 and 8, COO variant 2): a block takes ROWS
// consecutive rows (a "base"), whose entries form one contiguous range of
// the format's arrays (CSR: col, val; COO: row, col, val). A producer warp
// copies that range into shared memory with bulk copies (TMA) that signal an
// mbarrier. 2 ROWS consumer threads then work in lane pairs: lanes 2r and
// 2r+1 of a warp take the first and the second half of row r's entries, each
// in column order, with one fused multiply-add per entry, reading the
// entries from shared memory and x through the read-only path; a shuffle
// adds the halves. FP64 instructions do one entry with (nearly) all lanes
// busy for rows of similar length, 14-16 consumer warps hide the gather
// latency, and for banded or stencil matrices the lanes of a warp gather
// neighbouring x values.
// Where a row's entries start: CSR reads rowptr; COO finds it by binary
// search in the staged row indices (the lane pair searches for rows r and
// r + 1), and the range of each base comes from a plan array ustart (the
// first entry of every base, built once per format).
// Units (one pass of one base) go through two stages: the copies of the next
// unit are in flight while the consumers compute the current one, and the
// copies go through the TMA unit, not the load/store queue that the x
// gathers use. A range larger than the staging capacity `cap` (entries, a
// multiple of 4) is done in passes of `cap` entries; each lane adds the part
// of its half-row that lies in the pass.
// Every mbarrier wait is bounded (about 2 s): one that runs out sets
// g_wait_timeout and the block stops, after the producer has waited
// (bounded) for the copies it started.
// Shared memory, dynamic: two stages of col[cap + 4] (int32), for COO
// row[cap + 4] (int32), then val[cap + 4].
// ---------------------------------------------------------------------------
__device__ int g_wait_timeout;

constexpr long long CS_WAIT_CYCLES = 4000000000ll;

// Rows per base. COO: 128 (against 224 before: 128^3 stencil 194 -> 175 us,
// 1M-row uniform random 145 -> 135 us; 96 rows took 240 us). CSR: 256
// (variant 7) or 64 (variant 8). Small bases keep the staging ring small, so
// several blocks share an SM: faster where neighbouring rows gather nearby
// x (128^3 stencil 164 -> 146 us, 1M-row banded 92 -> 82 us), slower on
// random columns, whose gathers need the L1 that the rings then take
// (1M-row uniform 135 -> 162 us). The variant tuner picks per matrix.
template <bool COO, bool SMALL = false>
struct StreamShape {
  static constexpr int STAGES = 2;               // shared-memory stages in the ring
  static constexpr int ROWS = COO ? 128 : (SMALL ? 64 : 256);
  static constexpr int THREADS = 2 * ROWS + 32;  // lane pairs + one producer warp
  static constexpr int IDX = COO ? 8 : 4;        // index bytes per entry
};

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ bool mbar_test(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for the phase with the given parity to complete; false on timeout.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity,
                                          long long limit = CS_WAIT_CYCLES) {
  if (mbar_test(bar, parity)) return true;
  const long long t0 = clock64();
  do {
    if (mbar_test(bar, parity)) return true;
  } while (clock64() - t0 < limit);
  return mbar_test(bar, parity);
}

// Global -> shared bulk copy of `bytes` (a multiple of 16, both addresses
// 16-byte aligned) that signals `bar`.
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes,
                                          unsigned bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

size_t stream_smem_bytes(int64_t cap, size_t vsz, bool coo) {
  return (size_t)StreamShape<false>::STAGES * (size_t)(cap + 4) * ((coo ? 8 : 4) + vsz);
}

// K consecutive entries of a row, in order: all K gathers, then K
// multiply-adds into acc.
template <int K, class V, class X>
__device__ __forceinline__ X stream_group(const int32_t* c, const V* v, const X* __restrict__ x,
                                          X acc) {
  X xv[K];
#pragma unroll
  for (int j = 0; j < K; ++j) xv[j] = ld_x(x + c[j]);
#pragma unroll
  for (int j = 0; j < K; ++j) acc = fma_acc(v[j], xv[j], acc);
  return acc;
}

// One pass of one base: rows [base, bend), entries [p0, min(p0 + cap, e1)).
struct StreamUnit {
  int64_t tile, base, bend, p0, e1;
};

// rowptr: CSR row pointers, or for COO the plan array ustart (entry where
// each base starts; tile_rows == ROWS). row: COO row indices (CSR: unused).
// ACC: y[i] += the row's sum for rows with entries (others left as they are).
template <class V, class X, bool DOT, bool COO, bool ACC, bool SMALL>
__global__ void __launch_bounds__(StreamShape<COO, SMALL>::THREADS, 1)
stream_kernel(int64_t N, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ row,
              const int32_t* __restrict__ col, const V* __restrict__ val,
              const X* __restrict__ x, X* __restrict__ y, int64_t tile_rows, int64_t ntiles,
              int64_t tile0, int32_t cap, DotSpec dot) {
  using SS = StreamShape<COO, SMALL>;
  constexpr int ROWS = SS::ROWS;
  extern __shared__ __align__(16) unsigned char stream_smem[];
  __shared__ double scratch[SS::THREADS];
  constexpr int S = SS::STAGES;
  __shared__ __align__(8) uint64_t full[S], empty[S];
  __shared__ volatile int failed;
  if (skipped(dot)) return;
  constexpr int VG = 16 / sizeof(V);  // values per 16 bytes
  const size_t arr = (size_t)(cap + 4);
  const size_t buf_bytes = arr * (SS::IDX + sizeof(V));
  const int tid = threadIdx.x, lane = tid & 31;
  const bool producer = tid >= 2 * ROWS;
  auto scol = [&](int b) { return reinterpret_cast<int32_t*>(stream_smem + b * buf_bytes); };
  auto srow = [&](int b) { return reinterpret_cast<int32_t*>(stream_smem + b * buf_bytes + arr * 4); };
  auto sval = [&](int b) {
    return reinterpret_cast<V*>(stream_smem + b * buf_bytes + arr * SS::IDX);
  };
  auto start_base = [&](StreamUnit& u) {
    u.bend = min(min(N, (u.tile + 1) * tile_rows), u.base + ROWS);
    if constexpr (COO) {
      u.p0 = __ldg(rowptr + u.base / ROWS);
      u.e1 = __ldg(rowptr + u.base / ROWS + 1);
    } else {
      u.p0 = __ldg(rowptr + u.base);
      u.e1 = __ldg(rowptr + u.bend);
    }
  };
  // The unit after u: the next pass of the base, else the next base of the
  // tile, else the first base of the block's next tile (tile >= ntiles: none).
  auto advance = [&](StreamUnit u) {
    if (u.p0 + cap < u.e1) {
      u.p0 += cap;
      return u;
    }
    u.base += ROWS;
    if (u.base >= min(N, (u.tile + 1) * tile_rows)) {
      u.tile += gridDim.x;
      u.base = u.tile * tile_rows;
    }
    if (u.tile < ntiles) start_base(u);
    return u;
  };

  if (tid == 0) {
    for (int k = 0; k < S; ++k) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[k])), "r"(1)
                   : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty[k])),
                   "r"(2 * ROWS / 32)
                   : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    failed = 0;
  }
  __syncthreads();

  StreamUnit first;  // the block's tiles: tile0 + blockIdx.x, then every gridDim.x-th below ntiles
  first.tile = tile0 + blockIdx.x;
  first.base = first.tile * tile_rows;
  if (first.tile < ntiles) start_base(first);
  double part = 0.0;  // this block's share of the dot, over all its tiles

  if (producer) {
    // Lane 0 alone: stage k % S takes unit k; before refilling it, wait
    // until the consumers released its previous unit. The copy runs from p0
    // rounded down to 4 entries (16-byte aligned source) to at most 3
    // entries past the unit's end (inside the arrays' tail padding).
    if (lane == 0) {
      int64_t k = 0;
      for (StreamUnit u = first; u.tile < ntiles; u = advance(u), ++k) {
        const int st = (int)(k % S);
        if (k >= S && !mbar_wait(smem_u32(&empty[st]), (unsigned)(((k / S) - 1) & 1))) {
          atomicExch(&g_wait_timeout, 1);
          failed = 1;
          break;
        }
        if (failed) break;
        const int64_t p1 = min(u.e1, u.p0 + cap);
        const int64_t a0 = u.p0 & ~(int64_t)3;
        const unsigned bi = (unsigned)(((p1 - a0 + 3) >> 2) * 16);
        const unsigned bv = (unsigned)(((p1 - a0 + VG - 1) / VG) * 16);
        const unsigned bar = smem_u32(&full[st]);
        const unsigned total = p1 > u.p0 ? (COO ? 2 : 1) * bi + bv : 0u;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                     "r"(total)
                     : "memory");
        if (p1 > u.p0) {
          bulk_copy(scol(st), col + a0, bi, bar);
          if constexpr (COO) bulk_copy(srow(st), row + a0, bi, bar);
          bulk_copy(sval(st), val + a0, bv, bar);
        }
      }
      // Copies still in flight land before the block exits: wait (bounded)
      // for the last phase armed on each stage (already complete normally).
      for (int st = 0; st < S; ++st)
        if (k > st) mbar_wait(smem_u32(&full[st]), (unsigned)(((k - 1 - st) / S) & 1));
    }
    __syncwarp();
  } else {
    const unsigned FULL = 0xffffffffu;
    X acc = X(0);
    bool had = false;  // the row has entries (ACC)
    int64_t k = 0;
    for (StreamUnit cur = first; cur.tile < ntiles; ++k) {
      const int st = (int)(k % S);
      // The warp leaves together: the vote makes a timeout warp-uniform.
      if (!__all_sync(FULL, mbar_wait(smem_u32(&full[st]), (unsigned)((k / S) & 1)))) {
        if (lane == 0) {
          atomicExch(&g_wait_timeout, 1);
          failed = 1;
        }
        break;
      }
      const StreamUnit nxt = advance(cur);
      const int64_t i = cur.base + (tid >> 5) * 16 + (lane >> 1);
      const bool active = i < cur.bend;
      const int64_t a0 = cur.p0 & ~(int64_t)3;
      const int64_t p1 = min(cur.e1, cur.p0 + cap);
      const int32_t* c_s = scol(st);
      const V* v_s = sval(st);
      int32_t ra, rb;  // row i's staged entries
      if constexpr (COO) {
        // First staged entry of row i (even lane) or row i + 1 (odd lane).
        const int32_t* r_s = srow(st);
        const int32_t target = (int32_t)min(i, N) + (lane & 1);
        int32_t lo = (int32_t)(cur.p0 - a0), hi = (int32_t)(p1 - a0);
        while (lo < hi) {
          const int32_t mid = (lo + hi) >> 1;
          if (r_s[mid] < target) lo = mid + 1; else hi = mid;
        }
        const int32_t other = __shfl_xor_sync(FULL, lo, 1);
        ra = (lane & 1) ? other : lo;
        rb = (lane & 1) ? lo : other;
      } else {
        ra = active ? (int32_t)(max((int64_t)__ldg(rowptr + i), cur.p0) - a0) : 0;
        rb = active ? (int32_t)(min((int64_t)__ldg(rowptr + i + 1), p1) - a0) : 0;
      }
      if (active) {
        had = had || rb > ra;
        const int32_t mid = ra + ((rb - ra + 1) >> 1);
        int32_t e = (lane & 1) ? mid : ra;
        const int32_t e_end = (lane & 1) ? rb : mid;
        // Groups of gathers in flight, then their multiply-adds.
        for (; e + 16 <= e_end; e += 16) acc = stream_group<16>(c_s + e, v_s + e, x, acc);
        if (e + 8 <= e_end) {
          acc = stream_group<8>(c_s + e, v_s + e, x, acc);
          e += 8;
        }
        if (e + 4 <= e_end) {
          acc = stream_group<4>(c_s + e, v_s + e, x, acc);
          e += 4;
        }
        for (; e < e_end; ++e) acc = fma_acc(v_s[e], ld_x(x + c_s[e]), acc);
      }
      __syncwarp();
      if (lane == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty[st]))
                     : "memory");
      if (nxt.base != cur.base || nxt.tile >= ntiles) {  // the base's last pass
        acc += __shfl_xor_sync(FULL, acc, 1);  // first half + second half
        if (active && !(lane & 1)) {
          if constexpr (ACC) {
            if (had) y[i] += acc;
          } else {
            y[i] = acc;
            if constexpr (DOT) part += (double)acc * (double)x[i];
          }
        }
        acc = X(0);
        had = false;
      }
      cur = nxt;
      if (__any_sync(FULL, failed != 0)) break;
    }
  }
  if constexpr (DOT) {
    block_partial(dot, part, scratch);
    finish_dot(dot, gridDim.x, scratch);
  }
}

// Plan of the COO stream kernel: ustart[j] = first entry of row j * ROWS or
// later (lower bound in the sorted row indices), j = 0 .. nbases.
__global__ void coo_unit_start_kernel(const int32_t* __restrict__ row, int64_t nnz,
                                      int64_t nbases, int32_t rows, int32_t* __restrict__ ustart) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j > nbases) return;
  const int64_t target = j * rows;
  int64_t lo = 0, hi = nnz;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (row[mid] < target) lo = mid + 1; else hi = mid;
  }
  ustart[j] = (int32_t)lo;
}

// Longest row of a row-sorted COO. Each warp scans one contiguous span of
// 512-entry tiles, sixteen entries per lane from four 16-byte loads (row is
// 16-byte aligned; a load runs only when its first entry is below nnz, and
// the arrays' tail padding covers the rest of that group), with the next
// tile's loads in flight. A row that starts in a tile ends where the next
// row starts: the next start in the lane, else the first start of the lanes
// after it (from a ballot of the lanes holding a start), else the first
// start of a later tile of the span (the open row is carried from tile to
// tile). Only the row still open at the end of the span needs a search past
// it: one lane gallops (steps 1, 2, 4, ... then bisection). Rows that start
// before the span are measured by the span they start in. (One search per
// row start, the first form, left most lanes idle and ran at 0.09 of HBM.)
__global__ void coo_max_len_kernel(const int32_t* __restrict__ row, int64_t nnz,
                                   int32_t* __restrict__ out) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  constexpr int E = 16, TILE = 32 * E;  // entries per lane and per tile
  const int64_t ntiles = (nnz + TILE - 1) / TILE;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t per = (ntiles + nwarps - 1) / nwarps;
  const int64_t t_begin = w * per, t_end = min(ntiles, t_begin + per);
  const int4* r4 = reinterpret_cast<const int4*>(row);
  auto load = [&](int64_t tile, int h) {  // entries tile*TILE + E*lane + 4*h .. + 3
    const int64_t g = tile * (TILE / 4) + (E / 4) * lane + h;
    return 4 * g < nnz ? __ldcs(r4 + g) : make_int4(0, 0, 0, 0);
  };
  int64_t m = 0;
  int64_t open = -1;  // start of the row not yet closed (warp-uniform), -1: none
  int4 nq[E / 4];
#pragma unroll
  for (int h = 0; h < E / 4; ++h) nq[h] = t_begin < t_end ? load(t_begin, h) : make_int4(0, 0, 0, 0);
  for (int64_t tile = t_begin; tile < t_end; ++tile) {
    const int64_t e0 = tile * TILE + E * lane;
    int32_t v[E];
#pragma unroll
    for (int h = 0; h < E / 4; ++h) {
      v[4 * h] = nq[h].x;
      v[4 * h + 1] = nq[h].y;
      v[4 * h + 2] = nq[h].z;
      v[4 * h + 3] = nq[h].w;
    }
    if (tile + 1 < t_end) {  // the next tile in flight
#pragma unroll
      for (int h = 0; h < E / 4; ++h) nq[h] = load(tile + 1, h);
    }
    int32_t p = __shfl_up_sync(FULL, v[E - 1], 1);
    if (lane == 0 && e0 > 0) p = row[e0 - 1];
    unsigned sm = 0;  // which of the lane's entries start a row
    int prev = -1;
#pragma unroll
    for (int k = 0; k < E; ++k) {
      const int64_t e = e0 + k;
      if (e < nnz && (e == 0 || v[k] != p)) {
        sm |= 1u << k;
        if (prev >= 0) m = max(m, (int64_t)(k - prev));
        prev = k;
      }
      p = v[k];
    }
    // lanes holding a start; the next one after this lane closes its last row
    const unsigned B = __ballot_sync(FULL, sm != 0);
    const int fk = sm ? __ffs(sm) - 1 : 0, lk = sm ? 31 - __clz(sm) : 0;
    const unsigned above = lane == 31 ? 0u : (B & (FULL << (lane + 1)));
    const int nl = above ? __ffs(above) - 1 : lane;
    const int nfk = __shfl_sync(FULL, fk, nl);
    if (sm && above) m = max(m, (int64_t)(E * nl + nfk - E * lane - lk));
    if (B) {  // the tile's first start closes the open row; its last start opens one
      const int fl = __ffs(B) - 1, ll = 31 - __clz(B);
      const int ffk = __shfl_sync(FULL, fk, fl), llk = __shfl_sync(FULL, lk, ll);
      if (open >= 0) m = max(m, tile * TILE + E * fl + ffk - open);
      open = tile * TILE + E * ll + llk;
    }
  }
  if (lane == 0 && open >= 0) {
    // the row open at the span's end runs to the first entry with a larger row
    const int32_t r = row[open];
    int64_t lo = min(t_end * TILE, nnz) - 1, hi, step = 1;  // row[lo] == r
    for (;;) {
      hi = lo + step;
      if (hi >= nnz || row[hi] != r) break;
      lo = hi;
      step <<= 1;
    }
    hi = min(hi, nnz);
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) >> 1;
      if (row[mid] == r) lo = mid; else hi = mid;
    }
    m = max(m, hi - open);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(FULL, m, o));
  if (lane == 0 && m > 0) atomicMax(out, (int32_t)m);
}

// Self-tests of the bounded waits: a wait that nothing satisfies must give
// up after `limit` cycles and report it, and the kernel must return.
// 0: grid barrier of a cooperative launch whose block 1 leaves without
//    arriving (flag[0..1] its count); block 0 times out and sets flag[2].
// 1: an mbarrier that expects two arrivals and gets one; the wait times out.
__global__ void selftest_grid_barrier_kernel(unsigned* flag, long long limit) {
  if (blockIdx.x == 1) return;  // never arrives
  grid_barrier(reinterpret_cast<unsigned long long*>(flag), flag + 2, limit);
}
__global__ void selftest_mbarrier_kernel(unsigned* flag, long long limit) {
  __shared__ __align__(8) uint64_t mb;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mb)), "r"(2) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&mb)) : "memory");
    if (!mbar_wait(smem_u32(&mb), 0u, limit)) atomicExch(flag + 2, 1u);
  }
}

__global__ void max_len_kernel(const int32_t* __restrict__ rowptr, int64_t n,
                               int32_t* __restrict__ out) {
  int32_t m = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    m = max(m, rowptr[i + 1] - rowptr[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// Mean distance of entries from the diagonal, |col - row|, over `samples`
// evenly spaced rows: out[0] the sum of distances, out[1] the entries. It
// tells banded and stencil matrices (neighbouring rows read nearby x) from
// random columns, for the CSR stream kernel's base size.
__global__ void col_distance_kernel(const int32_t* __restrict__ rowptr,
                                    const int32_t* __restrict__ col, int64_t n, int64_t samples,
                                    unsigned long long* __restrict__ out) {
  unsigned long long sum = 0, cnt = 0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < samples;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t * n / samples;
    for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      const int64_t d = (int64_t)col[e] - i;
      sum += (unsigned long long)(d < 0 ? -d : d);
      ++cnt;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sum += __shfl_xor_sync(0xffffffffu, sum, o);
    cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  }
  if ((threadIdx.x & 31) == 0 && cnt) {
    atomicAdd(out, sum);
    atomicAdd(out + 1, cnt);
  }
}

// ---------------------------------------------------------------------------
// Segmented kernel for COO, nnz-balanced CSR ("merge") and the COO part of
// HYB. A warp owns a chunk of 128 consecutive entries, a lane 4 of them.
// Each lane sums its segments serially; a warp scan of (continues?, sum)
// pairs carries sums across lanes; rows that cross a chunk boundary leave
// per-chunk records that a second small kernel combines in entry order.
// Every row therefore has exactly one writer: deterministic, no atomics.
// ACCUM: add into y (HYB overflow) instead of writing, and leave rows
// without entries alone.
// ---------------------------------------------------------------------------
constexpr int SEG_VPT = 4;
constexpr int SEG_CHUNK = 32 * SEG_VPT;

template <class Acc>
struct SegCarry {
  int32_t* first_row;
  int32_t* last_row;
  int32_t* flags;  // bit 0: first row started before the chunk; bit 1: last row continues after
  Acc* head;       // chunk's share of its first row, when that row ends in the chunk
  Acc* tail;       // chunk's share of its last row, when that row continues after
};

template <class Acc>
SegCarry<Acc> seg_carry(const DBuf& b, int64_t nchunks) {
  SegCarry<Acc> c;
  char* p = (char*)b.p;
  c.first_row = (int32_t*)p;
  c.last_row = c.first_row + nchunks;
  c.flags = c.last_row + nchunks;
  size_t off = round_up((int64_t)nchunks * 12, 256);
  c.head = (Acc*)(p + off);
  c.tail = c.head + nchunks;
  return c;
}

size_t seg_carry_bytes(int64_t nchunks) { return round_up(nchunks * 12, 256) + nchunks * 16; }

__device__ __forceinline__ int64_t cdiv_dev(int64_t a, int64_t b) { return (a + b - 1) / b; }

template <bool CSR>
struct RowSrc {
  const int32_t* p;  // COO: row[nnz]; CSR: rowptr[N+1]
  int64_t nnz, nrows;
  const int32_t* chunk_row;
  // Row of entry e; CSR searches rows [lo, hi].
  __device__ __forceinline__ int32_t row_of(int64_t e, int32_t lo, int32_t hi) const {
    if constexpr (!CSR) {
      return __ldg(p + e);
    } else {
      // largest r in [lo, hi] with rowptr[r] <= e (the non-empty row holding e)
      while (lo < hi) {
        int32_t mid = (int32_t)(((int64_t)lo + hi + 1) >> 1);
        if (__ldg(p + mid) <= e) lo = mid; else hi = mid - 1;
      }
      return lo;
    }
  }
  // Does entry e (possibly == nnz) belong to row r?
  __device__ __forceinline__ bool in_row(int64_t e, int32_t r) const {
    if (e >= nnz) return false;
    if constexpr (!CSR) return __ldg(p + e) == r;
    else return e < __ldg(p + r + 1);
  }
};

template <class V, class X, bool CSR, bool ACCUM>
__global__ void __launch_bounds__(NT)
seg_kernel(RowSrc<CSR> src, const int32_t* __restrict__ col, const V* __restrict__ val,
           const X* __restrict__ x, X* __restrict__ y, SegCarry<X> carry, int64_t nchunks,
           const int32_t* skip) {
  using Acc = X;
  if (skip && *skip) return;
  const int lane = threadIdx.x & 31;
  const int64_t nnz = src.nnz;
  const unsigned FULL = 0xffffffffu;
  for (int64_t c = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 5; c < nchunks;
       c += ((int64_t)gridDim.x * NT) >> 5) {
    const int64_t s = c * SEG_CHUNK + (int64_t)lane * SEG_VPT;
    const bool valid = s < nnz;
    const int nh = valid ? (int)min((int64_t)SEG_VPT, nnz - s) : 0;
    int32_t lo = 0, hi = 0;
    if constexpr (CSR) {
      lo = __ldg(src.chunk_row + c);
      hi = __ldg(src.chunk_row + c + 1);
    }
    int32_t rr[SEG_VPT], cc[SEG_VPT];
    V vv[SEG_VPT];
    if (nh == SEG_VPT) {
      unpack(ld_stream(reinterpret_cast<const int4*>(col + s)), cc);
      if constexpr (sizeof(V) == 8) {
        unpack(ld_stream(reinterpret_cast<const double2*>(val + s)), (double*)vv);
        unpack(ld_stream(reinterpret_cast<const double2*>(val + s + 2)), (double*)vv + 2);
      } else {
        unpack(ld_stream(reinterpret_cast<const float4*>(val + s)), (float*)vv);
      }
      if constexpr (!CSR) unpack(ld_stream(reinterpret_cast<const int4*>(src.p + s)), rr);
    } else {
#pragma unroll
      for (int k = 0; k < SEG_VPT; ++k) {
        cc[k] = k < nh ? ld_stream(col + s + k) : 0;
        vv[k] = k < nh ? ld_stream(val + s + k) : V(0);
        if constexpr (!CSR) rr[k] = k < nh ? ld_stream(src.p + s + k) : 0;
      }
    }
    if constexpr (CSR) {
      if (valid) {
        int32_t r = src.row_of(s, lo, hi);
#pragma unroll
        for (int k = 0; k < SEG_VPT; ++k) {
          if (k < nh) {
            while (__ldg(src.p + r + 1) <= s + k) ++r;
          }
          rr[k] = r;
        }
      }
    }
    // Serial segmented sum over the lane's entries.
    Acc head = Acc(0), cur = Acc(0);
    int32_t head_row = -2, cur_row = -3;
    bool single = true;
    bool starts_before = false;
    if (valid) {
      cur_row = rr[0];
      // Entry s-1 lies in the previous chunk for lane 0: widen the search.
      int32_t plo = lo;
      if constexpr (CSR)
        if (lane == 0 && c > 0) plo = __ldg(src.chunk_row + c - 1);
      const int32_t prev = s == 0 ? -1 : src.row_of(s - 1, plo, hi);
      starts_before = prev == cur_row;
      if constexpr (!ACCUM)
        for (int32_t r = prev + 1; r < cur_row; ++r) y[r] = X(0);
#pragma unroll
      for (int k = 0; k < SEG_VPT; ++k) {
        if (k < nh) {
          const int32_t r = rr[k];
          const Acc xv = ld_x(x + cc[k]);
          if (r != cur_row) {
            if (single) {
              head = cur;
              head_row = cur_row;
              single = false;
            } else {
              if constexpr (ACCUM) y[cur_row] += cur; else y[cur_row] = cur;
            }
            if constexpr (!ACCUM)
              for (int32_t g = cur_row + 1; g < r; ++g) y[g] = X(0);
            cur_row = r;
            cur = Acc(0);
          }
          cur = fma(Acc(vv[k]), xv, cur);
        }
      }
      if (single) {
        head_row = cur_row;
        head = cur;
      }
    }
    const int32_t tail_row = cur_row;
    // Warp scan: S_l = T_l + a_l * S_{l-1}, a_l = (lane is one segment that
    // continues the previous lane's tail row).
    const int32_t prev_tail = __shfl_up_sync(FULL, tail_row, 1);
    const bool joins = valid && lane > 0 && head_row == prev_tail;
    Acc S = cur;
    int a = (single && joins) ? 1 : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const Acc Sp = __shfl_up_sync(FULL, S, o);
      const int ap = __shfl_up_sync(FULL, a, o);
      if (lane >= o) {
        if (a) S += Sp;
        a &= ap;
      }
    }
    const Acc S_prev = __shfl_up_sync(FULL, S, 1);
    const Acc carry_in = joins ? S_prev : Acc(0);
    // Chunk facts from lane 0.
    const int32_t first_row = __shfl_sync(FULL, head_row, 0);
    const bool chunk_starts_before = __shfl_sync(FULL, starts_before ? 1 : 0, 0) != 0;
    const int nvalid_lanes = (int)min((int64_t)32, cdiv_dev(nnz - c * SEG_CHUNK, SEG_VPT));
    if (valid) {
      auto emit = [&](int32_t r, Acc v) {
        if (r == first_row && chunk_starts_before) {
          carry.head[c] = v;
        } else {
          if constexpr (ACCUM) y[r] += v; else y[r] = v;
        }
      };
      if (!single) emit(head_row, head + carry_in);
      const int64_t e_next = s + nh;
      const bool cont = src.in_row(e_next, tail_row);
      const bool last_lane = lane == nvalid_lanes - 1;
      if (!cont) {
        emit(tail_row, S);
      } else if (last_lane) {
        carry.tail[c] = S;
      }
      if (last_lane) {
        carry.first_row[c] = first_row;
        carry.last_row[c] = tail_row;
        carry.flags[c] = (chunk_starts_before ? 1 : 0) | (cont ? 2 : 0);
        if constexpr (!ACCUM)
          if (e_next >= nnz)
            for (int64_t r = tail_row + 1; r < src.nrows; ++r) y[r] = X(0);
      }
    }
  }
}

// Combines the per-chunk records of rows that cross chunk boundaries, in
// entry order: the chunk where such a row ends writes it.
template <class X, bool ACCUM>
__global__ void seg_fixup_kernel(SegCarry<X> carry, int64_t nchunks, X* __restrict__ y,
                                 const int32_t* skip) {
  if (skip && *skip) return;
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nchunks) return;
  const int32_t fl = carry.flags[c];
  if (!(fl & 1)) return;
  const int32_t r = carry.first_row[c];
  if ((fl & 2) && carry.last_row[c] == r) return;  // passes through, ends later
  int64_t cl = c - 1;
  while (cl > 0 && (carry.flags[cl] & 3) == 3 && carry.first_row[cl] == r &&
         carry.last_row[cl] == r)
    --cl;
  X v = carry.tail[cl];
  for (int64_t k = cl + 1; k < c; ++k) v += carry.tail[k];
  v += carry.head[c];
  if constexpr (ACCUM) y[r] += v; else y[r] = v;
}

__global__ void chunk_row_kernel(const int32_t* __restrict__ rowptr, int64_t nrows, int64_t nnz,
                                 int64_t nchunks, int32_t* __restrict__ chunk_row) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c > nchunks) return;
  const int64_t e = min(c * SEG_CHUNK, nnz - 1);
  int64_t lo = 0, hi = nrows - 1;  // largest r with rowptr[r] <= e
  while (lo < hi) {
    int64_t mid = (lo + hi + 1) >> 1;
    if (rowptr[mid] <= e) lo = mid; else hi = mid - 1;
  }
  chunk_row[c] = (int32_t)lo;
}

// Dot product of two vectors with the same tile partition as the fused
// kernels (for formats whose SpMV cannot fuse it).
template <class X>
__global__ void __launch_bounds__(NT)
dot_tiles_kernel(int64_t N, const X* __restrict__ a, const X* __restrict__ b, int64_t tile_rows,
                 int64_t ntiles, DotSpec dot) {
  __shared__ double scratch[NT];
  if (skipped(dot)) return;
  double part = 0.0;  // this block's share of the dot, over all its tiles
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t t1 = min(N, (tile + 1) * tile_rows);
    for (int64_t i = tile * tile_rows + threadIdx.x; i < t1; i += NT)
      part += (double)a[i] * (double)b[i];
  }
  block_partial(dot, part, scratch);
  finish_dot(dot, gridDim.x, scratch);
}

template <class X>
__global__ void fill_kernel(X* __restrict__ y, int64_t n, X v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = v;
}

// ---------------------------------------------------------------------------
// Launch sizing
// ---------------------------------------------------------------------------
std::mutex g_occ_mu;
std::unordered_map<const void*, int> g_occ;

int resident_blocks(const void* fn) {
  std::lock_guard<std::mutex> lk(g_occ_mu);
  auto it = g_occ.find(fn);
  if (it != g_occ.end()) return it->second;
  int b = 0;
  DM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, NT, 0));
  b = std::max(1, b) * device().sms;
  g_occ[fn] = b;
  return b;
}

// Resident blocks of a kernel launched with `smem` bytes of dynamic shared
// memory, over all SMs.
std::map<std::pair<const void*, size_t>, int> g_occ_smem;
int resident_blocks_smem(const void* fn, size_t smem, int threads) {
  std::lock_guard<std::mutex> lk(g_occ_mu);
  auto key = std::make_pair(fn, smem);
  auto it = g_occ_smem.find(key);
  if (it != g_occ_smem.end()) return it->second;
  int b = 0;
  DM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, threads, smem));
  b = std::max(1, b) * device().sms;
  g_occ_smem[key] = b;
  return b;
}

// Grid for `work` units of a grid-stride kernel: at most the resident
// blocks, spread so every block gets the same number of units (+-1).
unsigned grid_for_units(const void* fn, int64_t work, size_t smem = 0, int threads = NT) {
  if (work <= 0) return 1;
  const int64_t res =
      smem || threads != NT ? resident_blocks_smem(fn, smem, threads) : resident_blocks(fn);
  const int64_t waves = cdiv(work, res);
  return (unsigned)std::max<int64_t>(1, cdiv(work, waves));
}

// Largest staging capacity of the stream kernel (entries): its two stages
// fit in one SM's shared memory.
constexpr size_t STREAM_SMEM_MAX = 200 * 1024;
int32_t stream_cap_max(size_t vsz, bool coo) {
  return (int32_t)(((STREAM_SMEM_MAX / StreamShape<false>::STAGES / ((coo ? 8 : 4) + vsz)) - 4) &
                   ~(size_t)63);
}

template <class V, class X, bool DOT, bool COO, bool ACC = false, bool SMALL = false>
void launch_stream_shape(const dynmat_s* A, const X* x, X* y, const DotSpec& d, cudaStream_t s,
                         int64_t tile0, int64_t tile1) {
  const Plan& P = A->plan;
  if (tile1 < 0) tile1 = P.ntiles;
  auto fn = stream_kernel<V, X, DOT, COO, ACC, SMALL>;
  constexpr int T = StreamShape<COO, SMALL>::THREADS;
  static std::once_flag once;
  std::call_once(once, [&] {
    DM_CUDA(cudaFuncSetAttribute(
        (const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
        (int)stream_smem_bytes(stream_cap_max(sizeof(V), COO), sizeof(V), COO)));
  });
  const size_t smem = stream_smem_bytes(P.stream_cap, sizeof(V), COO);
  const int32_t* starts = COO ? A->seg.unit_start.as<int32_t>() : A->csr.rowptr.as<int32_t>();
  const int32_t* row = COO ? A->coo.row.as<int32_t>() : nullptr;
  const int32_t* col = COO ? A->coo.col.as<int32_t>() : A->csr.col.as<int32_t>();
  const V* val = COO ? A->coo.val.as<V>() : A->csr.val.as<V>();
  fn<<<grid_for_units((const void*)fn, tile1 - tile0, smem, T), T, smem, s>>>(
      A->nrows, starts, row, col, val, x, y, P.tile_rows, tile1, tile0, P.stream_cap, d);
}

// The stream kernel of the plan: COO variant 2, CSR variant 7 (256-row
// bases) or 8 (64-row bases).
template <class V, class X, bool DOT, bool COO, bool ACC = false>
void launch_stream(const dynmat_s* A, const X* x, X* y, const DotSpec& d, cudaStream_t s,
                   int64_t tile0 = 0, int64_t tile1 = -1) {
  if (!COO && A->plan.variant == 8)
    launch_stream_shape<V, X, DOT, COO, ACC, true>(A, x, y, d, s, tile0, tile1);
  else
    launch_stream_shape<V, X, DOT, COO, ACC, false>(A, x, y, d, s, tile0, tile1);
}

template <class V, class X>
void launch_typed(const dynmat_s* A, const X* x, X* y, const DotSpec* dot, cudaStream_t s,
                  int64_t tile0 = 0, int64_t tile1 = -1) {
  const int64_t N = A->nrows, M = A->ncols;
  const Plan& P = A->plan;
  // DIA, ELL, the CSR vector and stream kernels and the COO stream kernel
  // can run a range of the plan's tiles [tile0, tile1); the other kernels
  // always run whole.
  const int64_t tr = P.tile_rows;
  if (tile1 < 0) tile1 = P.ntiles;
  const int64_t nt = tile1 - tile0;
  DotSpec d = dot ? *dot : DotSpec{};
  if (dot && !dot->partials) dot = nullptr;  // skip flag only: plain kernels
  switch (A->fmt) {
    case DYNMAT_DIA: {
      if (A->dia.ndiag == 0) {
        fill_kernel<X><<<grid_for_units((const void*)fill_kernel<X>, cdiv(N, NT)), NT, 0, s>>>(y, N, X(0));
        DM_CHECK_LAUNCH();
        if (dot) goto separate_dot;
        return;
      }
#define DM_DIA(NVV, AC, DT)                                                                 \
  {                                                                                         \
    auto fn = dia_kernel<V, X, NVV, AC, DT>;                                                \
    fn<<<grid_for_units((const void*)fn, nt), NT, 0, s>>>(                                  \
        N, M, (int)A->dia.ndiag, A->dia.offsets.as<int32_t>(), A->dia.off_min,              \
        A->dia.off_max, A->dia.val.as<V>(), A->dia.ld, x, y, tr, tile1, tile0, d);          \
  }
      // variants: 1 two rows per thread; 2 four rows; 3 two rows, half-size
      // tiles (more resident blocks); 4 as 3 with two chains per row;
      // 5 four rows with two chains per row (FP64 counts; FP32 doubles rows);
      // 6 (FP64 only, x 16-byte aligned) as 1 with the diagonals in runs;
      // 7 the diagonals split over a block's warps (small matrices)
      if (P.variant == 7) {  // rows of the tiles [tile0, tile1)
        const int64_t r0 = tile0 * tr, r1 = std::min(N, tile1 * tr);
        const int64_t groups = cdiv(r1 - r0, 32);
        if (dot) {
          auto fn = dia_split_kernel<V, X, true>;
          fn<<<grid_for_units((const void*)fn, groups), NT, 0, s>>>(
              M, A->dia.ndiag, A->dia.offsets.as<int32_t>(), A->dia.val.as<V>(), A->dia.ld, x, y,
              r0, r1, d);
        } else {
          auto fn = dia_split_kernel<V, X, false>;
          fn<<<grid_for_units((const void*)fn, groups), NT, 0, s>>>(
              M, A->dia.ndiag, A->dia.offsets.as<int32_t>(), A->dia.val.as<V>(), A->dia.ld, x, y,
              r0, r1, d);
        }
        DM_CHECK_LAUNCH();
        return;
      }
      if constexpr (std::is_same<V, double>::value && std::is_same<X, double>::value) {
        if (P.variant == 6 && P.runs.n > 0 && ((uintptr_t)x & 15u) == 0) {
          // fine_runs_grid: with one-pass tiles (large matrices), every
          // resident block, the tiles dealt out in turn, so blocks differ by
          // at most one small tile. The waves rule (equal tiles per block)
          // left some SMs a block more than others: 27-point 128^3 took
          // 116.7 us in 683 blocks of three 1024-row tiles, 112.6 us in the
          // 888 resident blocks (6 per SM) of four or five 512-row tiles
          // (120.8 us in 888 blocks of two or three 1024-row tiles; a tile
          // queue on an atomic counter 118.8 us).
          // A range of the tiles (a chunk of the host-buffer product, which
          // runs beside the next chunk on a second stream) keeps two tiles
          // per block, so that two chunks fit the resident blocks together.
          const bool fine = tr < (int64_t)NT * 4;
          const int64_t per_block = nt < P.ntiles ? 2 : 1;
          auto fine_runs_grid = [&](const void* f) {
            return fine ? (unsigned)std::min<int64_t>(cdiv(nt, per_block), resident_blocks(f))
                        : grid_for_units(f, nt);
          };
          if (dot) {
            // The fused dot takes 48 registers (5 blocks per SM); held to 40
            // (6 per SM) it spills a little. That form runs only where its
            // extra blocks save a wave of tiles: at 96^3, 864 tiles in one
            // wave instead of two (CG 101 -> 85 us per iteration). At 128^3
            // (4096 one-pass tiles) the two forms give the same CG iteration:
            // 150.8 and 151.1 us.
            auto fn = dia_runs_kernel<true>;
            auto fn6 = dia_runs_kernel<true, 6>;
            if (cdiv(nt, (int64_t)resident_blocks((const void*)fn6)) <
                cdiv(nt, (int64_t)resident_blocks((const void*)fn)))
              fn = fn6;
            fn<<<fine_runs_grid((const void*)fn), NT, 0, s>>>(
                N, M, (int)A->dia.ndiag, A->dia.offsets.as<int32_t>(), A->dia.off_min,
                A->dia.off_max, A->dia.val.as<double>(), A->dia.ld, x, y, tr, tile1, tile0,
                P.runs, d);
          } else {
            auto fn = dia_runs_kernel<false>;
            fn<<<fine_runs_grid((const void*)fn), NT, 0, s>>>(
                N, M, (int)A->dia.ndiag, A->dia.offsets.as<int32_t>(), A->dia.off_min,
                A->dia.off_max, A->dia.val.as<double>(), A->dia.ld, x, y, tr, tile1, tile0,
                P.runs, d);
          }
          DM_CHECK_LAUNCH();
          return;
        }
      }
      switch (P.variant) {
        case 2: if (dot) DM_DIA(2, 1, true) else DM_DIA(2, 1, false) break;
        case 4: if (dot) DM_DIA(1, 2, true) else DM_DIA(1, 2, false) break;
        case 5: if (dot) DM_DIA(2, 2, true) else DM_DIA(2, 2, false) break;
        default: if (dot) DM_DIA(1, 1, true) else DM_DIA(1, 1, false) break;
      }
#undef DM_DIA
      DM_CHECK_LAUNCH();
      return;
    }
    case DYNMAT_ELL:
    case DYNMAT_HYB: {
      const bool hyb = A->fmt == DYNMAT_HYB;
      const bool fuse = dot && !(hyb && A->coo.nnz > 0);
      if (P.variant == 2) {  // rows of the tiles [tile0, tile1)
        const int64_t r0 = tile0 * tr, r1 = std::min(N, tile1 * tr);
        const int64_t groups = cdiv(r1 - r0, 32);
        if (fuse) {
          auto fn = ell_split_kernel<V, X, true>;
          fn<<<grid_for_units((const void*)fn, groups), NT, 0, s>>>(
              A->ell.K, A->ell.col.as<int32_t>(), A->ell.val.as<V>(), A->ell.ld, x, y, r0, r1, d);
        } else {
          auto fn = ell_split_kernel<V, X, false>;
          fn<<<grid_for_units((const void*)fn, groups), NT, 0, s>>>(
              A->ell.K, A->ell.col.as<int32_t>(), A->ell.val.as<V>(), A->ell.ld, x, y, r0, r1, d);
        }
      } else if (fuse) {
        auto fn = ell_kernel<V, X, true>;
        fn<<<grid_for_units((const void*)fn, nt), NT, 0, s>>>(
            N, A->ell.K, A->ell.col.as<int32_t>(), A->ell.val.as<V>(), A->ell.ld, x, y, tr,
            tile1, tile0, d);
      } else if (tile0 != 0 || tile1 != P.ntiles) {
        auto fn = ell_kernel<V, X, false, true>;
        fn<<<grid_for_units((const void*)fn, nt), NT, 0, s>>>(
            N, A->ell.K, A->ell.col.as<int32_t>(), A->ell.val.as<V>(), A->ell.ld, x, y, tr,
            tile1, tile0, d);
      } else {
        auto fn = ell_kernel<V, X, false>;
        fn<<<grid_for_units((const void*)fn, nt), NT, 0, s>>>(
            N, A->ell.K, A->ell.col.as<int32_t>(), A->ell.val.as<V>(), A->ell.ld, x, y, tr,
            tile1, tile0, d);
      }
      DM_CHECK_LAUNCH();
      if (hyb && A->coo.nnz > 0) {
        RowSrc<false> src{A->coo.row.as<int32_t>(), A->coo.nnz, N, nullptr};
        auto carry = seg_carry<X>(A->seg.carry, A->seg.nchunks);
        auto fn = seg_kernel<V, X, false, true>;
        fn<<<grid_for_units((const void*)fn, cdiv(A->seg.nchunks, NT / 32)), NT, 0, s>>>(
            src, A->coo.col.as<int32_t>(), A->coo.val.as<V>(), x, y, carry, A->seg.nchunks, d.skip);
        DM_CHECK_LAUNCH();
        seg_fixup_kernel<X, true><<<(unsigned)cdiv(A->seg.nchunks, NT), NT, 0, s>>>(
            carry, A->seg.nchunks, y, d.skip);
        DM_CHECK_LAUNCH();
        if (dot) goto separate_dot;
      }
      return;
    }
    case DYNMAT_CSR: {
      if (P.variant == 7 || P.variant == 8) {
        if (dot) launch_stream<V, X, true, false>(A, x, y, d, s, tile0, tile1);
        else launch_stream<V, X, false, false>(A, x, y, d, s, tile0, tile1);
        DM_CHECK_LAUNCH();
        return;
      }
      if (P.variant >= 1 && P.variant <= 5) {
#define DM_CSRV(LN)                                                                         \
  {                                                                                         \
    if (dot) {                                                                              \
      auto fn = csr_vector_kernel<V, X, LN, true>;                                          \
      fn<<<grid_for_units((const void*)fn, nt), NT, 0, s>>>(                                \
          N, A->csr.rowptr.as<int32_t>(), A->csr.col.as<int32_t>(), A->csr.val.as<V>(), x, \
          y, tr, tile1, tile0, d);                                                          \
    } else {                                                                                \
      auto fn = csr_vector_kernel<V, X, LN, false>;                                         \
      fn<<<grid_for_units((const void*)fn, nt), NT, 0, s>>>(                                \
          N, A->csr.rowptr.as<int32_t>(), A->csr.col.as<int32_t>(), A->csr.val.as<V>(), x, \
          y, tr, tile1, tile0, d);                                                          \
    }                                                                                       \
  }
        switch (P.variant) {
          case 1: DM_CSRV(2); break;
          case 2: DM_CSRV(4); break;
          case 3: DM_CSRV(8); break;
          case 4: DM_CSRV(16); break;
          default: DM_CSRV(32); break;
        }
#undef DM_CSRV
        DM_CHECK_LAUNCH();
        return;
      }
      // merge (nnz-balanced)
      if (A->csr.nnz == 0) {
        fill_kernel<X><<<grid_for_units((const void*)fill_kernel<X>, cdiv(N, NT)), NT, 0, s>>>(y, N, X(0));
        DM_CHECK_LAUNCH();
      } else {
        RowSrc<true> src{A->csr.rowptr.as<int32_t>(), A->csr.nnz, N,
                         A->seg.chunk_row.as<int32_t>()};
        auto carry = seg_carry<X>(A->seg.carry, A->seg.nchunks);
        auto fn = seg_kernel<V, X, true, false>;
        fn<<<grid_for_units((const void*)fn, cdiv(A->seg.nchunks, NT / 32)), NT, 0, s>>>(
            src, A->csr.col.as<int32_t>(), A->csr.val.as<V>(), x, y, carry, A->seg.nchunks, d.skip);
        DM_CHECK_LAUNCH();
        seg_fixup_kernel<X, false><<<(unsigned)cdiv(A->seg.nchunks, NT), NT, 0, s>>>(
            carry, A->seg.nchunks, y, d.skip);
        DM_CHECK_LAUNCH();
      }
      if (dot) goto separate_dot;
      return;
    }
    case DYNMAT_COO: {
      if (P.variant == 2) {
        if (dot) launch_stream<V, X, true, true>(A, x, y, d, s, tile0, tile1);
        else launch_stream<V, X, false, true>(A, x, y, d, s, tile0, tile1);
        DM_CHECK_LAUNCH();
        return;
      }
      if (A->coo.nnz == 0) {
        fill_kernel<X><<<grid_for_units((const void*)fill_kernel<X>, cdiv(N, NT)), NT, 0, s>>>(y, N, X(0));
        DM_CHECK_LAUNCH();
      } else {
        RowSrc<false> src{A->coo.row.as<int32_t>(), A->coo.nnz, N, nullptr};
        auto carry = seg_carry<X>(A->seg.carry, A->seg.nchunks);
        auto fn = seg_kernel<V, X, false, false>;
        fn<<<grid_for_units((const void*)fn, cdiv(A->seg.nchunks, NT / 32)), NT, 0, s>>>(
            src, A->coo.col.as<int32_t>(), A->coo.val.as<V>(), x, y, carry, A->seg.nchunks, d.skip);
        DM_CHECK_LAUNCH();
        seg_fixup_kernel<X, false><<<(unsigned)cdiv(A->seg.nchunks, NT), NT, 0, s>>>(
            carry, A->seg.nchunks, y, d.skip);
        DM_CHECK_LAUNCH();
      }
      if (dot) goto separate_dot;
      return;
    }
  }
  return;
separate_dot: {
    auto fn = dot_tiles_kernel<X>;
    fn<<<grid_for_units((const void*)fn, P.ntiles), NT, 0, s>>>(N, x, y, P.tile_rows, P.ntiles, d);
    DM_CHECK_LAUNCH();
  }
}

}  // namespace

// CSR and COO kernel from the row-length distribution: rows of similar
// length, 4 or more on average -> stream kernel (entries staged in shared
// memory by TMA, a lane pair per row); skewed or very short rows ->
// nnz-balanced merge (CSR) or segmented (COO) kernel. The profiling tuner
// may override with any variant.
static int64_t tile_rows_for(const dynmat_s* A);

int auto_variant(const dynmat_s* A) {
  const int64_t N = std::max<int64_t>(A->nrows, 1);
  // The stream kernels walk every row in bases of a few hundred; below a
  // mean of 4 entries per row (e.g. the remote part of a partitioned
  // matrix) the nnz-balanced kernels do less work.
  auto stream_fits = [&](int64_t nnz, int64_t maxlen) {
    const double mean = (double)nnz / (double)N;
    return mean >= 4.0 && (double)maxlen <= 2.0 * mean + 32.0;
  };
  // DIA: the diagonals split over a block's warps (variant 7) when even
  // half-size tiles would number fewer than two per SM; half-size tiles
  // (variant 3) when the default tiles would; else, for FP64 values, the
  // diagonals in runs (variant 6; it needs an aligned x at launch and falls
  // back to 1 without one), else variant 1. 27-point stencil, FP64: 7 at 16^3
  // 8.2 against 16.4 us (3), at 48^3 16.4 against 18.4; at 64^3 3 is faster
  // (22.6 against 32.8 us).
  if (A->fmt == DYNMAT_DIA) {
    const int64_t r = A->vdt == DYNMAT_F64 ? 2 : 4;
    if (cdiv(A->nrows, NT * r) < 2 * device().sms) return 7;
    if (cdiv(A->nrows, 2 * NT * r) < 2 * device().sms) return 3;
    return A->vdt == DYNMAT_F64 && A->plan.runs.n > 0 ? 6 : 0;
  }
  // CSR: the stream kernel with 64-row bases (8) where neighbouring rows
  // read nearby x (mean |col - row| at most N/32 and 65,536: stencils and
  // banded matrices), else with 256-row bases (7); 6 when rows differ much.
  if (A->fmt == DYNMAT_CSR) {
    if (!stream_fits(A->csr.nnz, A->csr.maxlen)) return 6;
    const double local = std::min(65536.0, (double)N / 32.0);
    return A->csr.mean_dist <= local ? 8 : 7;
  }
  if (A->fmt == DYNMAT_COO)  // 1 segmented, 2 stream
    return stream_fits(A->coo.nnz, A->coo.maxlen) ? 2 : 1;
  // ELL and HYB: the slots split over a block's warps (2) when the row tiles
  // would number fewer than two per SM, as for DIA; else a thread per two rows
  // (1).
  if (A->fmt == DYNMAT_ELL || A->fmt == DYNMAT_HYB)
    return cdiv(A->nrows, tile_rows_for(A)) < 2 * device().sms ? 2 : 1;
  return 0;
}

// Row-tile size: 2 passes of the block over its rows, so a tile is 1024 rows
// (F64) or 2048 rows (F32) for DIA/ELL, and the partial-sum count stays small.
// DIA variants 3 and 4 use one pass per tile (twice the tiles, so more
// resident blocks on small problems). So does variant 6 where the default
// tiles would need more than one wave of its fused-dot kernel: it then runs
// on a grid of the resident blocks (see fine_runs_grid).
static int64_t tile_rows_for(const dynmat_s* A) {
  const int R = A->vdt == DYNMAT_F64 ? 2 : 4;
  if (A->fmt == DYNMAT_DIA && (A->plan.variant == 3 || A->plan.variant == 4))
    return (int64_t)NT * R;
  if (A->fmt == DYNMAT_DIA && A->plan.variant == 6 && A->vdt == DYNMAT_F64 &&
      cdiv(A->nrows, (int64_t)NT * R * 2) > resident_blocks((const void*)dia_runs_kernel<true, 6>))
    return (int64_t)NT * R;
  return (int64_t)NT * R * 2;
}

void prepare_spmv(dynmat_s* A, cudaStream_t s) {
  Plan& P = A->plan;
  ++A->gen;
  P.tile_rows = tile_rows_for(A);
  P.ntiles = std::max<int64_t>(1, cdiv(A->nrows, P.tile_rows));
  if (A->fmt == DYNMAT_CSR) {
    // longest row (int32 at 0) and the sampled distance sums (at 8 and 16)
    DBuf m(24, s);
    DM_CUDA(cudaMemsetAsync(m.p, 0, 24, s));
    if (A->nrows > 0) {
      max_len_kernel<<<(unsigned)std::min<int64_t>(cdiv(A->nrows, NT), 4096), NT, 0, s>>>(
          A->csr.rowptr.as<int32_t>(), A->nrows, m.as<int32_t>());
      DM_CHECK_LAUNCH();
      const int64_t samples = std::min<int64_t>(A->nrows, 4096);
      col_distance_kernel<<<(unsigned)cdiv(samples, NT), NT, 0, s>>>(
          A->csr.rowptr.as<int32_t>(), A->csr.col.as<int32_t>(), A->nrows, samples,
          reinterpret_cast<unsigned long long*>(m.as<char>() + 8));
      DM_CHECK_LAUNCH();
    }
    unsigned long long h[3] = {0, 0, 0};
    DM_CUDA(cudaMemcpyAsync(h, m.p, 24, cudaMemcpyDeviceToHost, s));
    DM_CUDA(cudaStreamSynchronize(s));
    A->csr.maxlen = (int32_t)(h[0] & 0xffffffffu);
    A->csr.mean_dist = h[2] ? (double)h[1] / (double)h[2] : 0.0;
  }
  if (A->fmt == DYNMAT_COO) {
    DBuf m(4, s);
    DM_CUDA(cudaMemsetAsync(m.p, 0, 4, s));
    if (A->coo.nnz > 0) {
      DM_REQUIRE(((uintptr_t)A->coo.row.p & 15u) == 0, DYNMAT_ERR_INVALID_ARG,
                 "internal: COO row array not 16-byte aligned");
      coo_max_len_kernel<<<(unsigned)std::min<int64_t>(cdiv(cdiv(A->coo.nnz, 512), NT / 32),
                                                       (int64_t)device().sms * 8),
                           NT, 0, s>>>(A->coo.row.as<int32_t>(), A->coo.nnz, m.as<int32_t>());
      DM_CHECK_LAUNCH();
    }
    int32_t h = 0;
    DM_CUDA(cudaMemcpyAsync(&h, m.p, 4, cudaMemcpyDeviceToHost, s));
    DM_CUDA(cudaStreamSynchronize(s));
    A->coo.maxlen = h;
  }
  P.runs.n = 0;
  A->dia.main_diag = -1;
  if (A->fmt == DYNMAT_DIA && A->dia.ndiag > 0) {
    std::vector<int32_t> off((size_t)A->dia.ndiag);
    DM_CUDA(cudaMemcpyAsync(off.data(), A->dia.offsets.p, off.size() * 4, cudaMemcpyDeviceToHost, s));
    DM_CUDA(cudaStreamSynchronize(s));
    A->dia.off_min = off.front();
    A->dia.off_max = off.back();
    const auto z = std::lower_bound(off.begin(), off.end(), 0);
    if (z != off.end() && *z == 0) A->dia.main_diag = z - off.begin();
    // Runs of consecutive offsets for variant 6 (none if there are too many).
    if (A->dia.ndiag <= (int64_t)DIA_RUNS * DIA_RUN_LEN) {
      DiaRuns R;
      R.n = 0;
      bool fits = true;
      for (size_t k = 0; k < off.size() && fits;) {
        size_t e = k + 1;
        while (e < off.size() && e - k < (size_t)DIA_RUN_LEN && off[e] == off[e - 1] + 1) ++e;
        if (R.n == DIA_RUNS) {
          fits = false;
          break;
        }
        R.start[R.n] = off[k];
        R.len[R.n] = (int32_t)(e - k);
        ++R.n;
        k = e;
      }
      if (fits) P.runs = R;
    }
  }
  P.variant = P.forced ? P.forced : auto_variant(A);
  P.stream_cap = 0;
  const bool coo_stream = A->fmt == DYNMAT_COO && P.variant == 2;
  const int rows = coo_stream          ? StreamShape<true>::ROWS
                   : P.variant == 8 ? StreamShape<false, true>::ROWS
                                    : StreamShape<false>::ROWS;
  if ((A->fmt == DYNMAT_CSR && (P.variant == 7 || P.variant == 8)) || coo_stream) {
    // Room for a base's rows at the longest row, or at the mean row length
    // plus 1/8 if that is less, in multiples of 64 entries; longer ranges
    // take more than one pass.
    const int64_t nnz = coo_stream ? A->coo.nnz : A->csr.nnz;
    const int64_t maxlen = coo_stream ? A->coo.maxlen : A->csr.maxlen;
    const double mean = (double)nnz / (double)std::max<int64_t>(A->nrows, 1);
    const int64_t want = round_up(
        std::min<int64_t>(maxlen * rows, (int64_t)std::ceil(mean * rows * 1.125) + 8), 64);
    P.stream_cap = (int32_t)std::min<int64_t>(std::max<int64_t>(want, 256),
                                              stream_cap_max(vsize(A->vdt), coo_stream));
  }
  P.tile_rows = tile_rows_for(A);  // depends on the variant
  if (P.stream_cap) P.tile_rows = rows;  // stream kernel: a tile is one base
  P.ntiles = std::max<int64_t>(1, cdiv(A->nrows, P.tile_rows));
  A->seg.nchunks = 0;
  A->seg.chunk_row.release();
  A->seg.carry.release();
  A->seg.unit_start.release();
  if (coo_stream) {
    const int64_t nb = cdiv(A->nrows, rows);
    A->seg.unit_start.alloc((nb + 1) * 4, s);
    coo_unit_start_kernel<<<(unsigned)cdiv(nb + 1, NT), NT, 0, s>>>(
        A->coo.row.as<int32_t>(), A->coo.nnz, nb, rows, A->seg.unit_start.as<int32_t>());
    DM_CHECK_LAUNCH();
  }
  int64_t seg_nnz = -1;
  if (A->fmt == DYNMAT_COO && !coo_stream) seg_nnz = A->coo.nnz;
  if (A->fmt == DYNMAT_HYB) seg_nnz = A->coo.nnz;
  if (A->fmt == DYNMAT_CSR && P.variant == 6) seg_nnz = A->csr.nnz;
  if (seg_nnz > 0) {
    const int64_t nch = cdiv(seg_nnz, SEG_CHUNK);
    A->seg.nchunks = nch;
    A->seg.carry.alloc(seg_carry_bytes(nch), s);
    if (A->fmt == DYNMAT_CSR) {
      A->seg.chunk_row.alloc((nch + 1) * 4, s);
      chunk_row_kernel<<<(unsigned)cdiv(nch + 1, NT), NT, 0, s>>>(
          A->csr.rowptr.as<int32_t>(), A->nrows, A->csr.nnz, nch, A->seg.chunk_row.as<int32_t>());
      DM_CHECK_LAUNCH();
    }
  }
}

// Blocking: raises DYNMAT_ERR_TIMEOUT (and clears the flag) when a bounded
// device-side wait ran out since the last check. Called by the blocking
// entry points, whose results would then be invalid.
void check_wait_timeout(cudaStream_t s) {
  int h = 0;
  DM_CUDA(cudaMemcpyFromSymbolAsync(&h, g_wait_timeout, sizeof h, 0, cudaMemcpyDeviceToHost, s));
  DM_CUDA(cudaStreamSynchronize(s));
  if (h) {
    const int z = 0;
    DM_CUDA(cudaMemcpyToSymbolAsync(g_wait_timeout, &z, sizeof z, 0, cudaMemcpyHostToDevice, s));
    DM_CUDA(cudaStreamSynchronize(s));
  }
  DM_REQUIRE(h == 0, DYNMAT_ERR_TIMEOUT,
             "a bounded wait in the CSR stream kernel's copy pipeline ran out; results since the "
             "last check are invalid");
}

}  // namespace dm

extern "C" dynmat_status dynmat_selftest_wait_timeout(int32_t which, int64_t cycles,
                                                     int32_t* timed_out, dynmat_stream_t stream) {
  using namespace dm;
  return guard([&] {
    DM_REQUIRE(timed_out && (which == 0 || which == 1) && cycles > 0 && cycles <= (1ll << 33),
               DYNMAT_ERR_INVALID_ARG, "bad self-test arguments");
    cudaStream_t s = (cudaStream_t)stream;
    DBuf flag(16, s);
    DM_CUDA(cudaMemsetAsync(flag.p, 0, 16, s));
    unsigned* f = flag.as<unsigned>();
    if (which == 0) {
      cudaLaunchConfig_t cfg{};
      cfg.gridDim = dim3(2);
      cfg.blockDim = dim3(32);
      cfg.stream = s;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeCooperative;
      attr[0].val.cooperative = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      DM_CUDA(cudaLaunchKernelEx(&cfg, selftest_grid_barrier_kernel, f, (long long)cycles));
    } else {
      selftest_mbarrier_kernel<<<1, 32, 0, s>>>(f, (long long)cycles);
      DM_CHECK_LAUNCH();
    }
    unsigned h[3] = {0, 0, 0};
    DM_CUDA(cudaMemcpyAsync(h, flag.p, sizeof h, cudaMemcpyDeviceToHost, s));
    DM_CUDA(cudaStreamSynchronize(s));
    *timed_out = h[2] ? 1 : 0;
  });
}

namespace dm {
// y rows of tiles [tile0, tile1) only (DIA and ELL): the pieces of a
// pipelined product. Rows outside the range are left as they are.
bool has_row_ranges(const dynmat_s* A) {
  const int v = A->plan.variant;
  return A->fmt == DYNMAT_DIA || A->fmt == DYNMAT_ELL ||
         (A->fmt == DYNMAT_HYB && A->coo.nnz == 0) ||  // no overflow: the ELL part alone
         (A->fmt == DYNMAT_CSR && ((v >= 1 && v <= 5) || v == 7 || v == 8)) ||
         (A->fmt == DYNMAT_COO && v == 2);
}

void spmv_rows(const dynmat_s* A, const void* x, void* y, dynmat_dtype vdt_vec, int64_t r0,
               int64_t r1, cudaStream_t s) {
  DM_REQUIRE(has_row_ranges(A), DYNMAT_ERR_INVALID_ARG,
             "row ranges are for DIA, ELL, HYB without overflow, CSR variants 1-5, 7 and 8 and "
             "COO variant 2");
  r1 = std::min<int64_t>(r1, A->nrows);
  if (r1 <= r0) return;
  // the plan's tiles, so every row is summed exactly as spmv sums it
  const int64_t tr = A->plan.tile_rows;
  DM_REQUIRE(r0 % tr == 0, DYNMAT_ERR_INVALID_ARG, "row range start %lld is not a multiple of %lld",
             (long long)r0, (long long)tr);
  const int64_t t0 = r0 / tr, t1 = cdiv(r1, tr);
  if (A->vdt == DYNMAT_F64) {
    DM_REQUIRE(vdt_vec == DYNMAT_F64, DYNMAT_ERR_INVALID_ARG, "F64 matrix values need F64 vectors");
    launch_typed<double, double>(A, (const double*)x, (double*)y, nullptr, s, t0, t1);
  } else if (vdt_vec == DYNMAT_F32) {
    launch_typed<float, float>(A, (const float*)x, (float*)y, nullptr, s, t0, t1);
  } else {
    launch_typed<float, double>(A, (const double*)x, (double*)y, nullptr, s, t0, t1);
  }
}

// Public-facing dispatch (vec_dt: type of x and y).
void spmv(const dynmat_s* A, const void* x, void* y, dynmat_dtype vdt_vec, cudaStream_t s) {
  spmv_dot(A, x, y, vdt_vec, nullptr, s);
}

void spmv_dot(const dynmat_s* A, const void* x, void* y, dynmat_dtype vdt_vec,
              const DotSpec* dot, cudaStream_t s) {
  spmv_skip(A, x, y, vdt_vec, dot, nullptr, s);
}

// As spmv_dot; without a dot, `skip` (device flag, may be NULL) makes every
// kernel of the product return at once while *skip != 0.
void spmv_skip(const dynmat_s* A, const void* x, void* y, dynmat_dtype vdt_vec,
               const DotSpec* dot, const int32_t* skip, cudaStream_t s) {
  if (A->nrows == 0) return;
  DotSpec only_skip{};
  only_skip.skip = skip;
  const DotSpec* ds = dot;
  if (!dot && skip) ds = &only_skip;
  // A DotSpec without partials runs the plain kernels with the skip flag.
  if (A->vdt == DYNMAT_F64) {
    DM_REQUIRE(vdt_vec == DYNMAT_F64, DYNMAT_ERR_INVALID_ARG,
               "F64 matrix values need F64 vectors");
    launch_typed<double, double>(A, (const double*)x, (double*)y, ds, s);
  } else if (vdt_vec == DYNMAT_F32) {
    launch_typed<float, float>(A, (const float*)x, (float*)y, ds, s);
  } else {
    launch_typed<float, double>(A, (const double*)x, (double*)y, ds, s);
  }
}

namespace {
// y += A x for the kernels with an accumulating form (COO and CSR stream
// kernels, the segmented COO and CSR-merge kernels): every row with entries
// gets its sum added once, rows without entries are left as they are.
template <class V, class X>
bool accumulate_typed(const dynmat_s* A, const X* x, X* y, cudaStream_t s) {
  if (A->fmt == DYNMAT_COO && A->plan.variant == 2) {
    launch_stream<V, X, false, true, true>(A, x, y, DotSpec{}, s);
    DM_CHECK_LAUNCH();
    return true;
  }
  if (A->fmt == DYNMAT_CSR && (A->plan.variant == 7 || A->plan.variant == 8)) {
    launch_stream<V, X, false, false, true>(A, x, y, DotSpec{}, s);
    DM_CHECK_LAUNCH();
    return true;
  }
  const bool coo = A->fmt == DYNMAT_COO;
  const bool merge = A->fmt == DYNMAT_CSR && A->plan.variant == 6;
  if (!coo && !merge) return false;
  const int64_t nnz = coo ? A->coo.nnz : A->csr.nnz;
  if (nnz == 0) return true;
  auto carry = seg_carry<X>(A->seg.carry, A->seg.nchunks);
  if (coo) {
    RowSrc<false> src{A->coo.row.as<int32_t>(), A->coo.nnz, A->nrows, nullptr};
    auto fn = seg_kernel<V, X, false, true>;
    fn<<<grid_for_units((const void*)fn, cdiv(A->seg.nchunks, NT / 32)), NT, 0, s>>>(
        src, A->coo.col.as<int32_t>(), A->coo.val.as<V>(), x, y, carry, A->seg.nchunks, nullptr);
  } else {
    RowSrc<true> src{A->csr.rowptr.as<int32_t>(), A->csr.nnz, A->nrows,
                     A->seg.chunk_row.as<int32_t>()};
    auto fn = seg_kernel<V, X, true, true>;
    fn<<<grid_for_units((const void*)fn, cdiv(A->seg.nchunks, NT / 32)), NT, 0, s>>>(
        src, A->csr.col.as<int32_t>(), A->csr.val.as<V>(), x, y, carry, A->seg.nchunks, nullptr);
  }
  DM_CHECK_LAUNCH();
  seg_fixup_kernel<X, true><<<(unsigned)cdiv(A->seg.nchunks, NT), NT, 0, s>>>(
      carry, A->seg.nchunks, y, nullptr);
  DM_CHECK_LAUNCH();
  return true;
}
}  // namespace

bool spmv_accumulate(const dynmat_s* A, const void* x, void* y, dynmat_dtype vdt_vec,
                     cudaStream_t s) {
  if (A->nrows == 0) return true;
  if (A->vdt == DYNMAT_F64) {
    DM_REQUIRE(vdt_vec == DYNMAT_F64, DYNMAT_ERR_INVALID_ARG,
               "F64 matrix values need F64 vectors");
    return accumulate_typed<double, double>(A, (const double*)x, (double*)y, s);
  }
  if (vdt_vec == DYNMAT_F32) return accumulate_typed<float, float>(A, (const float*)x, (float*)y, s);
  return accumulate_typed<float, double>(A, (const double*)x, (double*)y, s);
}

void dot_tiles(const dynmat_s* A, const void* a, const void* b, dynmat_dtype vdt_vec,
               const DotSpec& dot, cudaStream_t s) {
  const Plan& P = A->plan;
  if (vdt_vec == DYNMAT_F64) {
    auto fn = dot_tiles_kernel<double>;
    fn<<<grid_for_units((const void*)fn, P.ntiles), NT, 0, s>>>(
        A->nrows, (const double*)a, (const double*)b, P.tile_rows, P.ntiles, dot);
  } else {
    auto fn = dot_tiles_kernel<float>;
    fn<<<grid_for_units((const void*)fn, P.ntiles), NT, 0, s>>>(
        A->nrows, (const float*)a, (const float*)b, P.tile_rows, P.ntiles, dot);
  }
  DM_CHECK_LAUNCH();
}

}  // namespace dm

// ---------------------------------------------------------------------------
// COO SpMV that allocates nothing (dynmat_spmv_coo_noalloc).
//
// Some callers cannot allocate device memory at the time they multiply:
// allocators that are disabled or budget-locked while a solver is active,
// and latency-bound loops or hosts that forbid cudaMalloc on the hot path
// (it can synchronise the device or fail under memory pressure). For them
// the carry records of the segmented COO kernel live in one fixed array
// compiled into this library instead of in buffers owned by a handle.
// Every GPU that loads the library holds the array until the process exits.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_noalloc_scratch[4u << 20];

namespace dm {
namespace {

constexpr int64_t NOALLOC_SCRATCH_BYTES = 4 << 20;

std::mutex g_noalloc_mu;
void* g_noalloc_addr[64] = {};

// Device address of g_noalloc_scratch on the current device, looked up once
// per device (the name is only a host-side stand-in for it) and kept for
// the life of the process: a reset of the device's primary context
// (cudaDeviceReset) makes it stale, as the header states.
void* noalloc_scratch() {
  int dev = 0;
  DM_CUDA(cudaGetDevice(&dev));
  DM_REQUIRE(dev >= 0 && dev < 64, DYNMAT_ERR_INVALID_ARG, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    DM_REQUIRE(e == cudaSuccess && p, DYNMAT_ERR_CUDA,
               "cudaGetSymbolAddress of the fixed scratch array failed: %s",
               cudaGetErrorString(e));
    g_noalloc_addr[dev] = p;
  }
  return g_noalloc_addr[dev];
}

SegCarry<double> seg_carry_at(void* base, int64_t nchunks) {
  SegCarry<double> c;
  char* p = (char*)base;
  c.first_row = (int32_t*)p;
  c.last_row = c.first_row + nchunks;
  c.flags = c.last_row + nchunks;
  c.head = (double*)(p + round_up(nchunks * 12, 256));
  c.tail = c.head + nchunks;
  return c;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace
}  // namespace dm

extern "C" dynmat_status dynmat_spmv_coo_noalloc(int64_t nrows, int64_t nnz, const int32_t* row,
                                                 const int32_t* col, const double* val,
                                                 const double* x, double* y,
                                                 dynmat_stream_t stream) {
  using namespace dm;
  return guard([&] {
    DM_REQUIRE(nrows >= 0 && nnz >= 0, DYNMAT_ERR_INVALID_ARG, "negative size");
    DM_REQUIRE(nnz <= DYNMAT_NOALLOC_MAX_NNZ, DYNMAT_ERR_INVALID_ARG,
               "nnz %lld is over the %lld entries this call's fixed scratch array serves; "
               "use dynmat_spmv on a handle instead",
               (long long)nnz, (long long)DYNMAT_NOALLOC_MAX_NNZ);
    DM_REQUIRE(nrows == 0 || y, DYNMAT_ERR_INVALID_ARG, "null y");
    DM_REQUIRE(nnz == 0 || (row && col && val && x), DYNMAT_ERR_INVALID_ARG, "null input");
    DM_REQUIRE(aligned16(row) && aligned16(col) && aligned16(val), DYNMAT_ERR_INVALID_ARG,
               "row, col and val must start on 16-byte boundaries");
    cudaStream_t s = (cudaStream_t)stream;
    if (nrows == 0) return;
    if (nnz == 0) {
      fill_kernel<double><<<(unsigned)std::min<int64_t>(cdiv(nrows, NT), 4096), NT, 0, s>>>(
          y, nrows, 0.0);
      DM_CHECK_LAUNCH();
      return;
    }
    const int64_t nch = cdiv(nnz, SEG_CHUNK);
    // Every record the fix-up pass reads is written by the first pass of the
    // same call, so the array needs no clearing between calls.
    DM_REQUIRE((int64_t)seg_carry_bytes(nch) <= NOALLOC_SCRATCH_BYTES, DYNMAT_ERR_INVALID_ARG,
               "scratch too small for %lld chunks", (long long)nch);
    SegCarry<double> carry = seg_carry_at(noalloc_scratch(), nch);
    RowSrc<false> src{row, nnz, nrows, nullptr};
    auto fn = seg_kernel<double, double, false, false>;
    fn<<<grid_for_units((const void*)fn, cdiv(nch, NT / 32)), NT, 0, s>>>(src, col, val, x, y,
                                                                          carry, nch, nullptr);
    DM_CHECK_LAUNCH();
    seg_fixup_kernel<double, false><<<(unsigned)cdiv(nch, NT), NT, 0, s>>>(carry, nch, y, nullptr);
    DM_CHECK_LAUNCH();
  });
}
