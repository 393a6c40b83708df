// Format conversions (§III-B "Convert"): every conversion goes from the active
// format to COO and from COO to the target, as the paper's proxy policy
// states. Values are moved as raw 32/64-bit words, so every conversion is
// bit-exact; the only value test is DIA's "is this slot zero" (both signed
// zeros count as padding).
#include <algorithm>

#include "internal.cuh"

namespace dm {

extern double g_pad_limit;
int64_t hyb_width(const int32_t* rowptr, int64_t N, int64_t maxlen, int64_t vb, cudaStream_t s);

namespace {

constexpr int T = 256;

inline unsigned grid_for(int64_t n, int per_thread = 1) {
  int64_t b = cdiv(std::max<int64_t>(n, 1), (int64_t)T * per_thread);
  return (unsigned)std::min<int64_t>(b, 1 << 30);
}

// Grid of a group-per-row kernel (G lanes per row, a grid-stride loop over
// rows): enough blocks for every row or a few waves' worth, whichever is
// smaller.
inline unsigned group_grid(int64_t rows, int G) {
  const int64_t b = cdiv(std::max<int64_t>(rows, 1) * G, (int64_t)T);
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)device().sms * 16));
}

template <class W>
__device__ __forceinline__ bool word_is_zero(W w) {
  return (W)(w << 1) == 0;  // +0.0 or -0.0
}

// --- CSR ------------------------------------------------------------------

// rowptr[i] = first entry whose row >= i (lower bound in the sorted rows).
// (A search from the guess i * nnz / nrows, widened by doubling steps,
// measured 1.6x slower than this plain bisection at 128^3: the bisection's
// first steps hit the same entries in every thread and stay in cache.)
__global__ void rowptr_kernel(const int32_t* __restrict__ row, int64_t nnz, int64_t nrows,
                              int32_t* __restrict__ rowptr) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i > nrows) return;
  int64_t lo = 0, hi = nnz;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (row[mid] < i) lo = mid + 1; else hi = mid;
  }
  rowptr[i] = (int32_t)lo;
}

// row[e] = r for every e in [rowptr[r], rowptr[r+1]). A warp takes 32
// consecutive rows at a time: one coalesced load brings their row pointers,
// then the warp writes each row's range contiguously (coalesced stores);
// neighbouring warps take neighbouring rows. (A binary search per entry, the
// first form, ran at 0.1 of HBM; a group per row that loaded its own two
// row pointers was latency-bound at 0.18.)
__global__ void expand_rows_kernel(const int32_t* __restrict__ rowptr, int64_t nrows,
                                   int32_t* __restrict__ row) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; r0 < nrows;
       r0 += nwarps * 32) {
    const int64_t r = r0 + lane;
    const int32_t a = r < nrows ? rowptr[r] : 0;
    int32_t b = __shfl_down_sync(FULL, a, 1);
    if (lane == 31 || r + 1 >= nrows) b = r < nrows ? rowptr[r + 1] : 0;
    const int nr = (int)min((int64_t)32, nrows - r0);
    for (int j = 0; j < nr; ++j) {
      const int32_t aj = __shfl_sync(FULL, a, j), bj = __shfl_sync(FULL, b, j);
      for (int32_t e = aj + lane; e < bj; e += 32) row[e] = (int32_t)(r0 + j);
    }
  }
}

__global__ void row_lengths_kernel(const int32_t* __restrict__ rowptr, int64_t nrows,
                                   int32_t* __restrict__ len) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nrows) len[i] = rowptr[i + 1] - rowptr[i];
}

// --- DIA ------------------------------------------------------------------

__device__ __forceinline__ void mark_once(int32_t* flag, int64_t k) {
  if (flag[k] == 0) flag[k] = 1;
}

// flag[col - row + nrows - 1] = 1 for every entry. Many entries share an
// offset (27 distinct ones for the 27-point stencil), so a flag is read
// first and stored only while it is still 0: the hot flags stay in L1
// instead of every entry storing to the same few L2 lines (the stores
// contended, at 0.09 of HBM). VEC: four entries per thread from 16-byte
// loads of row and col (both 16-byte aligned; the arrays' tail padding
// covers the last group).
template <bool VEC>
__global__ void mark_offsets_kernel(const int32_t* __restrict__ row,
                                    const int32_t* __restrict__ col, int64_t nnz, int64_t nrows,
                                    int32_t* flag) {
  const int64_t base = nrows - 1;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (VEC) {
    const int64_t ng = (nnz + 3) / 4;
    auto mark4 = [&](int64_t g, const int4& r, const int4& c) {
      const int64_t e = 4 * g;
      mark_once(flag, (int64_t)c.x - r.x + base);
      if (e + 1 < nnz) mark_once(flag, (int64_t)c.y - r.y + base);
      if (e + 2 < nnz) mark_once(flag, (int64_t)c.z - r.z + base);
      if (e + 3 < nnz) mark_once(flag, (int64_t)c.w - r.w + base);
    };
    int64_t g = t;
    for (; g + stride < ng; g += 2 * stride) {  // two groups' loads in flight
      const int4 r0 = __ldcs(reinterpret_cast<const int4*>(row) + g);
      const int4 c0 = __ldcs(reinterpret_cast<const int4*>(col) + g);
      const int4 r1 = __ldcs(reinterpret_cast<const int4*>(row) + g + stride);
      const int4 c1 = __ldcs(reinterpret_cast<const int4*>(col) + g + stride);
      mark4(g, r0, c0);
      mark4(g + stride, r1, c1);
    }
    if (g < ng)
      mark4(g, __ldcs(reinterpret_cast<const int4*>(row) + g),
            __ldcs(reinterpret_cast<const int4*>(col) + g));
  } else {
    for (int64_t e = t; e < nnz; e += stride) mark_once(flag, (int64_t)col[e] - row[e] + base);
  }
}

__global__ void dia_offsets_kernel(const int32_t* __restrict__ flag,
                                   const int32_t* __restrict__ idx, int64_t span, int64_t nrows,
                                   int32_t* __restrict__ offsets) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < span && flag[k]) offsets[idx[k]] = (int32_t)(k - (nrows - 1));
}

// Thread per row i: the row's entries go to dval[d * ld + i]. Consecutive
// threads write consecutive slots of each diagonal (coalesced stores), and
// the strided reads of the rows' col and val come back from L1. (One thread
// per entry wrote 27 diagonals' lines per warp store, at 0.30 of HBM.)
template <class W>
__global__ void dia_scatter_kernel(const int32_t* __restrict__ rowptr,
                                   const int32_t* __restrict__ col, const W* __restrict__ val,
                                   int64_t nrows, int64_t ld, const int32_t* __restrict__ idx,
                                   W* __restrict__ dval) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrows) return;
  const int64_t e1 = rowptr[i + 1];
  for (int64_t e = rowptr[i]; e < e1; ++e) {
    const int64_t d = idx[(int64_t)col[e] - i + (nrows - 1)];
    dval[d * ld + i] = val[e];
  }
}

template <class W>
__global__ void dia_count_kernel(const int32_t* __restrict__ offsets, int64_t ndiag,
                                 const W* __restrict__ dval, int64_t nrows, int64_t ncols,
                                 int64_t ld, int32_t* __restrict__ cnt) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrows) return;
  int32_t c = 0;
  for (int64_t d = 0; d < ndiag; ++d) {
    int64_t j = i + offsets[d];
    if (j >= 0 && j < ncols && !word_is_zero(dval[d * ld + i])) ++c;
  }
  cnt[i] = c;
}

// Place of a kept slot among its group's kept slots, and the group's count:
// one ballot over the warp, masked to the G lanes of the group.
template <int G>
__device__ __forceinline__ void group_rank(bool keep, int& rank, int& total) {
  const unsigned lane = threadIdx.x & 31;
  const unsigned gmask = (G == 32 ? 0xffffffffu : ((1u << G) - 1u) << (lane & ~(unsigned)(G - 1)));
  const unsigned b = __ballot_sync(0xffffffffu, keep) & gmask;
  rank = __popc(b & ((1u << lane) - 1u));
  total = __popc(b);
}

// DIA to COO: a group of G lanes per row, lane j taking diagonals j, j + G,
// ...; the kept slots (in range, value not +-0) of the row are written as
// one contiguous run at start[i], in diagonal (= column) order. One thread
// per row, the first form, stored 27 scattered words per warp instruction
// and ran at 0.1 of HBM. All lanes of a warp make the same number of passes
// (the ballots), and neighbouring warps take neighbouring rows, so the
// sectors of the slot-major arrays serve several rows from L1. (Giving each
// warp its own run of 64 rows measured 1.5-2.4x slower: tens of thousands
// of short DRAM streams.)
template <class W, int G>
__global__ void dia_emit_kernel(const int32_t* __restrict__ offsets, int64_t ndiag,
                                const W* __restrict__ dval, int64_t nrows, int64_t ncols,
                                int64_t ld, const int32_t* __restrict__ start,
                                int32_t* __restrict__ orow, int32_t* __restrict__ ocol,
                                W* __restrict__ oval) {
  const int64_t groups = ((int64_t)gridDim.x * blockDim.x) / G;
  const int j = threadIdx.x % G;
  const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int64_t span = (nrows + (32 / G) - 1) / (32 / G) * (32 / G);  // whole warps
  for (int64_t i = g0; i < span; i += groups) {
    const bool row_ok = i < nrows;
    int64_t m = row_ok ? start[i] : 0;
    for (int64_t d0 = 0; d0 < ndiag; d0 += G) {
      const int64_t d = d0 + j;
      bool keep = false;
      int64_t c = 0;
      W w = 0;
      if (row_ok && d < ndiag) {
        c = i + offsets[d];
        if (c >= 0 && c < ncols) {
          w = dval[d * ld + i];
          keep = !word_is_zero(w);
        }
      }
      int rank, total;
      group_rank<G>(keep, rank, total);
      if (keep) {
        orow[m + rank] = (int32_t)i;
        ocol[m + rank] = (int32_t)c;
        oval[m + rank] = w;
      }
      m += total;
    }
  }
}

// DIA, ELL or HYB to COO through shared memory, for sources of up to a few
// dozen slots per row. A block takes ET consecutive rows: it copies their
// slot-major arrays into shared memory with coalesced loads (for each slot,
// the ET rows are contiguous; padded to ET + 1 words per slot, so that the
// transposed reads below hit distinct banks), then a warp per row ranks the
// kept slots by ballot and writes them as one contiguous run at start[i], in
// slot order (for DIA: in range and not +-0; for ELL: not padding), with a
// HYB row's overflow entries after them. The same output as dia_emit_kernel
// and ell_emit_kernel, whose reads of the slot arrays each touched 27-32
// lines per warp instruction (0.26-0.39 of HBM at 128^3).
constexpr int ET = 64;

template <class W, bool DIA>
size_t emit_tiled_smem(int64_t K) {
  return (size_t)K * (ET + 1) * (sizeof(W) + (DIA ? 0 : 4)) + (DIA ? (size_t)K * 4 : 0);
}

template <class W, bool DIA>
__global__ void __launch_bounds__(T)
emit_tiled_kernel(const int32_t* __restrict__ ecol, const int32_t* __restrict__ offsets,
                  const W* __restrict__ sval, int64_t nrows, int64_t ncols, int64_t ld, int64_t K,
                  const int32_t* __restrict__ crow, const int32_t* __restrict__ ccol,
                  const W* __restrict__ cval, int64_t ncoo, const int32_t* __restrict__ start,
                  int32_t* __restrict__ orow, int32_t* __restrict__ ocol, W* __restrict__ oval) {
  extern __shared__ __align__(16) unsigned char es_smem[];
  W* sv = reinterpret_cast<W*>(es_smem);                          // [K][ET + 1]
  int32_t* sc = reinterpret_cast<int32_t*>(sv + K * (ET + 1));  // ELL: [K][ET + 1]; DIA: offsets[K]
  const int64_t i0 = (int64_t)blockIdx.x * ET;
  const int rows = (int)(nrows - i0 < ET ? nrows - i0 : ET);
  // every slot's value is loaded (padding holds 0), not only after its
  // column: one round of loads instead of two; four slots per thread in flight
#pragma unroll 4
  for (int64_t idx = threadIdx.x; idx < K * ET; idx += T) {
    const int64_t k = idx / ET;
    const int r = (int)(idx % ET);
    W w = 0;
    if (r < rows) {
      w = sval[k * ld + i0 + r];
      if (!DIA) sc[k * (ET + 1) + r] = ecol[k * ld + i0 + r];
    }
    sv[k * (ET + 1) + r] = w;
  }
  if (DIA)
    for (int64_t k = threadIdx.x; k < K; k += T) sc[k] = offsets[k];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  for (int r = threadIdx.x >> 5; r < rows; r += T / 32) {
    const int64_t i = i0 + r;
    int64_t m = start[i];
    for (int64_t k0 = 0; k0 < K; k0 += 32) {
      const int64_t k = k0 + lane;
      bool keep = false;
      int64_t c = -1;
      W w = 0;
      if (k < K) {
        w = sv[k * (ET + 1) + r];
        if (DIA) {
          c = i + sc[k];
          keep = c >= 0 && c < ncols && !word_is_zero(w);
        } else {
          c = sc[k * (ET + 1) + r];
          keep = c >= 0;
        }
      }
      const unsigned b = __ballot_sync(0xffffffffu, keep);
      if (keep) {
        const int64_t o = m + __popc(b & ((1u << lane) - 1u));
        orow[o] = (int32_t)i;
        ocol[o] = (int32_t)c;
        oval[o] = w;
      }
      m += __popc(b);
    }
    if (!DIA && crow) {  // the row's overflow entries (HYB), after its ELL slots
      int64_t lo = 0, hi = ncoo;
      while (lo < hi) { int64_t mm = (lo + hi) >> 1; if (crow[mm] < i) lo = mm + 1; else hi = mm; }
      for (int64_t e = lo + lane; e < ncoo && crow[e] == i; e += 32) {
        orow[m + (e - lo)] = (int32_t)i;
        ocol[m + (e - lo)] = ccol[e];
        oval[m + (e - lo)] = cval[e];
      }
    }
  }
}

// --- ELL / HYB ------------------------------------------------------------

// Thread per row (rows up to ld so the padding rows are defined too): slots
// [0, min(len, K)) from the row's entries, the rest padding; with `ccol`
// set (HYB), entries beyond K go to the COO part at cstart[i].
template <class W>
__global__ void ell_fill_kernel(const int32_t* __restrict__ rowptr,
                                const int32_t* __restrict__ col, const W* __restrict__ val,
                                int64_t nrows, int64_t ld, int64_t K, int32_t* __restrict__ ecol,
                                W* __restrict__ evl, const int32_t* __restrict__ cstart,
                                int32_t* __restrict__ crow, int32_t* __restrict__ ccol,
                                W* __restrict__ cval) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ld) return;
  int64_t a = 0, len = 0;
  if (i < nrows) {
    a = rowptr[i];
    len = rowptr[i + 1] - a;
  }
  for (int64_t k = 0; k < K; ++k) {
    if (k < len) {
      ecol[k * ld + i] = col[a + k];
      evl[k * ld + i] = val[a + k];
    } else {
      ecol[k * ld + i] = -1;
      evl[k * ld + i] = 0;
    }
  }
  if (ccol && len > K) {
    int64_t m = cstart[i];
    for (int64_t k = K; k < len; ++k, ++m) {
      crow[m] = (int32_t)i;
      ccol[m] = col[a + k];
      cval[m] = val[a + k];
    }
  }
}

__global__ void ell_count_kernel(const int32_t* __restrict__ ecol, int64_t nrows, int64_t ld,
                                 int64_t K, const int32_t* __restrict__ crow, int64_t ncoo,
                                 int32_t* __restrict__ cnt) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrows) return;
  int32_t c = 0;
  for (int64_t k = 0; k < K; ++k) c += ecol[k * ld + i] >= 0;
  if (crow) {
    int64_t lo = 0, hi = ncoo;
    while (lo < hi) { int64_t m = (lo + hi) >> 1; if (crow[m] < i) lo = m + 1; else hi = m; }
    int64_t a = lo;
    lo = a; hi = ncoo;
    while (lo < hi) { int64_t m = (lo + hi) >> 1; if (crow[m] <= i) lo = m + 1; else hi = m; }
    c += (int32_t)(lo - a);
  }
  cnt[i] = c;
}

// ELL (and HYB) to COO, as dia_emit_kernel: a group of G lanes per row over
// the slots, the kept (non-padding) slots written contiguously at start[i];
// for HYB the row's overflow entries follow, found by one binary search in
// the COO part's rows and copied by the group.
template <class W, int G>
__global__ void ell_emit_kernel(const int32_t* __restrict__ ecol, const W* __restrict__ evl,
                                int64_t nrows, int64_t ld, int64_t K,
                                const int32_t* __restrict__ crow,
                                const int32_t* __restrict__ ccol, const W* __restrict__ cval,
                                int64_t ncoo, const int32_t* __restrict__ start,
                                int32_t* __restrict__ orow, int32_t* __restrict__ ocol,
                                W* __restrict__ oval) {
  const int64_t groups = ((int64_t)gridDim.x * blockDim.x) / G;
  const int j = threadIdx.x % G;
  const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int64_t span = (nrows + (32 / G) - 1) / (32 / G) * (32 / G);  // whole warps
  for (int64_t i = g0; i < span; i += groups) {
    const bool row_ok = i < nrows;
    int64_t m = row_ok ? start[i] : 0;
    for (int64_t k0 = 0; k0 < K; k0 += G) {
      const int64_t k = k0 + j;
      int32_t c = -1;
      W w = 0;
      if (row_ok && k < K) {
        c = ecol[k * ld + i];
        if (c >= 0) w = evl[k * ld + i];
      }
      int rank, total;
      group_rank<G>(c >= 0, rank, total);
      if (c >= 0) {
        orow[m + rank] = (int32_t)i;
        ocol[m + rank] = c;
        oval[m + rank] = w;
      }
      m += total;
    }
    if (crow && row_ok) {
      int64_t lo = 0, hi = ncoo;
      while (lo < hi) { int64_t mm = (lo + hi) >> 1; if (crow[mm] < i) lo = mm + 1; else hi = mm; }
      for (int64_t e = lo + j; e < ncoo && crow[e] == i; e += G) {
        orow[m + (e - lo)] = (int32_t)i;
        ocol[m + (e - lo)] = ccol[e];
        oval[m + (e - lo)] = cval[e];
      }
    }
  }
}

// Row-length histogram. Lanes of a warp with the same length add once
// (warp-aggregated), so a few common lengths do not serialise on atomics.
__global__ void len_hist_kernel(const int32_t* __restrict__ rowptr, int64_t nrows,
                                int32_t* __restrict__ hist) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool in = i < nrows;
  const unsigned active = __ballot_sync(0xffffffffu, in);
  if (!in) return;
  const int32_t len = rowptr[i + 1] - rowptr[i];
  const unsigned same = __match_any_sync(active, len);
  if ((threadIdx.x & 31) == __ffs(same) - 1) atomicAdd(&hist[len], __popc(same));
}

// K_h = argmin_k slot*k*N + over*(S1(k) - k*S0(k)), S0/S1 = suffix sums of
// counts / length*counts over lengths > k; ties to the smaller k. One block;
// the suffix sums run in chunks of blockDim from the top length down.
__global__ void hyb_width_kernel(const int32_t* __restrict__ hist, int64_t maxlen, int64_t nrows,
                                 int64_t slot, int64_t over, int64_t* __restrict__ out) {
  __shared__ long long s0[1024], s1[1024];
  __shared__ long long carry0, carry1;
  __shared__ long long best_cost[1024];
  __shared__ long long best_k[1024];
  const int t = threadIdx.x, nt = blockDim.x;
  if (t == 0) { carry0 = 0; carry1 = 0; }
  long long my_cost = -1, my_k = 0;
  __syncthreads();
  // lengths processed from maxlen downwards in chunks of nt
  for (int64_t top = maxlen; top >= 0; top -= nt) {
    int64_t l = top - t;  // this thread's length
    long long c0 = 0, c1 = 0;
    if (l >= 0) { c0 = hist[l]; c1 = (long long)l * hist[l]; }
    s0[t] = c0; s1[t] = c1;
    __syncthreads();
    // inclusive scan over t (t = 0 is the largest length)
    for (int o = 1; o < nt; o <<= 1) {
      long long a0 = t >= o ? s0[t - o] : 0, a1 = t >= o ? s1[t - o] : 0;
      __syncthreads();
      s0[t] += a0; s1[t] += a1;
      __syncthreads();
    }
    if (l >= 0) {
      // sums over lengths > l = carry + inclusive(t) - own
      long long S0 = carry0 + s0[t] - c0, S1 = carry1 + s1[t] - c1;
      long long cost = slot * l * nrows + over * (S1 - l * S0);
      if (my_cost < 0 || cost < my_cost || (cost == my_cost && l < my_k)) { my_cost = cost; my_k = l; }
    }
    __syncthreads();
    if (t == nt - 1) { carry0 += s0[t]; carry1 += s1[t]; }
    __syncthreads();
  }
  best_cost[t] = my_cost;
  best_k[t] = my_k;
  __syncthreads();
  if (t == 0) {
    long long bc = -1, bk = 0;
    for (int i = 0; i < nt; ++i) {
      long long c = best_cost[i];
      if (c < 0) continue;
      if (bc < 0 || c < bc || (c == bc && best_k[i] < bk)) { bc = c; bk = best_k[i]; }
    }
    out[0] = bk;
  }
}

__global__ void overflow_count_kernel(const int32_t* __restrict__ rowptr, int64_t nrows,
                                      int64_t K, int32_t* __restrict__ cnt) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nrows) cnt[i] = (int32_t)max((int64_t)0, (int64_t)(rowptr[i + 1] - rowptr[i]) - K);
}

// --- value type changes ----------------------------------------------------

__global__ void f64_to_f32_kernel(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];  // round to nearest even
}

__global__ void f32_to_f64_kernel(const float* __restrict__ a, double* __restrict__ b, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (double)a[i];
}

template <class W>
void build_typed(dynmat_s* A, const int32_t* row, const int32_t* col, const W* val, int64_t nnz,
                 dynmat_format fmt, cudaStream_t s) {
  const int64_t N = A->nrows, M = A->ncols;
  const int64_t vb = sizeof(W);
  const int64_t csr_bytes = (4 + vb) * nnz + 4 * (N + 1);
  switch (fmt) {
    case DYNMAT_COO: {
      A->coo.nnz = nnz;
      A->coo.row.alloc(nnz * 4, s);
      A->coo.col.alloc(nnz * 4, s);
      A->coo.val.alloc(nnz * vb, s);
      if (nnz) {
        DM_CUDA(cudaMemcpyAsync(A->coo.row.p, row, nnz * 4, cudaMemcpyDeviceToDevice, s));
        DM_CUDA(cudaMemcpyAsync(A->coo.col.p, col, nnz * 4, cudaMemcpyDeviceToDevice, s));
        DM_CUDA(cudaMemcpyAsync(A->coo.val.p, val, nnz * vb, cudaMemcpyDeviceToDevice, s));
      }
      break;
    }
    case DYNMAT_CSR: {
      A->csr.nnz = nnz;
      A->csr.rowptr.alloc((N + 1) * 4, s);
      A->csr.col.alloc(nnz * 4, s);
      A->csr.val.alloc(nnz * vb, s);
      csr_rowptr_from_rows(row, nnz, N, A->csr.rowptr.as<int32_t>(), s);
      if (nnz) {
        DM_CUDA(cudaMemcpyAsync(A->csr.col.p, col, nnz * 4, cudaMemcpyDeviceToDevice, s));
        DM_CUDA(cudaMemcpyAsync(A->csr.val.p, val, nnz * vb, cudaMemcpyDeviceToDevice, s));
      }
      break;
    }
    case DYNMAT_DIA: {
      const int64_t span = N + M - 1;
      int64_t ndiag = 0;
      DBuf flag, idx;
      if (span > 0 && nnz > 0) {
        flag.alloc(span * 4, s);
        idx.alloc(span * 4, s);
        DM_CUDA(cudaMemsetAsync(flag.p, 0, span * 4, s));
        mark_offsets(row, col, nnz, N, flag.as<int32_t>(), s);
        exclusive_scan_i32(flag.as<int32_t>(), idx.as<int32_t>(), span, &ndiag, s);
      }
      const int64_t dia_bytes = vb * ndiag * N + 4 * ndiag;
      DM_REQUIRE((double)dia_bytes <= g_pad_limit * (double)csr_bytes || nnz == 0,
                 DYNMAT_ERR_FORMAT_TOO_LARGE,
                 "DIA needs %lld diagonals (%lld bytes), over %.3g x the CSR bytes (%lld)",
                 (long long)ndiag, (long long)dia_bytes, g_pad_limit, (long long)csr_bytes);
      const int64_t ld = lead_dim(N);
      A->dia.ndiag = ndiag;
      A->dia.ld = ld;
      A->dia.offsets.alloc(std::max<int64_t>(ndiag, 1) * 4, s);
      A->dia.val.alloc(std::max<int64_t>(ndiag * ld, 1) * vb, s);
      if (ndiag) {
        dia_offsets_kernel<<<grid_for(span), T, 0, s>>>(flag.as<int32_t>(), idx.as<int32_t>(),
                                                        span, N, A->dia.offsets.as<int32_t>());
        DM_CHECK_LAUNCH();
        DM_CUDA(cudaMemsetAsync(A->dia.val.p, 0, ndiag * ld * vb, s));
        DBuf rowptr((N + 1) * 4, s);
        csr_rowptr_from_rows(row, nnz, N, rowptr.as<int32_t>(), s);
        dia_scatter_kernel<W><<<grid_for(N), T, 0, s>>>(rowptr.as<int32_t>(), col, val, N, ld,
                                                        idx.as<int32_t>(), A->dia.val.as<W>());
        DM_CHECK_LAUNCH();
      }
      break;
    }
    case DYNMAT_ELL:
    case DYNMAT_HYB: {
      DBuf rowptr((N + 1) * 4, s), len(std::max<int64_t>(N, 1) * 4, s);
      csr_rowptr_from_rows(row, nnz, N, rowptr.as<int32_t>(), s);
      row_lengths_kernel<<<grid_for(N), T, 0, s>>>(rowptr.as<int32_t>(), N, len.as<int32_t>());
      DM_CHECK_LAUNCH();
      const int64_t maxlen = reduce_max_i32(len.as<int32_t>(), N, s);
      const int64_t ld = lead_dim(N);
      int64_t K = maxlen, over = 0;
      DBuf cstart;
      if (fmt == DYNMAT_HYB) {
        K = hyb_width(rowptr.as<int32_t>(), N, maxlen, vb, s);
        DBuf ocnt(std::max<int64_t>(N, 1) * 4, s);
        cstart.alloc(std::max<int64_t>(N, 1) * 4, s);
        overflow_count_kernel<<<grid_for(N), T, 0, s>>>(rowptr.as<int32_t>(), N, K,
                                                        ocnt.as<int32_t>());
        DM_CHECK_LAUNCH();
        exclusive_scan_i32(ocnt.as<int32_t>(), cstart.as<int32_t>(), N, &over, s);
      } else {
        const int64_t ell_bytes = (4 + vb) * maxlen * N;
        DM_REQUIRE((double)ell_bytes <= g_pad_limit * (double)csr_bytes || nnz == 0,
                   DYNMAT_ERR_FORMAT_TOO_LARGE,
                   "ELL width %lld (%lld bytes) is over %.3g x the CSR bytes (%lld)",
                   (long long)maxlen, (long long)ell_bytes, g_pad_limit, (long long)csr_bytes);
      }
      A->ell.K = K;
      A->ell.ld = ld;
      A->ell.col.alloc(std::max<int64_t>(K * ld, 1) * 4, s);
      A->ell.val.alloc(std::max<int64_t>(K * ld, 1) * vb, s);
      if (fmt == DYNMAT_HYB) {
        A->coo.nnz = over;
        A->coo.row.alloc(over * 4, s);
        A->coo.col.alloc(over * 4, s);
        A->coo.val.alloc(over * vb, s);
      }
      if (K > 0 || over > 0) {
        ell_fill_kernel<W><<<grid_for(ld), T, 0, s>>>(
            rowptr.as<int32_t>(), col, val, N, ld, K, A->ell.col.as<int32_t>(), A->ell.val.as<W>(),
            fmt == DYNMAT_HYB ? cstart.as<int32_t>() : nullptr,
            fmt == DYNMAT_HYB ? A->coo.row.as<int32_t>() : nullptr,
            fmt == DYNMAT_HYB ? A->coo.col.as<int32_t>() : nullptr,
            fmt == DYNMAT_HYB ? A->coo.val.as<W>() : nullptr);
        DM_CHECK_LAUNCH();
      }
      break;
    }
  }
  A->nnz = nnz;
  A->fmt = fmt;
}

template <class W>
void to_coo_typed(const dynmat_s* A, Coo& out, cudaStream_t s) {
  const int64_t N = A->nrows, M = A->ncols;
  const int64_t vb = sizeof(W);
  switch (A->fmt) {
    case DYNMAT_COO:
    case DYNMAT_CSR: {
      const int64_t nnz = A->fmt == DYNMAT_COO ? A->coo.nnz : A->csr.nnz;
      out.nnz = nnz;
      out.row.alloc(nnz * 4, s);
      out.col.alloc(nnz * 4, s);
      out.val.alloc(nnz * vb, s);
      if (!nnz) break;
      if (A->fmt == DYNMAT_COO) {
        DM_CUDA(cudaMemcpyAsync(out.row.p, A->coo.row.p, nnz * 4, cudaMemcpyDeviceToDevice, s));
        DM_CUDA(cudaMemcpyAsync(out.col.p, A->coo.col.p, nnz * 4, cudaMemcpyDeviceToDevice, s));
        DM_CUDA(cudaMemcpyAsync(out.val.p, A->coo.val.p, nnz * vb, cudaMemcpyDeviceToDevice, s));
      } else {
        expand_rows_kernel<<<group_grid(cdiv(N, 32), 32), T, 0, s>>>(A->csr.rowptr.as<int32_t>(),
                                                                      N, out.row.as<int32_t>());
        DM_CHECK_LAUNCH();
        DM_CUDA(cudaMemcpyAsync(out.col.p, A->csr.col.p, nnz * 4, cudaMemcpyDeviceToDevice, s));
        DM_CUDA(cudaMemcpyAsync(out.val.p, A->csr.val.p, nnz * vb, cudaMemcpyDeviceToDevice, s));
      }
      break;
    }
    case DYNMAT_DIA: {
      DBuf cnt(std::max<int64_t>(N, 1) * 4, s), start(std::max<int64_t>(N, 1) * 4, s);
      int64_t m = 0;
      if (N > 0) {
        dia_count_kernel<W><<<grid_for(N), T, 0, s>>>(A->dia.offsets.as<int32_t>(), A->dia.ndiag,
                                                      A->dia.val.as<W>(), N, M, A->dia.ld,
                                                      cnt.as<int32_t>());
        DM_CHECK_LAUNCH();
        exclusive_scan_i32(cnt.as<int32_t>(), start.as<int32_t>(), N, &m, s);
      }
      out.nnz = m;
      out.row.alloc(m * 4, s);
      out.col.alloc(m * 4, s);
      out.val.alloc(m * vb, s);
      if (m && emit_tiled_smem<W, true>(A->dia.ndiag) <= 48 * 1024) {
        emit_tiled_kernel<W, true><<<(unsigned)cdiv(N, ET), T,
                                     emit_tiled_smem<W, true>(A->dia.ndiag), s>>>(
            nullptr, A->dia.offsets.as<int32_t>(), A->dia.val.as<W>(), N, M, A->dia.ld,
            A->dia.ndiag, nullptr, nullptr, nullptr, 0, start.as<int32_t>(),
            out.row.as<int32_t>(), out.col.as<int32_t>(), out.val.as<W>());
        DM_CHECK_LAUNCH();
      } else if (m) {
        if (A->dia.ndiag > 8)
          dia_emit_kernel<W, 32><<<group_grid(N, 32), T, 0, s>>>(
              A->dia.offsets.as<int32_t>(), A->dia.ndiag, A->dia.val.as<W>(), N, M, A->dia.ld,
              start.as<int32_t>(), out.row.as<int32_t>(), out.col.as<int32_t>(), out.val.as<W>());
        else
          dia_emit_kernel<W, 8><<<group_grid(N, 8), T, 0, s>>>(
              A->dia.offsets.as<int32_t>(), A->dia.ndiag, A->dia.val.as<W>(), N, M, A->dia.ld,
              start.as<int32_t>(), out.row.as<int32_t>(), out.col.as<int32_t>(), out.val.as<W>());
        DM_CHECK_LAUNCH();
      }
      break;
    }
    case DYNMAT_ELL:
    case DYNMAT_HYB: {
      const bool hyb = A->fmt == DYNMAT_HYB;
      const int32_t* crow = hyb ? A->coo.row.as<int32_t>() : nullptr;
      const int64_t ncoo = hyb ? A->coo.nnz : 0;
      DBuf cnt(std::max<int64_t>(N, 1) * 4, s), start(std::max<int64_t>(N, 1) * 4, s);
      int64_t m = 0;
      if (N > 0) {
        ell_count_kernel<<<grid_for(N), T, 0, s>>>(A->ell.col.as<int32_t>(), N, A->ell.ld,
                                                   A->ell.K, crow, ncoo, cnt.as<int32_t>());
        DM_CHECK_LAUNCH();
        exclusive_scan_i32(cnt.as<int32_t>(), start.as<int32_t>(), N, &m, s);
      }
      out.nnz = m;
      out.row.alloc(m * 4, s);
      out.col.alloc(m * 4, s);
      out.val.alloc(m * vb, s);
      const int32_t* hc = hyb ? A->coo.col.as<int32_t>() : nullptr;
      const W* hv = hyb ? A->coo.val.as<W>() : nullptr;
      if (m && A->ell.K > 0 && emit_tiled_smem<W, false>(A->ell.K) <= 48 * 1024) {
        emit_tiled_kernel<W, false><<<(unsigned)cdiv(N, ET), T,
                                      emit_tiled_smem<W, false>(A->ell.K), s>>>(
            A->ell.col.as<int32_t>(), nullptr, A->ell.val.as<W>(), N, M, A->ell.ld, A->ell.K,
            crow, hc, hv, ncoo, start.as<int32_t>(), out.row.as<int32_t>(),
            out.col.as<int32_t>(), out.val.as<W>());
        DM_CHECK_LAUNCH();
      } else if (m) {
        if (A->ell.K > 8)
          ell_emit_kernel<W, 32><<<group_grid(N, 32), T, 0, s>>>(
              A->ell.col.as<int32_t>(), A->ell.val.as<W>(), N, A->ell.ld, A->ell.K, crow, hc, hv,
              ncoo, start.as<int32_t>(), out.row.as<int32_t>(), out.col.as<int32_t>(),
              out.val.as<W>());
        else
          ell_emit_kernel<W, 8><<<group_grid(N, 8), T, 0, s>>>(
              A->ell.col.as<int32_t>(), A->ell.val.as<W>(), N, A->ell.ld, A->ell.K, crow, hc, hv,
              ncoo, start.as<int32_t>(), out.row.as<int32_t>(), out.col.as<int32_t>(),
              out.val.as<W>());
        DM_CHECK_LAUNCH();
      }
      break;
    }
  }
}

}  // namespace

// K_h of the HYB split for rows given by `rowptr` (blocking).
int64_t hyb_width(const int32_t* rowptr, int64_t N, int64_t maxlen, int64_t vb, cudaStream_t s) {
  DBuf hist((maxlen + 1) * 4, s), kout(16, s);
  DM_CUDA(cudaMemsetAsync(hist.p, 0, (maxlen + 1) * 4, s));
  if (N > 0) {
    len_hist_kernel<<<grid_for(N), T, 0, s>>>(rowptr, N, hist.as<int32_t>());
    DM_CHECK_LAUNCH();
  }
  hyb_width_kernel<<<1, 1024, 0, s>>>(hist.as<int32_t>(), maxlen, N, 4 + vb, 8 + vb,
                                      kout.as<int64_t>());
  DM_CHECK_LAUNCH();
  int64_t kh = 0;
  DM_CUDA(cudaMemcpyAsync(&kh, kout.p, 8, cudaMemcpyDeviceToHost, s));
  DM_CUDA(cudaStreamSynchronize(s));
  return kh;
}

void mark_offsets(const int32_t* row, const int32_t* col, int64_t nnz, int64_t nrows,
                  int32_t* flag, cudaStream_t s) {
  if (nnz <= 0) return;
  const unsigned grid = (unsigned)std::max<int64_t>(
      1, std::min<int64_t>(cdiv(cdiv(nnz, 4), T), (int64_t)device().sms * 8));
  if ((((uintptr_t)row | (uintptr_t)col) & 15u) == 0)
    mark_offsets_kernel<true><<<grid, T, 0, s>>>(row, col, nnz, nrows, flag);
  else
    mark_offsets_kernel<false><<<grid, T, 0, s>>>(row, col, nnz, nrows, flag);
  DM_CHECK_LAUNCH();
}

void csr_rowptr_from_rows(const int32_t* row, int64_t nnz, int64_t nrows, int32_t* rowptr,
                          cudaStream_t s) {
  rowptr_kernel<<<grid_for(nrows + 1), T, 0, s>>>(row, nnz, nrows, rowptr);
  DM_CHECK_LAUNCH();
}

void to_coo(const dynmat_s* A, Coo& out, cudaStream_t s) {
  if (A->vdt == DYNMAT_F64) to_coo_typed<uint64_t>(A, out, s);
  else to_coo_typed<uint32_t>(A, out, s);
}

// Builds `fmt` with value type `vdt` into the (empty) arrays of A from a
// canonical COO whose values have A->vdt; converts the value type first.
void build_from_coo(dynmat_s* A, const Coo& src, dynmat_format fmt, dynmat_dtype vdt,
                    cudaStream_t s) {
  const int64_t nnz = src.nnz;
  const void* val = src.val.p;
  DBuf conv;
  if (vdt != A->vdt) {
    conv.alloc(nnz * vsize(vdt), s);
    if (nnz) {
      if (vdt == DYNMAT_F32)
        f64_to_f32_kernel<<<grid_for(nnz), T, 0, s>>>(src.val.as<double>(), conv.as<float>(), nnz);
      else
        f32_to_f64_kernel<<<grid_for(nnz), T, 0, s>>>(src.val.as<float>(), conv.as<double>(), nnz);
      DM_CHECK_LAUNCH();
    }
    val = conv.p;
  }
  A->vdt = vdt;
  if (vdt == DYNMAT_F64)
    build_typed<uint64_t>(A, src.row.as<int32_t>(), src.col.as<int32_t>(),
                          (const uint64_t*)val, nnz, fmt, s);
  else
    build_typed<uint32_t>(A, src.row.as<int32_t>(), src.col.as<int32_t>(),
                          (const uint32_t*)val, nnz, fmt, s);
}

}  // namespace dm
