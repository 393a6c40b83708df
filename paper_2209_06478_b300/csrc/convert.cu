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

template <class W>
__device__ __forceinline__ bool word_is_zero(W w) {
  return (W)(w << 1) == 0;  // +0.0 or -0.0
}

// --- CSR ------------------------------------------------------------------

// rowptr[i] = first entry whose row >= i (lower bound in the sorted rows).
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

// row[e] = the row whose range [rowptr[r], rowptr[r+1]) holds e.
__global__ void expand_rows_kernel(const int32_t* __restrict__ rowptr, int64_t nrows,
                                   int64_t nnz, int32_t* __restrict__ row) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nnz) return;
  int64_t lo = 0, hi = nrows;  // largest r with rowptr[r] <= e
  while (hi - lo > 1) {
    int64_t mid = (lo + hi) >> 1;
    if (rowptr[mid] <= e) lo = mid; else hi = mid;
  }
  row[e] = (int32_t)lo;
}

__global__ void row_lengths_kernel(const int32_t* __restrict__ rowptr, int64_t nrows,
                                   int32_t* __restrict__ len) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nrows) len[i] = rowptr[i + 1] - rowptr[i];
}

// --- DIA ------------------------------------------------------------------

__global__ void dia_mark_kernel(const int32_t* __restrict__ row, const int32_t* __restrict__ col,
                                int64_t nnz, int64_t nrows, int32_t* __restrict__ flag) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < nnz) flag[(int64_t)col[e] - row[e] + (nrows - 1)] = 1;
}

__global__ void dia_offsets_kernel(const int32_t* __restrict__ flag,
                                   const int32_t* __restrict__ idx, int64_t span, int64_t nrows,
                                   int32_t* __restrict__ offsets) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < span && flag[k]) offsets[idx[k]] = (int32_t)(k - (nrows - 1));
}

template <class W>
__global__ void dia_scatter_kernel(const int32_t* __restrict__ row,
                                   const int32_t* __restrict__ col, const W* __restrict__ val,
                                   int64_t nnz, int64_t nrows, int64_t ld,
                                   const int32_t* __restrict__ idx, W* __restrict__ dval) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nnz) return;
  int64_t d = idx[(int64_t)col[e] - row[e] + (nrows - 1)];
  dval[d * ld + row[e]] = val[e];
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

template <class W>
__global__ void dia_emit_kernel(const int32_t* __restrict__ offsets, int64_t ndiag,
                                const W* __restrict__ dval, int64_t nrows, int64_t ncols,
                                int64_t ld, const int32_t* __restrict__ start,
                                int32_t* __restrict__ orow, int32_t* __restrict__ ocol,
                                W* __restrict__ oval) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrows) return;
  int64_t m = start[i];
  for (int64_t d = 0; d < ndiag; ++d) {
    int64_t j = i + offsets[d];
    if (j < 0 || j >= ncols) continue;
    W w = dval[d * ld + i];
    if (word_is_zero(w)) continue;
    orow[m] = (int32_t)i;
    ocol[m] = (int32_t)j;
    oval[m] = w;
    ++m;
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

template <class W>
__global__ void ell_emit_kernel(const int32_t* __restrict__ ecol, const W* __restrict__ evl,
                                int64_t nrows, int64_t ld, int64_t K,
                                const int32_t* __restrict__ crow,
                                const int32_t* __restrict__ ccol, const W* __restrict__ cval,
                                int64_t ncoo, const int32_t* __restrict__ start,
                                int32_t* __restrict__ orow, int32_t* __restrict__ ocol,
                                W* __restrict__ oval) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrows) return;
  int64_t m = start[i];
  for (int64_t k = 0; k < K; ++k) {
    int32_t c = ecol[k * ld + i];
    if (c < 0) continue;
    orow[m] = (int32_t)i;
    ocol[m] = c;
    oval[m] = evl[k * ld + i];
    ++m;
  }
  if (crow) {
    int64_t lo = 0, hi = ncoo;
    while (lo < hi) { int64_t mm = (lo + hi) >> 1; if (crow[mm] < i) lo = mm + 1; else hi = mm; }
    for (int64_t e = lo; e < ncoo && crow[e] == i; ++e, ++m) {
      orow[m] = (int32_t)i;
      ocol[m] = ccol[e];
      oval[m] = cval[e];
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
        dia_mark_kernel<<<grid_for(nnz), T, 0, s>>>(row, col, nnz, N, flag.as<int32_t>());
        DM_CHECK_LAUNCH();
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
        dia_scatter_kernel<W><<<grid_for(nnz), T, 0, s>>>(row, col, val, nnz, N, ld,
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
        expand_rows_kernel<<<grid_for(nnz), T, 0, s>>>(A->csr.rowptr.as<int32_t>(), N, nnz,
                                                        out.row.as<int32_t>());
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
      if (m) {
        dia_emit_kernel<W><<<grid_for(N), T, 0, s>>>(
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
      if (m) {
        ell_emit_kernel<W><<<grid_for(N), T, 0, s>>>(
            A->ell.col.as<int32_t>(), A->ell.val.as<W>(), N, A->ell.ld, A->ell.K, crow,
            hyb ? A->coo.col.as<int32_t>() : nullptr, hyb ? A->coo.val.as<W>() : nullptr, ncoo,
            start.as<int32_t>(), out.row.as<int32_t>(), out.col.as<int32_t>(), out.val.as<W>());
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
