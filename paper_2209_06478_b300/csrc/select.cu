// Run-time format selection (§IV-B picks the format at run time; §V-E's
// auto-tuner profiles each format and keeps the fastest).
//
// FEATURES mode: integer features of the COO view computed on the GPU and a
// deterministic byte-model rule evaluated by a one-thread kernel, so the
// choice is exactly reproducible. PROFILE mode: convert a copy to every
// admissible format (and every CSR kernel variant), time the SpMV with CUDA
// events and keep the fastest.
#include <algorithm>
#include <memory>
#include <vector>

#include "device.cuh"
#include "internal.cuh"

namespace dm {

// Kernel variants of a format run 1..variant_max (dynmat_set_variant): CSR 8,
// DIA 7, COO, ELL and HYB 2.
int variant_max(dynmat_format f) { return f == DYNMAT_CSR ? 8 : (f == DYNMAT_DIA ? 7 : 2); }

namespace {

constexpr int T = 256;

// sum of int32 flags / max(0, len - K) over rows, into an int64 slot
__global__ void count_kernel(const int32_t* __restrict__ flag, int64_t n,
                             unsigned long long* __restrict__ out) {
  unsigned long long c = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    c += (unsigned long long)flag[i];
  c = warp_sum(c);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

__global__ void overflow_kernel(const int32_t* __restrict__ rowptr, int64_t nrows, int64_t K,
                                unsigned long long* __restrict__ out) {
  unsigned long long c = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nrows;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t l = rowptr[i + 1] - rowptr[i];
    if (l > K) c += (unsigned long long)(l - K);
  }
  c = warp_sum(c);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

__global__ void lengths_kernel(const int32_t* __restrict__ rowptr, int64_t nrows,
                               int32_t* __restrict__ len) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nrows) len[i] = rowptr[i + 1] - rowptr[i];
}

// The rule: modelled bytes per format, padded formats over guard x CSR are
// excluded, the smallest wins, ties in the order DIA, ELL, CSR, HYB, COO.
__global__ void rule_kernel(dynmat_features* f, int64_t vb) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int64_t N = f->nrows, v = vb;
  f->bytes[DYNMAT_COO] = (8 + v) * f->nnz;
  f->bytes[DYNMAT_CSR] = (4 + v) * f->nnz + 4 * (N + 1);
  f->bytes[DYNMAT_DIA] = v * f->ndiag * N + 4 * f->ndiag;
  f->bytes[DYNMAT_ELL] = (4 + v) * f->maxlen * N;
  f->bytes[DYNMAT_HYB] = (4 + v) * f->hyb_k * N + (8 + v) * f->hyb_over;
  const int order[5] = {DYNMAT_DIA, DYNMAT_ELL, DYNMAT_CSR, DYNMAT_HYB, DYNMAT_COO};
  int best = -1;
  for (int t = 0; t < 5; ++t) {
    const int fm = order[t];
    if ((fm == DYNMAT_DIA || fm == DYNMAT_ELL) &&
        f->bytes[fm] > (int64_t)f->guard * f->bytes[DYNMAT_CSR])
      continue;
    if (best < 0 || f->bytes[fm] < f->bytes[best]) best = fm;
  }
  f->choice = best;
}

unsigned grid_of(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(n, T), (int64_t)device().sms * 16));
}

}  // namespace

void compute_features(const dynmat_s* A, int32_t guard, dynmat_features* out, cudaStream_t s) {
  Coo tmp;
  const Coo* c = &A->coo;
  if (A->fmt != DYNMAT_COO) {
    to_coo(A, tmp, s);
    c = &tmp;
  }
  const int64_t N = A->nrows, M = A->ncols, nnz = c->nnz;
  const int64_t vb = vsize(A->vdt);
  dynmat_features h{};
  h.nrows = N;
  h.ncols = M;
  h.nnz = nnz;
  h.guard = guard;
  DBuf cnt(16, s);
  DM_CUDA(cudaMemsetAsync(cnt.p, 0, 16, s));
  const int64_t span = N + M - 1;
  if (nnz > 0 && span > 0) {
    DBuf flag(span * 4, s);
    DM_CUDA(cudaMemsetAsync(flag.p, 0, span * 4, s));
    mark_offsets(c->row.as<int32_t>(), c->col.as<int32_t>(), nnz, N, flag.as<int32_t>(), s);
    count_kernel<<<grid_of(span), T, 0, s>>>(flag.as<int32_t>(), span,
                                             cnt.as<unsigned long long>());
    DM_CHECK_LAUNCH();
  }
  DBuf rowptr((N + 1) * 4, s), len(std::max<int64_t>(N, 1) * 4, s);
  csr_rowptr_from_rows(c->row.as<int32_t>(), nnz, N, rowptr.as<int32_t>(), s);
  if (N > 0) {
    lengths_kernel<<<(unsigned)cdiv(N, T), T, 0, s>>>(rowptr.as<int32_t>(), N, len.as<int32_t>());
    DM_CHECK_LAUNCH();
  }
  h.maxlen = reduce_max_i32(len.as<int32_t>(), N, s);
  h.hyb_k = hyb_width(rowptr.as<int32_t>(), N, h.maxlen, vb, s);
  if (N > 0) {
    overflow_kernel<<<grid_of(N), T, 0, s>>>(rowptr.as<int32_t>(), N, h.hyb_k,
                                             cnt.as<unsigned long long>() + 1);
    DM_CHECK_LAUNCH();
  }
  unsigned long long hc[2] = {0, 0};
  DM_CUDA(cudaMemcpyAsync(hc, cnt.p, 16, cudaMemcpyDeviceToHost, s));
  DM_CUDA(cudaStreamSynchronize(s));
  h.ndiag = (int64_t)hc[0];
  h.hyb_over = (int64_t)hc[1];
  DBuf df(sizeof(dynmat_features), s);
  DM_CUDA(cudaMemcpyAsync(df.p, &h, sizeof h, cudaMemcpyHostToDevice, s));
  rule_kernel<<<1, 32, 0, s>>>(df.as<dynmat_features>(), vb);
  DM_CHECK_LAUNCH();
  DM_CUDA(cudaMemcpyAsync(out, df.p, sizeof h, cudaMemcpyDeviceToHost, s));
  DM_CUDA(cudaStreamSynchronize(s));
}

// Median SpMV time of A (ms) with CUDA events on stream s.
double time_spmv(const dynmat_s* A, const void* x, void* y, dynmat_dtype vdt, cudaStream_t s,
                 int reps) {
  cudaEvent_t e0, e1;
  DM_CUDA(cudaEventCreate(&e0));
  DM_CUDA(cudaEventCreate(&e1));
  std::vector<float> t;
  for (int k = 0; k < reps + 2; ++k) {
    DM_CUDA(cudaEventRecord(e0, s));
    spmv(A, x, y, vdt, s);
    DM_CUDA(cudaEventRecord(e1, s));
    DM_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    DM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (k >= 2) t.push_back(ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::sort(t.begin(), t.end());
  return t[t.size() / 2];
}

// §V-E: profile every admissible format (and every CSR variant) and return
// the fastest; A itself is not modified.
void profile_select(const dynmat_s* A, dynmat_format* best_fmt, int32_t* best_variant,
                    cudaStream_t s) {
  dynmat_features f;
  compute_features(A, 3, &f, s);
  Coo tmp;
  const Coo* c = &A->coo;
  if (A->fmt != DYNMAT_COO) {
    to_coo(A, tmp, s);
    c = &tmp;
  }
  const size_t vb = vsize(A->vdt);
  DBuf x(std::max<int64_t>(A->ncols, 1) * vb, s), y(std::max<int64_t>(A->nrows, 1) * vb, s);
  DM_CUDA(cudaMemsetAsync(x.p, 0, x.bytes, s));
  double best = 1e30;
  *best_fmt = (dynmat_format)f.choice;
  *best_variant = 0;
  const dynmat_format order[5] = {DYNMAT_DIA, DYNMAT_ELL, DYNMAT_CSR, DYNMAT_HYB, DYNMAT_COO};
  for (dynmat_format fm : order) {
    if ((fm == DYNMAT_DIA || fm == DYNMAT_ELL) && f.bytes[fm] > 3 * f.bytes[DYNMAT_CSR]) continue;
    auto T2 = std::make_unique<dynmat_s>();
    T2->nrows = A->nrows;
    T2->ncols = A->ncols;
    T2->vdt = A->vdt;
    try {
      build_from_coo(T2.get(), *c, fm, A->vdt, s);
    } catch (const Fail&) {
      clear_error();
      continue;  // e.g. over the padding limit: not a candidate
    }
    for (int v = 1; v <= variant_max(fm); ++v) {
      T2->plan.forced = v;
      prepare_spmv(T2.get(), s);
      const double ms = time_spmv(T2.get(), x.p, y.p, A->vdt, s, 5);
      if (ms < best) {
        best = ms;
        *best_fmt = fm;
        *best_variant = v;
      }
    }
    free_format(T2.get(), s);
  }
  DM_CUDA(cudaStreamSynchronize(s));
}

}  // namespace dm

using namespace dm;

extern "C" {

dynmat_status dynmat_features_get(dynmat_t A, int32_t pad_guard, dynmat_features* out,
                                  dynmat_stream_t stream) {
  return dm::guard([&] {
    DM_REQUIRE(A && out, DYNMAT_ERR_INVALID_ARG, "null argument");
    DM_REQUIRE(pad_guard > 0, DYNMAT_ERR_INVALID_ARG, "guard must be positive");
    compute_features(A, pad_guard, out, (cudaStream_t)stream);
  });
}

dynmat_status dynmat_select_format(dynmat_t A, int mode, dynmat_format* out,
                                   dynmat_stream_t stream) {
  return dm::guard([&] {
    DM_REQUIRE(A && out, DYNMAT_ERR_INVALID_ARG, "null argument");
    DM_REQUIRE(mode == DYNMAT_SELECT_FEATURES || mode == DYNMAT_SELECT_PROFILE,
               DYNMAT_ERR_INVALID_ARG, "bad mode %d", mode);
    cudaStream_t s = (cudaStream_t)stream;
    if (mode == DYNMAT_SELECT_FEATURES) {
      dynmat_features f;
      compute_features(A, 3, &f, s);
      *out = (dynmat_format)f.choice;
    } else {
      int32_t v = 0;
      profile_select(A, out, &v, s);
    }
  });
}

dynmat_status dynmat_tune_variant(dynmat_t A, int32_t* variant_out, dynmat_stream_t stream) {
  return dm::guard([&] {
    DM_REQUIRE(A, DYNMAT_ERR_INVALID_ARG, "null handle");
    cudaStream_t s = (cudaStream_t)stream;
    const int vlo = 1, vhi = dm::variant_max(A->fmt);
    if (A->nrows > 0) {
      const size_t vb = vsize(A->vdt);
      DBuf x(std::max<int64_t>(A->ncols, 1) * vb, s), y(std::max<int64_t>(A->nrows, 1) * vb, s);
      DM_CUDA(cudaMemsetAsync(x.p, 0, x.bytes, s));
      // The automatic variant is the incumbent; another must beat it by 2%
      // (timing noise must not flip the choice).
      A->plan.forced = 0;
      prepare_spmv(A, s);
      int bv = std::max(A->plan.variant, vlo);
      A->plan.forced = bv;
      prepare_spmv(A, s);
      double best = time_spmv(A, x.p, y.p, A->vdt, s, 5);
      for (int v = vlo; v <= vhi; ++v) {
        if (v == bv) continue;
        A->plan.forced = v;
        prepare_spmv(A, s);
        const double ms = time_spmv(A, x.p, y.p, A->vdt, s, 5);
        if (ms < 0.98 * best) {
          best = ms;
          bv = v;
        }
      }
      A->plan.forced = bv;
      prepare_spmv(A, s);
      DM_CUDA(cudaStreamSynchronize(s));
    }
    if (variant_out) *variant_out = A->plan.variant;
  });
}

dynmat_status dynmat_autotune(dynmat_t A, dynmat_format* fmt_out, int32_t* variant_out,
                              dynmat_stream_t stream) {
  return dm::guard([&] {
    DM_REQUIRE(A, DYNMAT_ERR_INVALID_ARG, "null handle");
    cudaStream_t s = (cudaStream_t)stream;
    dynmat_format f = DYNMAT_CSR;
    int32_t v = 0;
    profile_select(A, &f, &v, s);
    convert_impl(A, f, A->vdt, s);
    if (v) {
      A->plan.forced = v;
      prepare_spmv(A, s);
      DM_CUDA(cudaStreamSynchronize(s));
    }
    if (fmt_out) *fmt_out = f;
    if (variant_out) *variant_out = A->plan.variant;
  });
}

}  // extern "C"
