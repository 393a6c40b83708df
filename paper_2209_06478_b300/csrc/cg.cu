// Conjugate gradient (§II-B: HPCG's CG; §IV-B: with the preconditioner
// disabled) and mixed-precision iterative refinement around an FP32 CG.
//
// One CG iteration is three launches on the caller's stream:
//   1. q = A p fused with p.q (tile partials, last block forms sigma and
//      alpha = rho / sigma, or flags breakdown);
//   2. x += alpha p, r -= alpha q fused with r.r (last block: convergence
//      test, beta = rho' / rho);
//   3. p = r + beta p.
// The scalars live on the device (CgState), every kernel returns at once when
// the solve is done, and `check_every` iterations are captured in one CUDA
// graph, so the host only reads the state between graph launches.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <memory>

#include "device.cuh"
#include "internal.cuh"

namespace dm {

namespace {

constexpr int NT = 256;

// 16-byte vectors of the CG vector type (2 doubles or 4 floats).
template <class X> struct V16;
template <> struct V16<double> {
  using T = double2;
  static constexpr int R = 2;
  __device__ static void get(const T& v, double* o) { o[0] = v.x; o[1] = v.y; }
  __device__ static T put(const double* o) { return make_double2(o[0], o[1]); }
};
template <> struct V16<float> {
  using T = float4;
  static constexpr int R = 4;
  __device__ static void get(const T& v, float* o) { o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w; }
  __device__ static T put(const float* o) { return make_float4(o[0], o[1], o[2], o[3]); }
};

// x += alpha p; r -= alpha q; r.r. Grid-stride over 16-byte groups (2
// doubles or 4 floats of each vector), two groups' loads in flight per
// thread, scalar tail; one partial of r.r per block.
template <class X>
__global__ void __launch_bounds__(NT)
cg_update_kernel(int64_t N, X* __restrict__ x, X* __restrict__ r, const X* __restrict__ p,
                 const X* __restrict__ q, DotSpec dot) {
  using VT = typename V16<X>::T;
  constexpr int R = V16<X>::R;
  constexpr int U = 2;
  __shared__ double scratch[NT];
  if (dot.st->done) return;
  const X a = (X)dot.st->alpha;
  const bool vec = (((uintptr_t)x | (uintptr_t)r | (uintptr_t)p | (uintptr_t)q) & 15u) == 0;
  const int64_t nv = vec ? N / R : 0;
  const int64_t stride = (int64_t)gridDim.x * NT;
  double part = 0.0;
  int64_t k = (int64_t)blockIdx.x * NT + threadIdx.x;
  for (; k + (U - 1) * stride < nv; k += U * stride) {
    X xv[U][R], pv[U][R], rv[U][R], qv[U][R];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t g = (k + u * stride) * R;
      V16<X>::get(*reinterpret_cast<const VT*>(x + g), xv[u]);
      V16<X>::get(*reinterpret_cast<const VT*>(p + g), pv[u]);
      V16<X>::get(*reinterpret_cast<const VT*>(r + g), rv[u]);
      V16<X>::get(*reinterpret_cast<const VT*>(q + g), qv[u]);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
#pragma unroll
      for (int j = 0; j < R; ++j) {
        xv[u][j] = fma(a, pv[u][j], xv[u][j]);
        rv[u][j] = fma(-a, qv[u][j], rv[u][j]);
        part = fma((double)rv[u][j], (double)rv[u][j], part);
      }
      const int64_t g = (k + u * stride) * R;
      *reinterpret_cast<VT*>(x + g) = V16<X>::put(xv[u]);
      *reinterpret_cast<VT*>(r + g) = V16<X>::put(rv[u]);
    }
  }
  for (; k < nv; k += stride) {
    X xv[R], pv[R], rv[R], qv[R];
    V16<X>::get(*reinterpret_cast<const VT*>(x + k * R), xv);
    V16<X>::get(*reinterpret_cast<const VT*>(p + k * R), pv);
    V16<X>::get(*reinterpret_cast<const VT*>(r + k * R), rv);
    V16<X>::get(*reinterpret_cast<const VT*>(q + k * R), qv);
#pragma unroll
    for (int j = 0; j < R; ++j) {
      xv[j] = fma(a, pv[j], xv[j]);
      rv[j] = fma(-a, qv[j], rv[j]);
      part = fma((double)rv[j], (double)rv[j], part);
    }
    *reinterpret_cast<VT*>(x + k * R) = V16<X>::put(xv);
    *reinterpret_cast<VT*>(r + k * R) = V16<X>::put(rv);
  }
  for (int64_t i = nv * R + (int64_t)blockIdx.x * NT + threadIdx.x; i < N; i += stride) {
    x[i] = fma(a, p[i], x[i]);
    const X ri = fma(-a, q[i], r[i]);
    r[i] = ri;
    part = fma((double)ri, (double)ri, part);
  }
  block_partial(dot, part, scratch);
  finish_dot(dot, gridDim.x, scratch);
}

template <class X>
__global__ void cg_direction_kernel(int64_t N, X* __restrict__ p, const X* __restrict__ r,
                                    const CgState* __restrict__ st) {
  using VT = typename V16<X>::T;
  constexpr int R = V16<X>::R;
  if (st->done) return;
  const X b = (X)st->beta;
  const bool vec = (((uintptr_t)p | (uintptr_t)r) & 15u) == 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (vec) {
    const int64_t nv = N / R;
    for (int64_t k = t; k < nv; k += stride) {
      X pv[R], rv[R];
      V16<X>::get(*reinterpret_cast<const VT*>(p + k * R), pv);
      V16<X>::get(*reinterpret_cast<const VT*>(r + k * R), rv);
#pragma unroll
      for (int j = 0; j < R; ++j) pv[j] = fma(b, pv[j], rv[j]);
      *reinterpret_cast<VT*>(p + k * R) = V16<X>::put(pv);
    }
    for (int64_t i = nv * R + t; i < N; i += stride) p[i] = fma(b, p[i], r[i]);
  } else {
    for (int64_t i = t; i < N; i += stride) p[i] = fma(b, p[i], r[i]);
  }
}

// r = b - q in FP64 (q = A x); optionally r32 = (float) r, d32 = 0,
// p32 = r32. Dot: r.r (FP64) or, with r32, the inner rho_0 = r32.r32.
template <bool INNER>
__global__ void __launch_bounds__(NT)
residual_kernel(int64_t N, const double* __restrict__ b, const double* __restrict__ q,
                double* __restrict__ r, double* __restrict__ p, float* __restrict__ r32,
                float* __restrict__ d32, float* __restrict__ p32, int64_t tile_rows,
                int64_t ntiles, DotSpec dot) {
  __shared__ double scratch[NT];
  double part = 0.0;  // this block's share of the dot, over all its tiles
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t t1 = min(N, (tile + 1) * tile_rows);
    for (int64_t i = tile * tile_rows + threadIdx.x; i < t1; i += NT) {
      const double ri = b[i] - q[i];
      if constexpr (INNER) {
        const float rf = (float)ri;
        r32[i] = rf;
        p32[i] = rf;
        d32[i] = 0.0f;
        part += (double)rf * (double)rf;
      } else {
        if (r) r[i] = ri;
        if (p) p[i] = ri;
        part += ri * ri;
      }
    }
  }
  block_partial(dot, part, scratch);
  finish_dot(dot, gridDim.x, scratch);
}

// Reliable updates, start (x = 0): r32 = p32 = (float) b, d32 = 0; b.b (FP64).
__global__ void __launch_bounds__(NT)
ru_init_kernel(int64_t N, const double* __restrict__ b, float* __restrict__ r32,
               float* __restrict__ p32, float* __restrict__ d32, int64_t tile_rows,
               int64_t ntiles, DotSpec dot) {
  __shared__ double scratch[NT];
  double part = 0.0;  // this block's share of the dot, over all its tiles
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t t1 = min(N, (tile + 1) * tile_rows);
    for (int64_t i = tile * tile_rows + threadIdx.x; i < t1; i += NT) {
      const double bi = b[i];
      const float bf = (float)bi;
      r32[i] = bf;
      p32[i] = bf;
      d32[i] = 0.0f;
      part = fma(bi, bi, part);
    }
  }
  block_partial(dot, part, scratch);
  finish_dot(dot, gridDim.x, scratch);
}

// Fold (only while one is due): x += (double) d32; d32 = 0.
__global__ void ru_fold_kernel(int64_t N, double* __restrict__ x, float* __restrict__ d32,
                               const int32_t* __restrict__ skip) {
  if (*skip) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    x[i] = x[i] + (double)d32[i];
    d32[i] = 0.0f;
  }
}

// After a fold: r = b - q with q = A x (FP64), r32 = (float) r, r.r (FP64).
__global__ void __launch_bounds__(NT)
ru_residual_kernel(int64_t N, const double* __restrict__ b, const double* __restrict__ q,
                   float* __restrict__ r32, int64_t tile_rows, int64_t ntiles, DotSpec dot) {
  __shared__ double scratch[NT];
  if (skipped(dot)) return;
  double part = 0.0;  // this block's share of the dot, over all its tiles
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t t1 = min(N, (tile + 1) * tile_rows);
    for (int64_t i = tile * tile_rows + threadIdx.x; i < t1; i += NT) {
      const double ri = b[i] - q[i];
      r32[i] = (float)ri;
      part = fma(ri, ri, part);
    }
  }
  block_partial(dot, part, scratch);
  finish_dot(dot, gridDim.x, scratch);
}

// r = b - A x from r32 already formed: inner start from the FP64 residual.
__global__ void add_correction_kernel(int64_t N, double* __restrict__ x,
                                      const float* __restrict__ d) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = x[i] + (double)d[i];
}

const int32_t* done_ptr(const CgState* st) {
  return (const int32_t*)((const char*)st + offsetof(CgState, done));
}

const int32_t* skip_fold_ptr(const CgState* st) {
  return (const int32_t*)((const char*)st + offsetof(CgState, skip_fold));
}

unsigned vec_grid(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(n, NT), (int64_t)device().sms * 8));
}

// Resident blocks of the update kernel on the whole GPU, capped by the work
// (16-byte groups); at most 8 x SMs, within the partials' capacity.
template <class X>
unsigned update_grid(int64_t n) {
  static int per_sm = 0;
  if (!per_sm) {
    DM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cg_update_kernel<X>, NT, 0));
    per_sm = std::max(1, std::min(per_sm, 8));
  }
  const int64_t groups = cdiv(std::max<int64_t>(n, 1), V16<X>::R);
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(groups, NT),
                                                          (int64_t)device().sms * per_sm));
}

unsigned tile_grid(int64_t ntiles) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)device().sms * 8));
}

// Work space carved from one allocation owned by the handle.
struct Work {
  double *r, *p, *q, *part;
  float *r32, *d32, *p32, *q32;
  CgState *st, *aux;
};

Work carve(dynmat_s* A, bool mixed, cudaStream_t s) {
  const int64_t N = A->nrows, nt = A->plan.ntiles;
  auto al = [](int64_t b) { return round_up(std::max<int64_t>(b, 16), 256); };
  // partials: one per tile or per block of any reducing kernel (<= 8 x SMs)
  const int64_t npart = std::max<int64_t>(nt, 8 * (int64_t)device().sms);
  const int64_t need = 3 * al(N * 8) + al(npart * 8) + (mixed ? 4 * al(N * 4) : 0) +
                       2 * al(sizeof(CgState));
  if ((int64_t)A->cg_work_bytes < need) {
    A->cg_work.alloc(need, s);
    A->cg_work_bytes = need;
  }
  char* b = (char*)A->cg_work.p;
  Work w{};
  w.r = (double*)b; b += al(N * 8);
  w.p = (double*)b; b += al(N * 8);
  w.q = (double*)b; b += al(N * 8);
  w.part = (double*)b; b += al(npart * 8);
  w.st = (CgState*)b; b += al(sizeof(CgState));
  w.aux = (CgState*)b; b += al(sizeof(CgState));
  if (mixed) {
    w.r32 = (float*)b; b += al(N * 4);
    w.d32 = (float*)b; b += al(N * 4);
    w.p32 = (float*)b; b += al(N * 4);
    w.q32 = (float*)b; b += al(N * 4);
  }
  return w;
}

struct Pinned {
  CgState* h = nullptr;
  Pinned() {
    if (cudaMallocHost((void**)&h, sizeof(CgState) * 2) != cudaSuccess) h = nullptr;
  }
};

CgState* pinned_state() {
  static thread_local Pinned p;
  DM_REQUIRE(p.h, DYNMAT_ERR_OOM, "pinned host allocation failed");
  return p.h;
}

void reset_state(CgState* st, double tol, int max_iters, cudaStream_t s) {
  CgState h{};
  h.tol = tol;
  h.max_iters = max_iters;
  DM_CUDA(cudaMemcpyAsync(st, &h, sizeof h, cudaMemcpyHostToDevice, s));
}

CgState read_state(const CgState* st, cudaStream_t s) {
  CgState* h = pinned_state();
  DM_CUDA(cudaMemcpyAsync(h, st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
  DM_CUDA(cudaStreamSynchronize(s));
  return *h;
}

// Plain dot a.b (FP64 vectors) with the plan's tiles, blocking.
double dot_f64(const dynmat_s* A, const double* a, const double* b, const Work& w,
               cudaStream_t s) {
  reset_state(w.aux, 0, 0, s);
  DotSpec d{w.part, w.aux, DOT_STORE, nullptr};
  dot_tiles(A, a, b, DYNMAT_F64, d, s);
  return read_state(w.aux, s).dot;
}

// ||b - A x||^2 (FP64, A's values), r = b - A x kept in w.r. Blocking.
double residual_sq(const dynmat_s* A, const double* b, const double* x, const Work& w,
                   cudaStream_t s) {
  spmv(A, x, w.q, DYNMAT_F64, s);
  reset_state(w.aux, 0, 0, s);
  DotSpec d{w.part, w.aux, DOT_STORE, nullptr};
  residual_kernel<false><<<tile_grid(A->plan.ntiles), NT, 0, s>>>(
      A->nrows, b, w.q, w.r, nullptr, nullptr, nullptr, nullptr, A->plan.tile_rows,
      A->plan.ntiles, d);
  DM_CHECK_LAUNCH();
  return read_state(w.aux, s).dot;
}

// Enqueues one CG iteration on vectors of type X (x, r, p, q) for matrix M.
template <class X>
void enqueue_iteration(const dynmat_s* M, X* x, X* r, X* p, X* q, const Work& w,
                       dynmat_dtype vdt_vec, cudaStream_t s) {
  DotSpec pq{w.part, w.st, DOT_CG_PQ, done_ptr(w.st)};
  spmv_dot(M, p, q, vdt_vec, &pq, s);
  DotSpec rr{w.part, w.st, DOT_CG_RR, done_ptr(w.st)};
  cg_update_kernel<X><<<update_grid<X>(M->nrows), NT, 0, s>>>(M->nrows, x, r, p, q, rr);
  DM_CHECK_LAUNCH();
  cg_direction_kernel<X><<<vec_grid(M->nrows), NT, 0, s>>>(M->nrows, p, r, w.st);
  DM_CHECK_LAUNCH();
}

// Runs iterations (each enqueued by `one`) until the device state `st` says
// done: the first iteration eagerly (it also sizes the grids), then graphs of
// `every` iterations; the host reads the state between graph launches.
template <class F>
CgState run_iterations(F one, const CgState* st, int every, cudaStream_t s) {
  CgState h = read_state(st, s);
  if (h.done) return h;
  one();
  h = read_state(st, s);
  if (h.done) return h;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  DM_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  try {
    for (int k = 0; k < every; ++k) one();
  } catch (...) {
    cudaStreamEndCapture(s, &g);
    if (g) cudaGraphDestroy(g);
    throw;
  }
  DM_CUDA(cudaStreamEndCapture(s, &g));
  cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphDestroy(g);
  DM_CUDA(e);
  try {
    for (;;) {
      DM_CUDA(cudaGraphLaunch(ge, s));
      h = read_state(st, s);
      if (h.done) break;
    }
  } catch (...) {
    cudaGraphExecDestroy(ge);
    throw;
  }
  cudaGraphExecDestroy(ge);
  return h;
}

template <class X>
CgState run_loop(const dynmat_s* M, X* x, X* r, X* p, X* q, const Work& w, dynmat_dtype vdt_vec,
                 int every, cudaStream_t s) {
  return run_iterations([&] { enqueue_iteration<X>(M, x, r, p, q, w, vdt_vec, s); }, w.st, every,
                        s);
}

dynmat_s* fp32_copy(dynmat_s* A, cudaStream_t s) {
  if (A->vdt == DYNMAT_F32) return A;
  if (A->shadow32) return A->shadow32;
  Coo tmp;
  const Coo* c = &A->coo;
  if (A->fmt != DYNMAT_COO) {
    to_coo(A, tmp, s);
    c = &tmp;
  }
  auto S = std::make_unique<dynmat_s>();
  S->nrows = A->nrows;
  S->ncols = A->ncols;
  S->vdt = A->vdt;
  build_from_coo(S.get(), *c, A->fmt, DYNMAT_F32, s);
  S->values_exact_f32 = 1;
  S->plan.forced = A->plan.forced;
  prepare_spmv(S.get(), s);
  A->shadow32 = S.release();
  return A->shadow32;
}

void solve(dynmat_s* A, const double* b, double* x, const cg_opts& o, cg_result* res,
           cudaStream_t s) {
  const int64_t N = A->nrows;
  const int every = o.check_every > 0 ? o.check_every : 25;
  memset(res, 0, sizeof *res);
  if (o.precision == CG_FP64) {
    Work w = carve(A, false, s);
    const Plan& P = A->plan;
    // r = b - A x0, p = r, rho = r.r
    spmv(A, x, w.q, DYNMAT_F64, s);
    reset_state(w.st, o.tol, o.max_iters, s);
    DotSpec init{w.part, w.st, DOT_CG_INIT, nullptr};
    residual_kernel<false><<<tile_grid(P.ntiles), NT, 0, s>>>(
        N, b, w.q, w.r, w.p, nullptr, nullptr, nullptr, P.tile_rows, P.ntiles, init);
    DM_CHECK_LAUNCH();
    CgState h = run_loop<double>(A, x, w.r, w.p, w.q, w, DYNMAT_F64, every, s);
    res->status = h.status;
    res->iterations = h.iter;
    res->rel_residual = h.rel;
    const double rr = residual_sq(A, b, x, w, s);
    const double bb = dot_f64(A, b, b, w, s);
    res->true_rel_residual = bb > 0 ? std::sqrt(rr) / std::sqrt(bb) : std::sqrt(rr);
    return;
  }
  if (o.precision == CG_MIXED_RELIABLE) {
    // One FP32 CG whose correction is folded into the FP64 x, with an FP64
    // residual, whenever the recursive residual has dropped by delta (or
    // looks converged); the search direction is kept across folds.
    dynmat_s* A32 = fp32_copy(A, s);
    Work w = carve(A, true, s);  // A's tile count >= A32's: its partials serve both
    const Plan& P = A->plan;
    const Plan& P32 = A32->plan;
    DM_CUDA(cudaMemsetAsync(x, 0, N * 8, s));
    CgState h0{};
    h0.tol = o.tol;
    h0.max_iters = o.max_iters;
    h0.delta = o.delta > 0 ? o.delta : 0.1;
    h0.skip_fold = 1;
    DM_CUDA(cudaMemcpyAsync(w.st, &h0, sizeof h0, cudaMemcpyHostToDevice, s));
    DotSpec init{w.part, w.st, DOT_RU_INIT, nullptr};
    ru_init_kernel<<<tile_grid(P32.ntiles), NT, 0, s>>>(N, b, w.r32, w.p32, w.d32, P32.tile_rows,
                                                        P32.ntiles, init);
    DM_CHECK_LAUNCH();
    const int32_t* skipf = skip_fold_ptr(w.st);
    auto one = [&] {
      DotSpec pq{w.part, w.st, DOT_CG_PQ, done_ptr(w.st)};
      spmv_dot(A32, w.p32, w.q32, DYNMAT_F32, &pq, s);
      DotSpec rr{w.part, w.st, DOT_RU_RR, done_ptr(w.st)};
      cg_update_kernel<float><<<update_grid<float>(N), NT, 0, s>>>(N, w.d32, w.r32, w.p32,
                                                                  w.q32, rr);
      DM_CHECK_LAUNCH();
      ru_fold_kernel<<<vec_grid(N), NT, 0, s>>>(N, x, w.d32, skipf);
      DM_CHECK_LAUNCH();
      spmv_skip(A, x, w.q, DYNMAT_F64, nullptr, skipf, s);
      DotSpec fold{w.part, w.st, DOT_RU_FOLD, skipf};
      ru_residual_kernel<<<tile_grid(P.ntiles), NT, 0, s>>>(N, b, w.q, w.r32, P.tile_rows,
                                                            P.ntiles, fold);
      DM_CHECK_LAUNCH();
      cg_direction_kernel<float><<<vec_grid(N), NT, 0, s>>>(N, w.p32, w.r32, w.st);
      DM_CHECK_LAUNCH();
    };
    CgState h = run_iterations(one, w.st, every, s);
    res->status = h.status;
    res->iterations = h.iter;
    res->outer_iterations = h.folds;
    res->rel_residual = h.rel;
    const double rr = residual_sq(A, b, x, w, s);
    const double bb = dot_f64(A, b, b, w, s);
    res->true_rel_residual = bb > 0 ? std::sqrt(rr) / std::sqrt(bb) : std::sqrt(rr);
    return;
  }
  // Mixed precision: FP64 outer refinement, FP32 inner CG.
  dynmat_s* A32 = fp32_copy(A, s);
  Work w = carve(A, true, s);
  Work w32 = w;  // the inner solve uses A32's tile plan on the same buffers
  if (A32 != A) {
    Work t = carve(A32, false, s);
    w32.part = t.part;
    w32.st = t.st;
    w32.aux = t.aux;
  }
  DM_CUDA(cudaMemsetAsync(x, 0, N * 8, s));
  const double bb = dot_f64(A, b, b, w, s);
  const double bn = std::sqrt(bb);
  int outer = 0, inner_total = 0;
  double rel = 0;
  int status = DYNMAT_ERR_NOT_CONVERGED;
  for (;;) {
    const double rr = residual_sq(A, b, x, w, s);  // w.r = b - A x (FP64)
    rel = bn > 0 ? std::sqrt(rr) / bn : std::sqrt(rr);
    if (rel <= o.tol) {
      status = DYNMAT_OK;
      break;
    }
    if (outer >= o.max_outer) break;
    ++outer;
    // inner start: r32 = (float) r, d = 0, p32 = r32, rho_0 = r32.r32
    const Plan& P32 = A32->plan;
    reset_state(w32.st, o.inner_tol, o.max_iters, s);
    DotSpec init{w32.part, w32.st, DOT_CG_INIT, nullptr};
    residual_kernel<true><<<tile_grid(P32.ntiles), NT, 0, s>>>(
        N, b, w.q, nullptr, nullptr, w.r32, w.d32, w.p32, P32.tile_rows, P32.ntiles, init);
    DM_CHECK_LAUNCH();
    CgState h = run_loop<float>(A32, w.d32, w.r32, w.p32, w.q32, w32, DYNMAT_F32, every, s);
    inner_total += h.iter;
    add_correction_kernel<<<vec_grid(N), NT, 0, s>>>(N, x, w.d32);
    DM_CHECK_LAUNCH();
  }
  res->status = status;
  res->iterations = inner_total;
  res->outer_iterations = outer;
  res->rel_residual = rel;
  res->true_rel_residual = rel;
}

}  // namespace

// Helpers of the batched solver (batch.cu): FP64 residual r = b - A x with
// ||r||^2, optionally forming the FP32 inner start (r32 = p32 = (float) r,
// d32 = 0) and returning r32.r32 instead; plain dot a.b; x += (double) d.
double batch_residual(const dynmat_s* A, const double* b, const double* x, double* r,
                      double* q, float* r32, float* d32, float* p32, double* part,
                      CgState* aux_state, bool inner_init, cudaStream_t s) {
  const Plan& P = A->plan;
  spmv(A, x, q, DYNMAT_F64, s);
  reset_state(aux_state, 0, 0, s);
  DotSpec d{part, aux_state, DOT_STORE, nullptr};
  if (inner_init)
    residual_kernel<true><<<tile_grid(P.ntiles), NT, 0, s>>>(
        A->nrows, b, q, nullptr, nullptr, r32, d32, p32, P.tile_rows, P.ntiles, d);
  else
    residual_kernel<false><<<tile_grid(P.ntiles), NT, 0, s>>>(
        A->nrows, b, q, r, nullptr, nullptr, nullptr, nullptr, P.tile_rows, P.ntiles, d);
  DM_CHECK_LAUNCH();
  return read_state(aux_state, s).dot;
}

double batch_dot(const dynmat_s* A, const double* a, const double* b, double* part,
                 CgState* aux_state, cudaStream_t s) {
  reset_state(aux_state, 0, 0, s);
  DotSpec d{part, aux_state, DOT_STORE, nullptr};
  dot_tiles(A, a, b, DYNMAT_F64, d, s);
  return read_state(aux_state, s).dot;
}

double batch_ru_init(const dynmat_s* A, const double* b, float* r32, float* p32, float* d32,
                     double* part, CgState* aux_state, cudaStream_t s) {
  const Plan& P = A->plan;
  reset_state(aux_state, 0, 0, s);
  DotSpec d{part, aux_state, DOT_STORE, nullptr};
  ru_init_kernel<<<tile_grid(P.ntiles), NT, 0, s>>>(A->nrows, b, r32, p32, d32, P.tile_rows,
                                                    P.ntiles, d);
  DM_CHECK_LAUNCH();
  return read_state(aux_state, s).dot;
}

void batch_add_correction(int64_t N, double* x, const float* d, cudaStream_t s) {
  add_correction_kernel<<<vec_grid(N), NT, 0, s>>>(N, x, d);
  DM_CHECK_LAUNCH();
}

// One non-blocking solver stream and one ordering event per thread and device.
cudaStream_t solver_stream() {
  static thread_local cudaStream_t st[64] = {};
  const int d = device().id;
  if (!st[d]) DM_CUDA(cudaStreamCreateWithFlags(&st[d], cudaStreamNonBlocking));
  return st[d];
}

cudaEvent_t solver_event() {
  static thread_local cudaEvent_t ev[64] = {};
  const int d = device().id;
  if (!ev[d]) DM_CUDA(cudaEventCreateWithFlags(&ev[d], cudaEventDisableTiming));
  return ev[d];
}

}  // namespace dm

using namespace dm;

namespace dm {
namespace {
// HPCG's PCG (§II-B) on the finest level of M with one V-cycle as the
// preconditioner: textbook preconditioned CG, each iteration
//   q = A p and p.q (alpha); x += alpha p, r -= alpha q and r.r (test);
//   z = M^{-1} r; r.z (beta); p = z + beta p,
// every kernel skipping once the device state says done; check_every
// iterations per CUDA graph as for CG.
void pcg(dynmat_mg_s* M, const double* b, double* x, const cg_opts& o, cg_result* res,
         cudaStream_t s) {
  dynmat_s* A = const_cast<dynmat_s*>(mg_matrix(M));
  const int64_t N = A->nrows;
  const int every = o.check_every > 0 ? o.check_every : 25;
  memset(res, 0, sizeof *res);
  Work w = carve(A, false, s);
  DBuf zb(N * 8, s);
  double* z = zb.as<double>();
  const Plan& P = A->plan;
  const int32_t* done = done_ptr(w.st);
  spmv(A, x, w.q, DYNMAT_F64, s);
  reset_state(w.st, o.tol, o.max_iters, s);
  DotSpec init{w.part, w.st, DOT_CG_INIT, nullptr};
  residual_kernel<false><<<tile_grid(P.ntiles), NT, 0, s>>>(
      N, b, w.q, w.r, nullptr, nullptr, nullptr, nullptr, P.tile_rows, P.ntiles, init);
  DM_CHECK_LAUNCH();
  mg_vcycle(M, w.r, z, done, s);
  DM_CUDA(cudaMemcpyAsync(w.p, z, N * 8, cudaMemcpyDeviceToDevice, s));
  dot_tiles(A, w.r, z, DYNMAT_F64, DotSpec{w.part, w.st, DOT_PCG_RZ0, done}, s);
  auto one = [&] {
    DotSpec pq{w.part, w.st, DOT_CG_PQ, done};
    spmv_dot(A, w.p, w.q, DYNMAT_F64, &pq, s);
    DotSpec rr{w.part, w.st, DOT_PCG_RR, done};
    cg_update_kernel<double><<<update_grid<double>(N), NT, 0, s>>>(N, x, w.r, w.p, w.q, rr);
    DM_CHECK_LAUNCH();
    mg_vcycle(M, w.r, z, done, s);
    dot_tiles(A, w.r, z, DYNMAT_F64, DotSpec{w.part, w.st, DOT_PCG_RZ, done}, s);
    cg_direction_kernel<double><<<vec_grid(N), NT, 0, s>>>(N, w.p, z, w.st);
    DM_CHECK_LAUNCH();
  };
  CgState h = run_iterations(one, w.st, every, s);
  res->status = h.status;
  res->iterations = h.iter;
  res->rel_residual = h.rel;
  const double rr2 = residual_sq(A, b, x, w, s);
  const double bb = dot_f64(A, b, b, w, s);
  res->true_rel_residual = bb > 0 ? std::sqrt(rr2) / std::sqrt(bb) : std::sqrt(rr2);
}
}  // namespace
}  // namespace dm

extern "C" dynmat_status pcg_solve(dynmat_mg_t M, const double* b, double* x, const cg_opts* opts,
                                   cg_result* res, dynmat_stream_t stream) {
  return dm::guard([&] {
    DM_REQUIRE(M && b && x && opts && res, DYNMAT_ERR_INVALID_ARG, "null argument");
    DM_REQUIRE(opts->precision == CG_FP64, DYNMAT_ERR_INVALID_ARG, "PCG runs in FP64");
    DM_REQUIRE(opts->max_iters >= 0 && opts->tol >= 0, DYNMAT_ERR_INVALID_ARG,
               "bad tolerance or iteration limit");
    cudaStream_t user = (cudaStream_t)stream;
    cudaStream_t s = solver_stream();
    cudaEvent_t ev = solver_event();
    DM_CUDA(cudaEventRecord(ev, user));
    DM_CUDA(cudaStreamWaitEvent(s, ev, 0));
    try {
      pcg(M, b, x, *opts, res, s);
      check_wait_timeout(s);
      mg_check_timeout(M, s);
    } catch (...) {
      cudaEventRecord(ev, s);
      cudaStreamWaitEvent(user, ev, 0);
      throw;
    }
    DM_CUDA(cudaEventRecord(ev, s));
    DM_CUDA(cudaStreamWaitEvent(user, ev, 0));
  });
}

extern "C" dynmat_status cg_solve(dynmat_t A, const double* b, double* x, const cg_opts* opts,
                                  cg_result* res, dynmat_stream_t stream) {
  return dm::guard([&] {
    DM_REQUIRE(A && b && x && opts && res, DYNMAT_ERR_INVALID_ARG, "null argument");
    DM_REQUIRE(A->nrows == A->ncols, DYNMAT_ERR_INVALID_ARG, "CG needs a square matrix");
    DM_REQUIRE(opts->precision == CG_FP64 || opts->precision == CG_MIXED ||
                   opts->precision == CG_MIXED_RELIABLE,
               DYNMAT_ERR_INVALID_ARG, "bad precision");
    DM_REQUIRE(opts->max_iters >= 0 && opts->tol >= 0, DYNMAT_ERR_INVALID_ARG,
               "bad tolerance or iteration limit");
    DM_REQUIRE(opts->precision != CG_MIXED || (opts->max_outer >= 0 && opts->inner_tol > 0),
               DYNMAT_ERR_INVALID_ARG, "bad refinement options");
    DM_REQUIRE(opts->precision != CG_MIXED_RELIABLE || (opts->delta >= 0 && opts->delta < 1),
               DYNMAT_ERR_INVALID_ARG, "fold ratio delta must lie in [0, 1)");
    if (A->nrows == 0) {
      memset(res, 0, sizeof *res);
      return;
    }
    // The solve runs on a library-owned non-blocking stream (graph capture is
    // not allowed on the legacy default stream), ordered after the caller's
    // stream on entry and before it on return.
    cudaStream_t user = (cudaStream_t)stream;
    cudaStream_t s = solver_stream();
    cudaEvent_t ev = solver_event();
    DM_CUDA(cudaEventRecord(ev, user));
    DM_CUDA(cudaStreamWaitEvent(s, ev, 0));
    try {
      solve(A, b, x, *opts, res, s);
      check_wait_timeout(s);
    } catch (...) {
      cudaEventRecord(ev, s);
      cudaStreamWaitEvent(user, ev, 0);
      throw;
    }
    DM_CUDA(cudaEventRecord(ev, s));
    DM_CUDA(cudaStreamWaitEvent(user, ev, 0));
  });
}
