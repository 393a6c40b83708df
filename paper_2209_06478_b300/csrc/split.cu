// Local / remote split of a partitioned matrix (§IV-B, §V-E).
//
// With the rows of a problem spread over processes, each process's matrix
// has a square local part (columns it owns) and a rectangular remote part
// (columns owned elsewhere, renumbered 0..n_ext-1 in the order of its halo
// list). Storing the two as separate dynamic matrices lets each take its own
// format: the local part stays regular (DIA for a stencil) while the remote
// part is sparse and irregular (COO or CSR). A product is
//   x_ext = x_src[halo]            (the halo exchange; here a device gather)
//   y     = A_loc x_loc
//   y    += A_rem x_ext
// All three steps are kernels of this library, on the caller's stream.
#include "device.cuh"
#include "internal.cuh"

namespace dm {
namespace {

constexpr int T = 256;

template <class X>
__global__ void gather_kernel(const X* __restrict__ src, const int32_t* __restrict__ idx, int64_t n,
                              X* __restrict__ dst) {
  for (int64_t k = (int64_t)blockIdx.x * T + threadIdx.x; k < n; k += (int64_t)gridDim.x * T)
    dst[k] = src[idx[k]];
}

template <class X>
__global__ void add_kernel(X* __restrict__ y, const X* __restrict__ t, int64_t n) {
  for (int64_t k = (int64_t)blockIdx.x * T + threadIdx.x; k < n; k += (int64_t)gridDim.x * T)
    y[k] += t[k];
}

unsigned grid_of(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(n, T), (int64_t)device().sms * 8));
}

void gather(const void* src, const int32_t* idx, int64_t n, void* dst, dynmat_dtype vdt,
            cudaStream_t s) {
  if (n <= 0) return;
  if (vdt == DYNMAT_F64)
    gather_kernel<double><<<grid_of(n), T, 0, s>>>((const double*)src, idx, n, (double*)dst);
  else
    gather_kernel<float><<<grid_of(n), T, 0, s>>>((const float*)src, idx, n, (float*)dst);
  DM_CHECK_LAUNCH();
}

// y += A x: in one pass where the format's kernel accumulates (COO, CSR
// merge); otherwise the product goes to the handle's scratch vector and one
// add follows.
void spmv_acc(dynmat_s* A, const void* x, void* y, dynmat_dtype vdt, cudaStream_t s) {
  const int64_t n = A->nrows;
  if (n == 0) return;
  if (spmv_accumulate(A, x, y, vdt, s)) return;
  const size_t bytes = (size_t)n * vsize(vdt);
  if (A->acc_tmp.bytes < DBuf::padded(bytes)) A->acc_tmp.alloc(bytes, s);
  spmv(A, x, A->acc_tmp.p, vdt, s);
  if (vdt == DYNMAT_F64)
    add_kernel<double><<<grid_of(n), T, 0, s>>>((double*)y, A->acc_tmp.as<double>(), n);
  else
    add_kernel<float><<<grid_of(n), T, 0, s>>>((float*)y, A->acc_tmp.as<float>(), n);
  DM_CHECK_LAUNCH();
}

}  // namespace
}  // namespace dm

using namespace dm;

extern "C" {

dynmat_status dynmat_gather(const void* src, const int32_t* idx, int64_t n, void* dst,
                            dynmat_dtype vec_dtype, dynmat_stream_t stream) {
  return guard([&] {
    DM_REQUIRE(n >= 0, DYNMAT_ERR_INVALID_ARG, "negative length");
    DM_REQUIRE(n == 0 || (src && idx && dst), DYNMAT_ERR_INVALID_ARG, "null argument");
    DM_REQUIRE(vec_dtype == DYNMAT_F64 || vec_dtype == DYNMAT_F32, DYNMAT_ERR_INVALID_ARG,
               "bad vector dtype");
    gather(src, idx, n, dst, vec_dtype, (cudaStream_t)stream);
  });
}

dynmat_status dynmat_spmv_acc(dynmat_t A, const void* x, void* y, dynmat_dtype vec_dtype,
                              dynmat_stream_t stream) {
  return guard([&] {
    DM_REQUIRE(A && (A->nrows == 0 || (x && y)), DYNMAT_ERR_INVALID_ARG, "null argument");
    DM_REQUIRE(vec_dtype == DYNMAT_F64 || vec_dtype == DYNMAT_F32, DYNMAT_ERR_INVALID_ARG,
               "bad vector dtype");
    spmv_acc(A, x, y, vec_dtype, (cudaStream_t)stream);
  });
}

dynmat_status dynmat_split_spmv(dynmat_t A_loc, dynmat_t A_rem, const int32_t* halo, int64_t n_ext,
                                const void* x_src, const void* x_loc, void* x_ext, void* y,
                                dynmat_dtype vec_dtype, dynmat_stream_t stream) {
  return guard([&] {
    DM_REQUIRE(A_loc, DYNMAT_ERR_INVALID_ARG, "null local matrix");
    DM_REQUIRE(A_loc->nrows == A_loc->ncols, DYNMAT_ERR_INVALID_ARG,
               "local part must be square (%lld x %lld)", (long long)A_loc->nrows,
               (long long)A_loc->ncols);
    DM_REQUIRE(n_ext >= 0, DYNMAT_ERR_INVALID_ARG, "negative halo length");
    DM_REQUIRE(vec_dtype == DYNMAT_F64 || vec_dtype == DYNMAT_F32, DYNMAT_ERR_INVALID_ARG,
               "bad vector dtype");
    if (A_rem) {
      DM_REQUIRE(A_rem->nrows == A_loc->nrows && A_rem->ncols == n_ext, DYNMAT_ERR_INVALID_ARG,
                 "remote part must be %lld x %lld (is %lld x %lld)", (long long)A_loc->nrows,
                 (long long)n_ext, (long long)A_rem->nrows, (long long)A_rem->ncols);
      DM_REQUIRE(n_ext == 0 || (halo && x_src && x_ext), DYNMAT_ERR_INVALID_ARG,
                 "null halo argument");
    }
    DM_REQUIRE(A_loc->nrows == 0 || (x_loc && y), DYNMAT_ERR_INVALID_ARG, "null vector");
    cudaStream_t s = (cudaStream_t)stream;
    if (A_rem && n_ext > 0) gather(x_src, halo, n_ext, x_ext, vec_dtype, s);
    spmv(A_loc, x_loc, y, vec_dtype, s);
    if (A_rem && n_ext > 0 && A_rem->nnz > 0) spmv_acc(A_rem, x_ext, y, vec_dtype, s);
  });
}

}  // extern "C"
