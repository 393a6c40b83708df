// Diagonal extraction and update for every format (§III-D: the containers
// support diagonal update and extraction; §IV-B: HPCG's CG test modifies the
// matrix diagonal, so the dynamic matrix must update the active format's
// diagonal in place). One traversal per format visits each stored (i, i)
// entry with an operation: read it, overwrite it, or count it.
//  - COO (and HYB's COO part): entries with row == col.
//  - CSR: a binary search of column i in row i (columns ascend).
//  - DIA: the offset-0 diagonal; every one of its slots counts as stored.
//  - ELL (and HYB's ELL part): the slots of row i in column order.
#include <algorithm>
#include <vector>

#include "device.cuh"
#include "internal.cuh"

namespace dm {
namespace {

constexpr int T = 256;

// An operation on each stored diagonal entry; done() runs once per thread
// at the end of a kernel, with the whole warp converged.
template <class V>
struct ReadOp {
  V* d;
  __device__ void operator()(int64_t i, V* slot) { d[i] = *slot; }
  __device__ void done() {}
};
template <class V>
struct WriteOp {
  const V* d;
  __device__ void operator()(int64_t i, V* slot) { *slot = d[i]; }
  __device__ void done() {}
};
// Counts in a register; one atomic per warp at the end.
template <class V>
struct CountOp {
  unsigned long long* c;
  unsigned n;
  __device__ void operator()(int64_t, V*) { ++n; }
  __device__ void done() {
    unsigned t = n;
    for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0 && t) atomicAdd(c, (unsigned long long)t);
  }
};

unsigned grid_of(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(n, T), (int64_t)device().sms * 8));
}

template <class V, class Op>
__global__ void coo_diag_kernel(const int32_t* __restrict__ row, const int32_t* __restrict__ col,
                                V* __restrict__ val, int64_t nnz, Op op) {
  for (int64_t e = (int64_t)blockIdx.x * T + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * T)
    if (row[e] == col[e]) op(row[e], val + e);
  op.done();
}

// CSR: a binary search of column i in row i (columns ascend). (Four rows
// per thread searched in lockstep, or eight lanes per row loading 32 columns
// at a time, both measured slower at 128^3.)
template <class V, class Op>
__global__ void csr_diag_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                V* __restrict__ val, int64_t n, Op op) {
  for (int64_t i = (int64_t)blockIdx.x * T + threadIdx.x; i < n; i += (int64_t)gridDim.x * T) {
    int32_t lo = rowptr[i], hi = rowptr[i + 1];
    while (lo < hi) {
      const int32_t mid = lo + ((hi - lo) >> 1);
      if (col[mid] < i) lo = mid + 1; else hi = mid;
    }
    if (lo < rowptr[i + 1] && col[lo] == i) op(i, val + lo);
  }
  op.done();
}

template <class V, class Op>
__global__ void dia_diag_kernel(V* __restrict__ dval, int64_t d0, int64_t ld, int64_t n, Op op) {
  for (int64_t i = (int64_t)blockIdx.x * T + threadIdx.x; i < n; i += (int64_t)gridDim.x * T)
    op(i, dval + d0 * ld + i);
  op.done();
}

// Slots of row i hold its entries in column order, then padding (col -1);
// four slots' columns are loaded at a time.
template <class V, class Op>
__global__ void ell_diag_kernel(const int32_t* __restrict__ ecol, V* __restrict__ eval, int64_t ld,
                                int64_t K, int64_t n, Op op) {
  constexpr int PER = 4;
  for (int64_t i = (int64_t)blockIdx.x * T + threadIdx.x; i < n; i += (int64_t)gridDim.x * T) {
    for (int64_t k0 = 0; k0 < K; k0 += PER) {
      int32_t c[PER];
#pragma unroll
      for (int j = 0; j < PER; ++j) c[j] = k0 + j < K ? __ldg(ecol + (k0 + j) * ld + i) : -1;
      bool stop = false;
#pragma unroll
      for (int j = 0; j < PER; ++j) {
        if (stop) continue;
        if (c[j] < 0 || c[j] > i) {
          stop = true;
        } else if (c[j] == i) {
          op(i, eval + (k0 + j) * ld + i);
          stop = true;
        }
      }
      if (stop) break;
    }
  }
  op.done();
}

// Index of the offset-0 diagonal of a DIA matrix, or -1 (a host copy kept
// with the format).
int64_t dia_main(const dynmat_s* A) {
  return A->dia.ndiag > 0 ? A->dia.main_diag : -1;
}

template <class V, class Op>
void visit(dynmat_s* A, Op op, cudaStream_t s) {
  const int64_t n = std::min(A->nrows, A->ncols);
  if (n == 0) return;
  auto coo = [&](Coo& c) {
    if (c.nnz == 0) return;
    coo_diag_kernel<V, Op><<<grid_of(c.nnz), T, 0, s>>>(c.row.as<int32_t>(), c.col.as<int32_t>(),
                                                       c.val.as<V>(), c.nnz, op);
    DM_CHECK_LAUNCH();
  };
  auto ell = [&]() {
    if (A->ell.K == 0) return;
    ell_diag_kernel<V, Op><<<grid_of(n), T, 0, s>>>(A->ell.col.as<int32_t>(), A->ell.val.as<V>(),
                                                   A->ell.ld, A->ell.K, n, op);
    DM_CHECK_LAUNCH();
  };
  switch (A->fmt) {
    case DYNMAT_COO: coo(A->coo); break;
    case DYNMAT_CSR:
      csr_diag_kernel<V, Op><<<grid_of(n), T, 0, s>>>(A->csr.rowptr.as<int32_t>(),
                                                     A->csr.col.as<int32_t>(), A->csr.val.as<V>(),
                                                     n, op);
      DM_CHECK_LAUNCH();
      break;
    case DYNMAT_DIA: {
      const int64_t d0 = dia_main(A);
      if (d0 >= 0) {
        dia_diag_kernel<V, Op><<<grid_of(n), T, 0, s>>>(A->dia.val.as<V>(), d0, A->dia.ld, n, op);
        DM_CHECK_LAUNCH();
      }
      break;
    }
    case DYNMAT_ELL: ell(); break;
    case DYNMAT_HYB:
      ell();
      coo(A->coo);
      break;
  }
}

// Stored diagonal entries (i < min(nrows, ncols)); blocking.
int64_t count_diag(dynmat_s* A, cudaStream_t s) {
  DBuf c(8, s);
  DM_CUDA(cudaMemsetAsync(c.p, 0, 8, s));
  if (A->vdt == DYNMAT_F64)
    visit<double>(A, CountOp<double>{c.as<unsigned long long>(), 0u}, s);
  else
    visit<float>(A, CountOp<float>{c.as<unsigned long long>(), 0u}, s);
  unsigned long long h = 0;
  DM_CUDA(cudaMemcpyAsync(&h, c.p, 8, cudaMemcpyDeviceToHost, s));
  DM_CUDA(cudaStreamSynchronize(s));
  return (int64_t)h;
}

}  // namespace
}  // namespace dm

using namespace dm;

extern "C" {

dynmat_status dynmat_diagonal(dynmat_t A, void* diag, dynmat_stream_t stream) {
  return guard([&] {
    DM_REQUIRE(A, DYNMAT_ERR_INVALID_ARG, "null handle");
    const int64_t n = std::min(A->nrows, A->ncols);
    DM_REQUIRE(n == 0 || diag, DYNMAT_ERR_INVALID_ARG, "null diagonal");
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) return;
    // absent entries read as 0 (a DIA main diagonal stores every slot)
    if (!(A->fmt == DYNMAT_DIA && dia_main(A) >= 0))
      DM_CUDA(cudaMemsetAsync(diag, 0, (size_t)n * vsize(A->vdt), s));
    if (A->vdt == DYNMAT_F64)
      visit<double>(A, ReadOp<double>{(double*)diag}, s);
    else
      visit<float>(A, ReadOp<float>{(float*)diag}, s);
    DM_CUDA(cudaStreamSynchronize(s));
  });
}

dynmat_status dynmat_set_diagonal(dynmat_t A, const void* diag, dynmat_stream_t stream) {
  return guard([&] {
    DM_REQUIRE(A, DYNMAT_ERR_INVALID_ARG, "null handle");
    const int64_t n = std::min(A->nrows, A->ncols);
    DM_REQUIRE(n == 0 || diag, DYNMAT_ERR_INVALID_ARG, "null diagonal");
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) return;
    const int64_t stored = A->fmt == DYNMAT_DIA ? (dia_main(A) >= 0 ? n : 0) : count_diag(A, s);
    DM_REQUIRE(stored == n, DYNMAT_ERR_INVALID_ARG,
               "%lld of the %lld diagonal entries are stored; the update needs all of them",
               (long long)stored, (long long)n);
    if (A->vdt == DYNMAT_F64)
      visit<double>(A, WriteOp<double>{(const double*)diag}, s);
    else
      visit<float>(A, WriteOp<float>{(const float*)diag}, s);
    // Values changed: the FP32 copy of the mixed solver is stale, and the
    // FP32-exactness flag can only stay set if the new diagonal is exact.
    if (A->shadow32) {
      destroy_handle(A->shadow32, s);
      A->shadow32 = nullptr;
    }
    if (A->vdt == DYNMAT_F64 && A->values_exact_f32)
      A->values_exact_f32 = values_exact_in_f32(diag, n, A->vdt, s);
    DM_CUDA(cudaStreamSynchronize(s));
  });
}

}  // extern "C"
