// HPCG problem generation on the device (§II-B: Poisson on a regular 3-D
// grid, 27-point stencil; the 7-point variant for the served mix). Builds the
// canonical COO directly in device memory — row i = ix + nx*(iy + ny*iz),
// neighbours in ascending column order, diagonal points-1, off-diagonal -1 —
// then converts it to the requested format, so a large problem never passes
// through host memory.
#include <algorithm>
#include <memory>

#include "internal.cuh"

namespace dm {
namespace {

constexpr int T = 256;

__device__ __forceinline__ bool in_box(int dz, int dy, int dx, int points) {
  if (points == 27) return true;
  return (dz != 0) + (dy != 0) + (dx != 0) <= 1;
}

__global__ void stencil_count_kernel(int64_t nx, int64_t ny, int64_t nz, int points,
                                     int32_t* __restrict__ cnt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t N = nx * ny * nz;
  if (i >= N) return;
  const int64_t ix = i % nx, iy = (i / nx) % ny, iz = i / (nx * ny);
  int c = 0;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        if (!in_box(dz, dy, dx, points)) continue;
        const int64_t jx = ix + dx, jy = iy + dy, jz = iz + dz;
        if (jx >= 0 && jx < nx && jy >= 0 && jy < ny && jz >= 0 && jz < nz) ++c;
      }
  cnt[i] = c;
}

template <class W>
__global__ void stencil_fill_kernel(int64_t nx, int64_t ny, int64_t nz, int points,
                                    const int32_t* __restrict__ start, int32_t* __restrict__ row,
                                    int32_t* __restrict__ col, W* __restrict__ val) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t N = nx * ny * nz;
  if (i >= N) return;
  const int64_t ix = i % nx, iy = (i / nx) % ny, iz = i / (nx * ny);
  int64_t m = start[i];
  // (dz, dy, dx) in lexicographic order = ascending column offsets
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        if (!in_box(dz, dy, dx, points)) continue;
        const int64_t jx = ix + dx, jy = iy + dy, jz = iz + dz;
        if (!(jx >= 0 && jx < nx && jy >= 0 && jy < ny && jz >= 0 && jz < nz)) continue;
        row[m] = (int32_t)i;
        col[m] = (int32_t)(i + dz * nx * ny + dy * nx + dx);
        val[m] = (dz == 0 && dy == 0 && dx == 0) ? W(points - 1) : W(-1);
        ++m;
      }
}

}  // namespace
}  // namespace dm

using namespace dm;

extern "C" dynmat_status dynmat_create_stencil(dynmat_t* out, int64_t nx, int64_t ny, int64_t nz,
                                               int32_t points, dynmat_format fmt,
                                               dynmat_dtype vdtype, dynmat_stream_t stream) {
  return dm::guard([&] {
    DM_REQUIRE(out, DYNMAT_ERR_INVALID_ARG, "out is NULL");
    DM_REQUIRE(nx > 0 && ny > 0 && nz > 0, DYNMAT_ERR_INVALID_ARG, "grid sizes must be positive");
    DM_REQUIRE(points == 7 || points == 27, DYNMAT_ERR_INVALID_ARG, "points must be 7 or 27");
    DM_REQUIRE(vdtype == DYNMAT_F64 || vdtype == DYNMAT_F32, DYNMAT_ERR_INVALID_ARG,
               "bad value dtype");
    DM_REQUIRE(fmt >= DYNMAT_COO && fmt <= DYNMAT_HYB, DYNMAT_ERR_INVALID_ARG, "bad format");
    const int64_t N = nx * ny * nz;
    DM_REQUIRE(N < INT32_MAX && N * points < INT32_MAX, DYNMAT_ERR_INVALID_ARG,
               "grid too large for int32 indices");
    cudaStream_t s = (cudaStream_t)stream;
    device();
    DBuf cnt(N * 4, s), start(N * 4, s);
    stencil_count_kernel<<<(unsigned)cdiv(N, T), T, 0, s>>>(nx, ny, nz, points,
                                                            cnt.as<int32_t>());
    DM_CHECK_LAUNCH();
    int64_t nnz = 0;
    exclusive_scan_i32(cnt.as<int32_t>(), start.as<int32_t>(), N, &nnz, s);
    auto A = std::make_unique<dynmat_s>();
    A->nrows = A->ncols = N;
    A->vdt = vdtype;
    A->fmt = DYNMAT_COO;
    A->coo.nnz = nnz;
    A->coo.row.alloc(nnz * 4, s);
    A->coo.col.alloc(nnz * 4, s);
    A->coo.val.alloc(nnz * vsize(vdtype), s);
    if (vdtype == DYNMAT_F64)
      stencil_fill_kernel<double><<<(unsigned)cdiv(N, T), T, 0, s>>>(
          nx, ny, nz, points, start.as<int32_t>(), A->coo.row.as<int32_t>(),
          A->coo.col.as<int32_t>(), A->coo.val.as<double>());
    else
      stencil_fill_kernel<float><<<(unsigned)cdiv(N, T), T, 0, s>>>(
          nx, ny, nz, points, start.as<int32_t>(), A->coo.row.as<int32_t>(),
          A->coo.col.as<int32_t>(), A->coo.val.as<float>());
    DM_CHECK_LAUNCH();
    A->nnz = nnz;
    A->values_exact_f32 = 1;
    prepare_spmv(A.get(), s);
    if (fmt != DYNMAT_COO) convert_impl(A.get(), fmt, vdtype, s);
    DM_CUDA(cudaStreamSynchronize(s));
    *out = A.release();
  });
}
