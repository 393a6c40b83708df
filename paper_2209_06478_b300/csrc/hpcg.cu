// HPCG's multigrid preconditioner (§II-B: the benchmark's PCG uses a
// symmetric Gauss-Seidel smoother inside multigrid; the paper runs CG with the
// preconditioner disabled, §IV-B). Level l is the stencil on the grid halved
// l times; each level is a dynamic matrix in DIA (FP64).
//  - Smoother: one symmetric Gauss-Seidel sweep in colour order, colour(i) =
//    7 - ((ix & 1) + 2 (iy & 1) + 4 (iz & 1)); no two stencil neighbours
//    share a colour, so a colour's rows are updated in parallel, one launch
//    per colour: forward colours 0..7, backward 7..0. The coarse grid's
//    points (all coordinates even) are colour 7 so that the last colour of a
//    sweep, whose residual the sweep zeroes, is not the one injected.
//    z_i = (r_i - sum_{j != i} a_ij z_j) / a_ii with the diagonals in
//    ascending offset order (DIA slots outside the grid hold 0).
//  - V-cycle: z = 0; the coarsest level is one sweep; otherwise pre-smooth,
//    t = r - A z, coarse r = t at the coarse points (injection), the coarse
//    V-cycle, z += coarse z at the coarse points, post-smooth.
// Every kernel takes the solver's `done` flag and returns at once when it is
// set, so iterations replayed after convergence cost no work.
#include <array>
#include <memory>
#include <vector>

#include "device.cuh"
#include "internal.cuh"

struct dynmat_mg_s {
  int32_t levels = 0, points = 27;
  std::vector<std::array<int64_t, 3>> dims;
  std::vector<dynmat_s*> A;   // owned
  std::vector<int32_t> d0;    // index of the offset-0 diagonal per level
  std::vector<dm::DBuf> r, z, t;
  // Per level, the DIA values again (the main diagonal as its reciprocal),
  // colour by colour: colour c's block holds
  // ndiag x count_c values, value d of the colour's k-th point at d*count_c+k
  // (contiguous reads in a colour pass; the natural layout serves the SpMV).
  std::vector<dm::DBuf> valc;
  std::vector<std::array<int64_t, 8>> cstart;  // first value of each colour's block
  // Grid barrier of the fused smoother: arrivals, generation, timeout flag.
  dm::DBuf bar;
};

namespace dm {
namespace {

constexpr int T = 256;

unsigned grid_of(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(n, T), (int64_t)device().sms * 8));
}

// Points of a colour: coordinates with parities (px, py, pz), the colour's
// k-th point in x-fastest order of the half grid.
struct ColourGrid {
  int64_t nx, ny, nz, cx, cy, cz;
  int px, py, pz;
  __host__ __device__ ColourGrid(int64_t nx_, int64_t ny_, int64_t nz_, int parity)
      : nx(nx_), ny(ny_), nz(nz_), px(parity & 1), py((parity >> 1) & 1), pz((parity >> 2) & 1) {
    cx = (nx - px + 1) / 2;
    cy = (ny - py + 1) / 2;
    cz = (nz - pz + 1) / 2;
  }
  __host__ __device__ int64_t count() const { return cx * cy * cz; }
  __host__ __device__ int64_t row(int64_t k) const {
    const int64_t a = k % cx, b = (k / cx) % cy, c = k / (cx * cy);
    return (2 * a + px) + nx * ((2 * b + py) + ny * (2 * c + pz));
  }
};

struct Offsets {
  int32_t o[27];
};

// Copies the DIA values of one colour into its colour-major block; the main
// diagonal (index d0) is stored as its reciprocal, so that the smoother
// multiplies instead of dividing (an FP64 division costs several FP64
// instructions on this GPU).
__global__ void colour_values_kernel(ColourGrid g, int ndiag, int d0, const double* __restrict__ val,
                                     int64_t ld, double* __restrict__ out) {
  const int64_t n = g.count();
  for (int64_t k = (int64_t)blockIdx.x * T + threadIdx.x; k < n; k += (int64_t)gridDim.x * T) {
    const int64_t i = g.row(k);
    for (int d = 0; d < ndiag; ++d) {
      const double a = val[(int64_t)d * ld + i];
      out[(int64_t)d * n + k] = d == d0 ? 1.0 / a : a;
    }
  }
}

// ---------------------------------------------------------------------------
// The whole symmetric sweep in one cooperative launch: the 15 colour passes
// (0..7, then 6..0) separated by a grid barrier, instead of 15 launches
// whose fixed cost dominates on the coarse levels. z, written by other
// blocks between passes, is read through L2 (ld.global.cg), never from a
// possibly stale L1 line.
// The barrier (grid_barrier) is bounded: on timeout a block sets bar[2] and
// returns; the host reports DYNMAT_ERR_TIMEOUT and resets the barrier.
// ---------------------------------------------------------------------------
struct ColourStarts {
  int64_t s[8];
};

template <int ND>
__global__ void __launch_bounds__(T)
symgs_sweep_kernel(int64_t nx, int64_t ny, int64_t nz, Offsets offs,
                   const double* __restrict__ valc, ColourStarts cs,
                   const double* __restrict__ r, double* z, const int32_t* __restrict__ skip,
                   unsigned* bar) {
  constexpr int D0 = ND / 2;
  if (skip && *skip) return;
  const int64_t N = nx * ny * nz;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int step = 0; step < 15; ++step) {
    const int colour = step < 8 ? step : 14 - step;
    const ColourGrid g(nx, ny, nz, 7 - colour);
    int64_t start = 0;  // cs.s[colour] without indexing the parameter array
#pragma unroll
    for (int c = 0; c < 8; ++c)
      if (c == colour) start = cs.s[c];
    const double* vc = valc + start;
    const int64_t n = g.count();
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
      const int64_t i = g.row(k);
      double v[ND], zz[ND];
#pragma unroll
      for (int d = 0; d < ND; ++d) v[d] = __ldg(vc + (int64_t)d * n + k);
#pragma unroll
      for (int d = 0; d < ND; ++d) {
        if (d == D0) continue;
        const int64_t j = min(max(i + (int64_t)offs.o[d], (int64_t)0), N - 1);
        zz[d] = __ldcg(z + j);
      }
      double acc = __ldg(r + i);
#pragma unroll
      for (int d = 0; d < ND; ++d)
        if (d != D0) acc = fma(-v[d], zz[d], acc);
      z[i] = acc * v[D0];
    }
    if (step < 14 && !grid_barrier(bar)) return;
  }
}

__global__ void sub_kernel(const double* __restrict__ r, double* __restrict__ t, int64_t n,
                           const int32_t* __restrict__ skip) {
  if (skip && *skip) return;
  for (int64_t i = (int64_t)blockIdx.x * T + threadIdx.x; i < n; i += (int64_t)gridDim.x * T)
    t[i] = r[i] - t[i];
}

// coarse (cx, cy, cz) <-> fine (2cx, 2cy, 2cz)
__global__ void restrict_kernel(const double* __restrict__ fine, int64_t fnx, int64_t fny,
                                double* __restrict__ coarse, int64_t nx, int64_t ny, int64_t nz,
                                const int32_t* __restrict__ skip) {
  if (skip && *skip) return;
  const int64_t n = nx * ny * nz;
  for (int64_t i = (int64_t)blockIdx.x * T + threadIdx.x; i < n; i += (int64_t)gridDim.x * T) {
    const int64_t x = i % nx, y = (i / nx) % ny, zz = i / (nx * ny);
    coarse[i] = fine[2 * x + fnx * (2 * y + fny * 2 * zz)];
  }
}

__global__ void prolong_kernel(double* __restrict__ fine, int64_t fnx, int64_t fny,
                               const double* __restrict__ coarse, int64_t nx, int64_t ny, int64_t nz,
                               const int32_t* __restrict__ skip) {
  if (skip && *skip) return;
  const int64_t n = nx * ny * nz;
  for (int64_t i = (int64_t)blockIdx.x * T + threadIdx.x; i < n; i += (int64_t)gridDim.x * T) {
    const int64_t x = i % nx, y = (i / nx) % ny, zz = i / (nx * ny);
    const int64_t f = 2 * x + fnx * (2 * y + fny * 2 * zz);
    fine[f] = fine[f] + coarse[i];
  }
}

void symgs(dynmat_mg_s* M, int l, const double* r, double* z, const int32_t* skip,
           cudaStream_t s) {
  const auto& d = M->dims[l];
  Offsets offs{};
  // the stencil's offsets: (dz, dy, dx) lexicographic, as the DIA holds them
  int k = 0;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const bool face = (dz != 0) + (dy != 0) + (dx != 0) <= 1;
        if (M->points == 27 || face) offs.o[k++] = (int32_t)(dz * d[0] * d[1] + dy * d[0] + dx);
      }
  ColourStarts cs{};
  for (int c = 0; c < 8; ++c) cs.s[c] = M->cstart[l][c];
  // Colour 7 ends the forward pass and would start the backward one: its
  // neighbours have not changed in between, so the second update would give
  // the same bits and is skipped (15 passes per sweep). A colour of a coarse
  // level is a few thousand points: blocks of 32 or 64 threads put it on more
  // SMs (the FP64 pipe of each SM is narrow). The grid stays within what is
  // co-resident, which the cooperative launch checks.
  const int64_t cnt = ColourGrid(d[0], d[1], d[2], 0).count(), sms = device().sms;
  const int bs = cnt < sms * 64 ? 32 : (cnt < sms * 512 ? 64 : T);
  const void* fn = M->points == 27 ? (const void*)symgs_sweep_kernel<27>
                                   : (const void*)symgs_sweep_kernel<7>;
  int per_sm = 0;
  DM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, bs, 0));
  const unsigned grid = (unsigned)std::max<int64_t>(
      1, std::min<int64_t>(cdiv(cnt, bs), std::max(per_sm, 1) * sms));
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(bs);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const double* vc = M->valc[l].as<double>();
  unsigned* bar = M->bar.as<unsigned>();
  if (M->points == 27)
    DM_CUDA(cudaLaunchKernelEx(&cfg, symgs_sweep_kernel<27>, (int64_t)d[0], (int64_t)d[1],
                               (int64_t)d[2], offs, vc, cs, r, z, skip, bar));
  else
    DM_CUDA(cudaLaunchKernelEx(&cfg, symgs_sweep_kernel<7>, (int64_t)d[0], (int64_t)d[1],
                               (int64_t)d[2], offs, vc, cs, r, z, skip, bar));
}

void vcycle_level(dynmat_mg_s* M, int l, const double* r, double* z, const int32_t* skip,
                  cudaStream_t s) {
  const auto& d = M->dims[l];
  const int64_t n = d[0] * d[1] * d[2];
  DM_CUDA(cudaMemsetAsync(z, 0, n * sizeof(double), s));
  symgs(M, l, r, z, skip, s);
  if (l == M->levels - 1) return;
  double* t = M->t[l].as<double>();
  spmv_skip(M->A[l], z, t, DYNMAT_F64, nullptr, skip, s);
  sub_kernel<<<grid_of(n), T, 0, s>>>(r, t, n, skip);
  DM_CHECK_LAUNCH();
  const auto& c = M->dims[l + 1];
  const int64_t nc = c[0] * c[1] * c[2];
  double* rc = M->r[l + 1].as<double>();
  double* zc = M->z[l + 1].as<double>();
  restrict_kernel<<<grid_of(nc), T, 0, s>>>(t, d[0], d[1], rc, c[0], c[1], c[2], skip);
  DM_CHECK_LAUNCH();
  vcycle_level(M, l + 1, rc, zc, skip, s);
  prolong_kernel<<<grid_of(nc), T, 0, s>>>(z, d[0], d[1], zc, c[0], c[1], c[2], skip);
  DM_CHECK_LAUNCH();
  symgs(M, l, r, z, skip, s);
}

void destroy_mg(dynmat_mg_s* M, cudaStream_t s) {
  if (!M) return;
  for (auto* A : M->A)
    if (A) dynmat_destroy(A, s);
  for (auto& b : M->r) b.release();
  for (auto& b : M->z) b.release();
  for (auto& b : M->t) b.release();
  for (auto& b : M->valc) b.release();
  M->bar.release();
  delete M;
}

}  // namespace

void mg_vcycle(dynmat_mg_s* M, const double* r, double* z, const int32_t* skip, cudaStream_t s) {
  vcycle_level(M, 0, r, z, skip, s);
}

const dynmat_s* mg_matrix(const dynmat_mg_s* M) { return M->A[0]; }

// Blocking: DYNMAT_ERR_TIMEOUT (and a reset barrier) if a smoother's grid
// barrier timed out since the last check.
void mg_check_timeout(dynmat_mg_s* M, cudaStream_t s) {
  unsigned h[3] = {0, 0, 0};
  DM_CUDA(cudaMemcpyAsync(h, M->bar.p, sizeof h, cudaMemcpyDeviceToHost, s));
  DM_CUDA(cudaStreamSynchronize(s));
  if (h[2]) {
    DM_CUDA(cudaMemsetAsync(M->bar.p, 0, 16, s));
    DM_CUDA(cudaStreamSynchronize(s));
  }
  DM_REQUIRE(h[2] == 0, DYNMAT_ERR_TIMEOUT,
             "a grid barrier of the multigrid smoother timed out; results since the last check "
             "are invalid");
}

}  // namespace dm

using namespace dm;

extern "C" {

dynmat_status dynmat_mg_create(dynmat_mg_t* out, int64_t nx, int64_t ny, int64_t nz,
                               int32_t points, int32_t levels, dynmat_stream_t stream) {
  return guard([&] {
    DM_REQUIRE(out, DYNMAT_ERR_INVALID_ARG, "out is NULL");
    DM_REQUIRE(levels >= 1 && levels <= 8, DYNMAT_ERR_INVALID_ARG, "levels must be 1..8");
    DM_REQUIRE(points == 7 || points == 27, DYNMAT_ERR_INVALID_ARG, "points must be 7 or 27");
    const int64_t div = (int64_t)1 << (levels - 1);
    DM_REQUIRE(nx > 0 && ny > 0 && nz > 0 && nx % div == 0 && ny % div == 0 && nz % div == 0,
               DYNMAT_ERR_INVALID_ARG, "grid %lld x %lld x %lld must divide by 2^(levels-1) = %lld",
               (long long)nx, (long long)ny, (long long)nz, (long long)div);
    // every level keeps all the stencil's diagonals (distinct offsets)
    const int64_t least = points == 27 ? 3 : 2;
    DM_REQUIRE(nx / div >= least && ny / div >= least && nz / div >= least,
               DYNMAT_ERR_INVALID_ARG,
               "the coarsest grid must have at least %lld points per dimension",
               (long long)least);
    cudaStream_t s = (cudaStream_t)stream;
    std::unique_ptr<dynmat_mg_s, void (*)(dynmat_mg_s*)> M(
        new dynmat_mg_s, [](dynmat_mg_s* m) { destroy_mg(m, nullptr); });
    M->levels = levels;
    M->points = points;
    for (int l = 0; l < levels; ++l) {
      const std::array<int64_t, 3> d = {nx >> l, ny >> l, nz >> l};
      M->dims.push_back(d);
      dynmat_t A = nullptr;
      const dynmat_status st =
          dynmat_create_stencil(&A, d[0], d[1], d[2], points, DYNMAT_DIA, DYNMAT_F64, stream);
      if (st != DYNMAT_OK) throw Fail{st};
      M->A.push_back(A);
      // the offset-0 diagonal: offsets ascend, so it is the one with zero
      const int64_t nd = A->dia.ndiag;
      std::vector<int32_t> off((size_t)nd);
      DM_CUDA(cudaMemcpyAsync(off.data(), A->dia.offsets.p, nd * 4, cudaMemcpyDeviceToHost, s));
      DM_CUDA(cudaStreamSynchronize(s));
      int32_t d0 = -1;
      for (int64_t k = 0; k < nd; ++k)
        if (off[k] == 0) d0 = (int32_t)k;
      DM_REQUIRE(d0 >= 0, DYNMAT_ERR_INVALID_ARG, "level %d has no main diagonal", l);
      DM_REQUIRE(d0 == nd / 2 && nd == points, DYNMAT_ERR_INVALID_ARG,
                 "level %d: unexpected stencil diagonals", l);
      M->d0.push_back(d0);
      {
        std::array<int64_t, 8> starts{};
        int64_t total = 0;
        for (int colour = 0; colour < 8; ++colour) {
          starts[colour] = total;
          total += ColourGrid(d[0], d[1], d[2], 7 - colour).count() * nd;
        }
        M->valc.emplace_back(std::max<int64_t>(total, 1) * 8, s);
        for (int colour = 0; colour < 8; ++colour) {
          const ColourGrid g(d[0], d[1], d[2], 7 - colour);
          if (g.count() == 0) continue;
          colour_values_kernel<<<grid_of(g.count()), T, 0, s>>>(
              g, (int)nd, d0, A->dia.val.as<double>(), A->dia.ld,
              M->valc.back().as<double>() + starts[colour]);
          DM_CHECK_LAUNCH();
        }
        M->cstart.push_back(starts);
      }
      const int64_t n = d[0] * d[1] * d[2];
      M->r.emplace_back(l > 0 ? n * 8 : 8, s);
      M->z.emplace_back(l > 0 ? n * 8 : 8, s);
      M->t.emplace_back(l + 1 < levels ? n * 8 : 8, s);
    }
    M->bar.alloc(16, s);
    DM_CUDA(cudaMemsetAsync(M->bar.p, 0, 16, s));
    DM_CUDA(cudaStreamSynchronize(s));
    *out = M.release();
  });
}

dynmat_status dynmat_mg_destroy(dynmat_mg_t M, dynmat_stream_t stream) {
  return guard([&] { destroy_mg(M, (cudaStream_t)stream); });
}

dynmat_status dynmat_mg_level(dynmat_mg_t M, int32_t level, dynmat_t* A_out, int64_t* dims_out) {
  return guard([&] {
    DM_REQUIRE(M, DYNMAT_ERR_INVALID_ARG, "null hierarchy");
    DM_REQUIRE(level >= 0 && level < M->levels, DYNMAT_ERR_INVALID_ARG, "level %d out of range",
               level);
    if (A_out) *A_out = M->A[level];
    if (dims_out)
      for (int k = 0; k < 3; ++k) dims_out[k] = M->dims[level][k];
  });
}

dynmat_status dynmat_mg_symgs(dynmat_mg_t M, int32_t level, const double* r, double* z,
                              dynmat_stream_t stream) {
  return guard([&] {
    DM_REQUIRE(M, DYNMAT_ERR_INVALID_ARG, "null hierarchy");
    DM_REQUIRE(level >= 0 && level < M->levels, DYNMAT_ERR_INVALID_ARG, "level %d out of range",
               level);
    DM_REQUIRE(r && z, DYNMAT_ERR_INVALID_ARG, "null vector");
    symgs(M, level, r, z, nullptr, (cudaStream_t)stream);
  });
}

dynmat_status dynmat_mg_apply(dynmat_mg_t M, const double* r, double* z, dynmat_stream_t stream) {
  return guard([&] {
    DM_REQUIRE(M, DYNMAT_ERR_INVALID_ARG, "null hierarchy");
    DM_REQUIRE(r && z, DYNMAT_ERR_INVALID_ARG, "null vector");
    mg_vcycle(M, r, z, nullptr, (cudaStream_t)stream);
  });
}

}  // extern "C"
