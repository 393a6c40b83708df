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
//    coarse r = (r - A z) at the coarse points (injection: the residual is
//    formed only there, in one kernel), the coarse V-cycle, z += coarse z at
//    the coarse points, post-smooth.
//  - A sweep that starts from z = 0 (every pre-smoothing, and the coarsest
//    level) skips, in its forward pass, the neighbours of colours not yet
//    updated: their z is still 0, so their products are exactly 0.
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
  std::vector<dm::DBuf> r, z;
  // Per level, the DIA values again (the main diagonal as its reciprocal),
  // colour by colour: colour c's block holds
  // ndiag x count_c values, value d of the colour's k-th point at d*count_c+k
  // (contiguous reads in a colour pass; the natural layout serves the SpMV).
  std::vector<dm::DBuf> valc;
  std::vector<std::array<int64_t, 8>> cstart;  // first value of each colour's block
  // Grid barriers of the fused smoother, one per launch site (level l,
  // zero start or not: site 2 l + zs), 16 bytes each: a 64-bit arrival
  // count and a timeout flag. A site always launches the same grid, which
  // keeps its count a multiple of the grid between launches.
  dm::DBuf bar;
  int nbar = 0;
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
// The barrier (grid_barrier) is bounded: on timeout a block sets its site's
// flag and returns; the host reports DYNMAT_ERR_TIMEOUT and resets the
// barriers.
// ---------------------------------------------------------------------------
struct ColourStarts {
  int64_t s[8];
};

// Colour of the neighbour at stencil slot d of a point of colour `colour`:
// the neighbour's coordinate parities differ by those of the offset.
__host__ __device__ constexpr int neighbour_colour(int nd, int colour, int d) {
  const int dx = nd == 27 ? d % 3 - 1 : (d == 2 ? -1 : d == 4 ? 1 : 0);
  const int dy = nd == 27 ? (d / 3) % 3 - 1 : (d == 1 ? -1 : d == 5 ? 1 : 0);
  const int dz = nd == 27 ? d / 9 - 1 : (d == 0 ? -1 : d == 6 ? 1 : 0);
  const int q = (dx & 1) | ((dy & 1) << 1) | ((dz & 1) << 2);
  return 7 - ((7 - colour) ^ q);
}

// Slots a colour pass reads (bit d): all of them, or, in the forward pass of
// a sweep that starts from z = 0, the diagonal and the neighbours of earlier
// colours (the later ones still hold z = 0, so their products are exactly 0).
__host__ __device__ constexpr uint32_t live_slots(int nd, int colour, bool zero_forward) {
  uint32_t m = 0;
  for (int d = 0; d < nd; ++d)
    if (!zero_forward || d == nd / 2 || neighbour_colour(nd, colour, d) < colour) m |= 1u << d;
  return m;
}

// One colour pass: z_i = (r_i - sum_{j != i} a_ij z_j) / a_ii over the
// colour's points, slots outside LIVE skipped.
template <int ND, uint32_t LIVE>
__device__ __forceinline__ void colour_pass(int64_t nx, int64_t ny, int64_t nz, int colour,
                                            const Offsets& offs, const double* __restrict__ valc,
                                            int64_t start, const double* __restrict__ r,
                                            double* z) {
  constexpr int D0 = ND / 2;
  const ColourGrid g(nx, ny, nz, 7 - colour);
  const int64_t N = nx * ny * nz;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const double* vc = valc + start;
  const int64_t n = g.count();
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
    const int64_t i = g.row(k);
    double v[ND], zz[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d)
      if ((LIVE >> d) & 1) v[d] = __ldg(vc + (int64_t)d * n + k);
#pragma unroll
    for (int d = 0; d < ND; ++d) {
      if (d == D0 || !((LIVE >> d) & 1)) continue;
      const int64_t j = min(max(i + (int64_t)offs.o[d], (int64_t)0), N - 1);
      zz[d] = __ldcg(z + j);
    }
    double acc = __ldg(r + i);
#pragma unroll
    for (int d = 0; d < ND; ++d)
      if (d != D0 && ((LIVE >> d) & 1)) acc = fma(-v[d], zz[d], acc);
    z[i] = acc * v[D0];
  }
}

// The forward pass of a zero-start sweep, colours C..7, each with its own
// compile-time slot set, separated by grid barriers. False on a barrier
// timeout.
template <int ND, int C>
__device__ __forceinline__ bool zero_forward(int64_t nx, int64_t ny, int64_t nz, const Offsets& offs,
                                             const double* __restrict__ valc, const ColourStarts& cs,
                                             const double* __restrict__ r, double* z, unsigned* bar) {
  if constexpr (C < 8) {
    colour_pass<ND, live_slots(ND, C, true)>(nx, ny, nz, C, offs, valc, cs.s[C], r, z);
    if (!grid_barrier(bar)) return false;
    return zero_forward<ND, C + 1>(nx, ny, nz, offs, valc, cs, r, z, bar);
  } else {
    return true;
  }
}

template <int ND, bool ZERO_START>
__global__ void __launch_bounds__(T, ND == 27 ? 2 : 6)
symgs_sweep_kernel(int64_t nx, int64_t ny, int64_t nz, Offsets offs,
                   const double* __restrict__ valc, ColourStarts cs,
                   const double* __restrict__ r, double* z, const int32_t* __restrict__ skip,
                   unsigned* bar) {
  constexpr uint32_t ALL = (1u << ND) - 1;
  if (skip && *skip) return;
  int step = 0;
  if constexpr (ZERO_START) {
    if (!zero_forward<ND, 0>(nx, ny, nz, offs, valc, cs, r, z, bar)) return;
    step = 8;
  }
  for (; step < 15; ++step) {
    const int colour = step < 8 ? step : 14 - step;
    int64_t start = 0;  // cs.s[colour] without indexing the parameter array
#pragma unroll
    for (int c = 0; c < 8; ++c)
      if (c == colour) start = cs.s[c];
    colour_pass<ND, ALL>(nx, ny, nz, colour, offs, valc, start, r, z);
    if (step < 14 && !grid_barrier(bar)) return;
  }
}

// Coarse r = (r - A z) at the coarse points (all coordinates even: colour 7,
// whose k-th point is coarse point k). The off-diagonal values come from
// colour 7's colour-major block, the diagonal from the DIA array; the
// products are summed in slot order, then subtracted from r.
template <int ND>
__global__ void __launch_bounds__(T)
residual_restrict_kernel(ColourGrid g, Offsets offs, const double* __restrict__ valc7,
                         const double* __restrict__ diag, const double* __restrict__ r,
                         const double* __restrict__ z, double* __restrict__ rc,
                         const int32_t* __restrict__ skip) {
  constexpr int D0 = ND / 2;
  if (skip && *skip) return;
  const int64_t N = g.nx * g.ny * g.nz, n = g.count();
  for (int64_t k = (int64_t)blockIdx.x * T + threadIdx.x; k < n; k += (int64_t)gridDim.x * T) {
    const int64_t i = g.row(k);
    double v[ND], zz[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) {
      v[d] = d == D0 ? __ldg(diag + i) : __ldg(valc7 + (int64_t)d * n + k);
      const int64_t j = min(max(i + (int64_t)offs.o[d], (int64_t)0), N - 1);
      zz[d] = __ldg(z + j);
    }
    double acc = 0.0;
#pragma unroll
    for (int d = 0; d < ND; ++d) acc = fma(v[d], zz[d], acc);
    rc[k] = __ldg(r + i) - acc;
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

// The stencil's offsets on level l: (dz, dy, dx) lexicographic, as the DIA
// holds them.
Offsets stencil_offsets(const dynmat_mg_s* M, int l) {
  const auto& d = M->dims[l];
  Offsets offs{};
  int k = 0;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const bool face = (dz != 0) + (dy != 0) + (dx != 0) <= 1;
        if (M->points == 27 || face) offs.o[k++] = (int32_t)(dz * d[0] * d[1] + dy * d[0] + dx);
      }
  return offs;
}

// One symmetric sweep on level l; zero_start: z is 0 when it begins.
void symgs(dynmat_mg_s* M, int l, const double* r, double* z, const int32_t* skip,
           bool zero_start, cudaStream_t s) {
  const auto& d = M->dims[l];
  const Offsets offs = stencil_offsets(M, l);
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
  const void* fn =
      M->points == 27
          ? (zero_start ? (const void*)symgs_sweep_kernel<27, true> : (const void*)symgs_sweep_kernel<27, false>)
          : (zero_start ? (const void*)symgs_sweep_kernel<7, true> : (const void*)symgs_sweep_kernel<7, false>);
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
  unsigned* bar = M->bar.as<unsigned>() + 4 * (2 * l + (zero_start ? 1 : 0));
  void* args[] = {(void*)&d[0], (void*)&d[1], (void*)&d[2], (void*)&offs, (void*)&vc,
                  (void*)&cs, (void*)&r, (void*)&z, (void*)&skip, (void*)&bar};
  DM_CUDA(cudaLaunchKernelExC(&cfg, fn, args));
}

void vcycle_level(dynmat_mg_s* M, int l, const double* r, double* z, const int32_t* skip,
                  cudaStream_t s) {
  const auto& d = M->dims[l];
  const int64_t n = d[0] * d[1] * d[2];
  DM_CUDA(cudaMemsetAsync(z, 0, n * sizeof(double), s));
  symgs(M, l, r, z, skip, true, s);
  if (l == M->levels - 1) return;
  const auto& c = M->dims[l + 1];
  const int64_t nc = c[0] * c[1] * c[2];
  double* rc = M->r[l + 1].as<double>();
  double* zc = M->z[l + 1].as<double>();
  {
    const ColourGrid g7(d[0], d[1], d[2], 0);  // colour 7: the coarse points, in coarse order
    const Offsets offs = stencil_offsets(M, l);
    const double* valc7 = M->valc[l].as<double>() + M->cstart[l][7];
    const dynmat_s* A = M->A[l];
    const double* diag = A->dia.val.as<double>() + (int64_t)M->d0[l] * A->dia.ld;
    if (M->points == 27)
      residual_restrict_kernel<27><<<grid_of(nc), T, 0, s>>>(g7, offs, valc7, diag, r, z, rc, skip);
    else
      residual_restrict_kernel<7><<<grid_of(nc), T, 0, s>>>(g7, offs, valc7, diag, r, z, rc, skip);
    DM_CHECK_LAUNCH();
  }
  vcycle_level(M, l + 1, rc, zc, skip, s);
  prolong_kernel<<<grid_of(nc), T, 0, s>>>(z, d[0], d[1], zc, c[0], c[1], c[2], skip);
  DM_CHECK_LAUNCH();
  symgs(M, l, r, z, skip, false, s);
}

void destroy_mg(dynmat_mg_s* M, cudaStream_t s) {
  if (!M) return;
  for (auto* A : M->A)
    if (A) dynmat_destroy(A, s);
  for (auto& b : M->r) b.release();
  for (auto& b : M->z) b.release();
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
  std::vector<unsigned> h((size_t)4 * M->nbar, 0u);
  DM_CUDA(cudaMemcpyAsync(h.data(), M->bar.p, h.size() * sizeof(unsigned), cudaMemcpyDeviceToHost,
                          s));
  DM_CUDA(cudaStreamSynchronize(s));
  bool timed_out = false;
  for (int k = 0; k < M->nbar; ++k) timed_out = timed_out || h[4 * k + 2] != 0;
  if (timed_out) {  // counts left mid-barrier: start every site afresh
    DM_CUDA(cudaMemsetAsync(M->bar.p, 0, (size_t)16 * M->nbar, s));
    DM_CUDA(cudaStreamSynchronize(s));
  }
  DM_REQUIRE(!timed_out, DYNMAT_ERR_TIMEOUT,
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
    }
    M->nbar = 2 * levels;
    M->bar.alloc((size_t)16 * M->nbar, s);
    DM_CUDA(cudaMemsetAsync(M->bar.p, 0, (size_t)16 * M->nbar, s));
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
    symgs(M, level, r, z, nullptr, false, (cudaStream_t)stream);
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
