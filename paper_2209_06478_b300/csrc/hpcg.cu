// HPCG's multigrid preconditioner (§II-B: the benchmark's PCG uses a
// symmetric Gauss-Seidel smoother inside multigrid; the paper runs CG with the
// preconditioner disabled, §IV-B). Level l is the stencil on the grid halved
// l times; each level is a dynamic matrix in DIA (FP64).
//  - Smoother: one symmetric Gauss-Seidel sweep in colour order, colour(i) =
//    7 - ((ix & 1) + 2 (iy & 1) + 4 (iz & 1)); no two stencil neighbours
//    share a colour, so a colour's rows are updated in parallel, one pass
//    per colour: forward colours 0..7, backward 7..0. The coarse grid's
//    points (all coordinates even) are colour 7 so that the last colour of a
//    sweep, whose residual the sweep zeroes, is not the one injected.
//    z_i = (r_i - sum_{j != i} a_ij z_j) / a_ii with the diagonals in
//    ascending offset order (DIA slots outside the grid hold 0).
//  - V-cycle: z = 0; the coarsest level is one sweep; otherwise pre-smooth,
//    coarse r = (r - A z) at the coarse points (injection: the residual is
//    formed only there), the coarse V-cycle, z += coarse z at the coarse
//    points, post-smooth. Launches: the finest level's two sweeps, and
//    everything between them (all coarser levels and the transfers) as one
//    cooperative launch; or, where the smallest levels fit one thread-block
//    cluster, three: the descent to them and the ascent from them on the
//    grid, and the smallest levels on the cluster.
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
  // Grid barriers, one per launch site (the sweep of level l with zero start
  // or not: site 2 l + zs; the coarse cycle: site 2 levels; its descent and
  // ascent around a cluster: sites 2 levels + 1 and + 2): the 64-bit
  // arrival counts of all sites, then their timeout flags. A count is cleared
  // before each launch of its site.
  dm::DBuf bar;
  int nbar = 0;
  // The coarse levels cl_first..levels-1 run on one thread-block cluster of
  // cl_ctas CTAs (0: no cluster; the whole coarse cycle on the grid). Per
  // level, its distributed arrays hold 2^cl_lp z-planes per CTA, and its z
  // and r slices start at byte cl_z and cl_r of each CTA's shared memory.
  int cl_ctas = 0, cl_first = 0;
  size_t cl_smem = 0;
  uint32_t cl_vbuf = 0, cl_pts = 0, cl_info = 0;  // byte offsets of the buffers and tables
  std::vector<uint32_t> cl_lp, cl_z, cl_r;
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
  // In 32 bits: a level has fewer than 2^31 points (checked at creation),
  // and 64-bit divisions are long emulated sequences on the critical path of
  // every colour pass.
  __host__ __device__ int64_t row(int64_t k) const {
    uint32_t x, y, z;
    coords(k, x, y, z);
    return (int64_t)(x + (uint32_t)nx * (y + (uint32_t)ny * z));
  }
  __host__ __device__ void coords(int64_t k, uint32_t& x, uint32_t& y, uint32_t& z) const {
    const uint32_t kk = (uint32_t)k, ux = (uint32_t)cx, uy = (uint32_t)cy;
    const uint32_t q = kk / ux, a = kk - q * ux, c = q / uy, b = q - c * uy;
    x = 2 * a + px;
    y = 2 * b + py;
    z = 2 * c + pz;
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
// flag and returns; pcg_solve reports DYNMAT_ERR_TIMEOUT and clears the
// flags.
// ---------------------------------------------------------------------------
struct ColourStarts {
  int64_t s[8];
};

// Colour of the neighbour at stencil slot d of a point of colour `colour`:
// the neighbour's coordinate parities differ by those of the offset.
// The offset (dx, dy, dz) of stencil slot d: the slots in (dz, dy, dx)
// lexicographic order, 27 points or the 7 of the faces and the centre.
__host__ __device__ constexpr int slot_dx(int nd, int d) {
  return nd == 27 ? d % 3 - 1 : (d == 2 ? -1 : d == 4 ? 1 : 0);
}
__host__ __device__ constexpr int slot_dy(int nd, int d) {
  return nd == 27 ? (d / 3) % 3 - 1 : (d == 1 ? -1 : d == 5 ? 1 : 0);
}
__host__ __device__ constexpr int slot_dz(int nd, int d) {
  return nd == 27 ? d / 9 - 1 : (d == 0 ? -1 : d == 6 ? 1 : 0);
}

__host__ __device__ constexpr int neighbour_colour(int nd, int colour, int d) {
  const int dx = slot_dx(nd, d), dy = slot_dy(nd, d), dz = slot_dz(nd, d);
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

// The points [0, n) of a pass, block b taking the consecutive run
// [b m, (b + 1) m) with m = ceil(n / blocks): a pass of a few thousand points
// still spreads over every SM (one FP64 pipe each, and narrow), and a block's
// loads stay coalesced.
struct BlockRange {
  int64_t k, end;
  int64_t step;
  __device__ explicit BlockRange(int64_t n) {  // n < 2^31
    const int64_t m = ((uint32_t)n + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = (int64_t)blockIdx.x * m;
    k = b0 + threadIdx.x;
    end = min(n, b0 + m);
    step = blockDim.x;
  }
  __device__ bool more() const { return k < end; }
  __device__ void next() { k += step; }
};

// A launch's grid barrier: its arrival count (cleared by the host before
// the launch) and its timeout flag.
struct GridBar {
  unsigned long long* count;
  unsigned* timeout;
};

// One level as the device sees it.
struct MgLevel {
  int64_t nx, ny, nz;
  Offsets offs;
  ColourStarts cs;
  const double* valc;  // colour-major values, the diagonal as its reciprocal
  const double* diag;  // the DIA's main diagonal (the residual's a_ii)
  const double* r;     // right-hand side
  double* z;           // solution
};

// One colour pass: z_i = (r_i - sum_{j != i} a_ij z_j) / a_ii over the
// colour's points, slots outside LIVE skipped. SPLIT (27 points): the
// neighbours are summed per z-plane in three chains (9, 8 and 9 products)
// added at the end, a third of the latency of one 26-product chain (a
// dependent FP64 multiply-add takes 64 cycles here): for the coarse levels,
// whose passes are too small to hide it. r and z may have been written
// earlier in the launch: both are read through L2.
template <int ND, uint32_t LIVE, bool SPLIT>
__device__ __forceinline__ void colour_pass(const MgLevel& L, int colour, int64_t start) {
  constexpr int D0 = ND / 2;
  constexpr int PLANES = SPLIT && ND == 27 ? 3 : 1;
  const ColourGrid g(L.nx, L.ny, L.nz, 7 - colour);
  const int64_t N = L.nx * L.ny * L.nz;
  const double* vc = L.valc + start;
  const int64_t n = g.count();
  if constexpr (!SPLIT && ND == 27) {
    // Plane by plane (the 9 slots of dz = -1, 0, +1): 9 values and 9
    // neighbours in flight at a time, one chain in slot order (the same
    // sums as below), so the pass fits in 64 registers.
    for (BlockRange br(n); br.more(); br.next()) {
      const int64_t k = br.k;
      const int64_t i = g.row(k);
      double acc = __ldcg(L.r + i), inv = 0.0;
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        double v[9], zz[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) {
          const int d = 9 * p + q;
          if ((LIVE >> d) & 1) v[q] = __ldg(vc + (int64_t)d * n + k);
          if (d == D0 || !((LIVE >> d) & 1)) continue;
          const int64_t j = min(max(i + (int64_t)L.offs.o[d], (int64_t)0), N - 1);
          zz[q] = __ldcg(L.z + j);
        }
#pragma unroll
        for (int q = 0; q < 9; ++q) {
          const int d = 9 * p + q;
          if (d == D0) inv = v[q];
          else if ((LIVE >> d) & 1) acc = fma(-v[q], zz[q], acc);
        }
      }
      L.z[i] = acc * inv;
    }
    return;
  }
  for (BlockRange br(n); br.more(); br.next()) {
    const int64_t k = br.k;
    const int64_t i = g.row(k);
    double v[ND], zz[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d)
      if ((LIVE >> d) & 1) v[d] = __ldg(vc + (int64_t)d * n + k);
#pragma unroll
    for (int d = 0; d < ND; ++d) {
      if (d == D0 || !((LIVE >> d) & 1)) continue;
      const int64_t j = min(max(i + (int64_t)L.offs.o[d], (int64_t)0), N - 1);
      zz[d] = __ldcg(L.z + j);
    }
    double acc[PLANES];
    acc[0] = __ldcg(L.r + i);
#pragma unroll
    for (int p = 1; p < PLANES; ++p) acc[p] = 0.0;
#pragma unroll
    for (int d = 0; d < ND; ++d)
      if (d != D0 && ((LIVE >> d) & 1)) {
        const int p = PLANES == 3 ? d / 9 : 0;
        acc[p] = fma(-v[d], zz[d], acc[p]);
      }
    double t = acc[0];
#pragma unroll
    for (int p = 1; p < PLANES; ++p) t = t + acc[p];
    L.z[i] = t * v[D0];
  }
}

// The forward pass of a zero-start sweep, colours C..7, each with its own
// compile-time slot set, separated by grid barriers. False on a barrier
// timeout.
template <int ND, bool SPLIT, int C>
__device__ __forceinline__ bool zero_forward(const MgLevel& L, const GridBar& bar) {
  if constexpr (C < 8) {
    colour_pass<ND, live_slots(ND, C, true), SPLIT>(L, C, L.cs.s[C]);
    if (!grid_barrier(bar.count, bar.timeout)) return false;
    return zero_forward<ND, SPLIT, C + 1>(L, bar);
  } else {
    return true;
  }
}

// One symmetric sweep: colours 0..7 then 6..0 (colour 7's second update
// would repeat the same bits), a grid barrier between passes and none after
// the last. False on a barrier timeout.
template <int ND, bool ZERO_START, bool SPLIT>
__device__ __forceinline__ bool sweep(const MgLevel& L, const GridBar& bar) {
  constexpr uint32_t ALL = (1u << ND) - 1;
  int step = 0;
  if constexpr (ZERO_START) {
    if (!zero_forward<ND, SPLIT, 0>(L, bar)) return false;
    step = 8;
  }
  for (; step < 15; ++step) {
    const int colour = step < 8 ? step : 14 - step;
    int64_t start = 0;  // L.cs.s[colour] without a dynamic index into the parameter
#pragma unroll
    for (int c = 0; c < 8; ++c)
      if (c == colour) start = L.cs.s[c];
    colour_pass<ND, ALL, SPLIT>(L, colour, start);
    if (step < 14 && !grid_barrier(bar.count, bar.timeout)) return false;
  }
  return true;
}

// Four blocks of 256 per SM (27 points: at most 64 registers, which the
// plane-by-plane pass fits without spilling): 32 warps per SM, so that while
// some wait on a plane's loads others keep the FP64 pipe busy. Two blocks
// (the whole point's 53 loads in flight, 124 registers) took 944 us per
// 128^3 V-cycle, three 858 us, four 825 us, five 882 us.
template <int ND, bool ZERO_START>
__global__ void __launch_bounds__(T, ND == 27 ? 4 : 6)
symgs_sweep_kernel(MgLevel L, const int32_t* __restrict__ skip, GridBar bar) {
  if (skip && *skip) return;
  sweep<ND, ZERO_START, false>(L, bar);
}

// Coarse r = (r - A z) at the coarse points of level F (all coordinates
// even: colour 7, whose k-th point is coarse point k). The off-diagonal
// values come from colour 7's colour-major block, the diagonal from the DIA
// array; the products are summed in slot order, then subtracted from r.
template <int ND>
__device__ __forceinline__ void residual_restrict(const MgLevel& F, double* rc) {
  constexpr int D0 = ND / 2;
  const ColourGrid g(F.nx, F.ny, F.nz, 0);
  const int64_t N = F.nx * F.ny * F.nz, n = g.count();
  const double* valc7 = F.valc + F.cs.s[7];
  for (BlockRange br(n); br.more(); br.next()) {
    const int64_t k = br.k;
    const int64_t i = g.row(k);
    double v[ND], zz[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) {
      v[d] = d == D0 ? __ldg(F.diag + i) : __ldg(valc7 + (int64_t)d * n + k);
      const int64_t j = min(max(i + (int64_t)F.offs.o[d], (int64_t)0), N - 1);
      zz[d] = __ldcg(F.z + j);
    }
    double acc = 0.0;
#pragma unroll
    for (int d = 0; d < ND; ++d) acc = fma(v[d], zz[d], acc);
    rc[k] = __ldcg(F.r + i) - acc;
  }
}

// z_F += z_C at the coarse points of level F.
__device__ __forceinline__ void prolong(const MgLevel& F, const double* zc) {
  const ColourGrid g(F.nx, F.ny, F.nz, 0);
  const int64_t n = g.count();
  for (BlockRange br(n); br.more(); br.next()) {
    const int64_t k = br.k;
    const int64_t f = g.row(k);
    F.z[f] = __ldcg(F.z + f) + __ldcg(zc + k);
  }
}

struct MgPlan {
  int32_t levels;
  MgLevel L[8];
};

// The descent of a V-cycle on the whole grid, down to level lc's right-hand
// side: z = 0 on levels 1..lc-1, level 1's right-hand side from level 0's
// residual, then per level l < lc its zero-start sweep and level l+1's
// right-hand side from its residual. False on a barrier timeout.
template <int ND>
__device__ __forceinline__ bool cycle_down(const MgPlan& P, int lc, const GridBar& bar) {
  for (int l = 1; l < lc; ++l) {  // zero-start sweeps begin from z = 0
    const int64_t n = P.L[l].nx * P.L[l].ny * P.L[l].nz;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
      P.L[l].z[i] = 0.0;
  }
  residual_restrict<ND>(P.L[0], const_cast<double*>(P.L[1].r));
  for (int l = 1; l < lc; ++l) {
    if (!grid_barrier(bar.count, bar.timeout)) return false;
    if (!sweep<ND, true, true>(P.L[l], bar)) return false;
    if (!grid_barrier(bar.count, bar.timeout)) return false;
    residual_restrict<ND>(P.L[l], const_cast<double*>(P.L[l + 1].r));
  }
  return true;
}

// The ascent from level lc's solution (complete when this begins): per
// level l = lc-1..1, z_l += z_{l+1} at the coarse points and the
// post-smoothing sweep; then level 0's prolongation.
template <int ND>
__device__ __forceinline__ void cycle_up(const MgPlan& P, int lc, const GridBar& bar) {
  for (int l = lc - 1; l >= 1; --l) {
    prolong(P.L[l], P.L[l + 1].z);
    if (!grid_barrier(bar.count, bar.timeout)) return;
    if (!sweep<ND, false, true>(P.L[l], bar)) return;
    if (!grid_barrier(bar.count, bar.timeout)) return;
  }
  prolong(P.L[0], P.L[1].z);
}

// Everything of a V-cycle between level 0's two sweeps, in one cooperative
// launch: the descent to the coarsest level, its (zero-start) sweep, the
// ascent. Grid barriers separate the steps, instead of about ten launches
// whose gaps and short tails dominate on these small grids; the coarse passes
// split their multiply-add chains (see colour_pass). Used when no coarse
// level fits the cluster kernel below.
template <int ND>
__global__ void __launch_bounds__(T, 2)
coarse_cycle_kernel(MgPlan P, const int32_t* __restrict__ skip, GridBar bar) {
  if (skip && *skip) return;
  const int lc = P.levels - 1;
  if (!cycle_down<ND>(P, lc, bar)) return;
  {  // cycle_down zeroes z below lc only
    const int64_t n = P.L[lc].nx * P.L[lc].ny * P.L[lc].nz;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
      P.L[lc].z[i] = 0.0;
  }
  if (!grid_barrier(bar.count, bar.timeout)) return;
  if (!sweep<ND, true, true>(P.L[lc], bar)) return;
  if (!grid_barrier(bar.count, bar.timeout)) return;
  cycle_up<ND>(P, lc, bar);
}

// With the coarse levels lc..levels-1 on one thread-block cluster: the
// descent to level lc's right-hand side, and, in a second launch, the ascent
// from its solution.
template <int ND>
__global__ void __launch_bounds__(T, 2)
coarse_down_kernel(MgPlan P, int lc, const int32_t* __restrict__ skip, GridBar bar) {
  if (skip && *skip) return;
  cycle_down<ND>(P, lc, bar);
}

template <int ND>
__global__ void __launch_bounds__(T, 2)
coarse_up_kernel(MgPlan P, int lc, const int32_t* __restrict__ skip, GridBar bar) {
  if (skip && *skip) return;
  cycle_up<ND>(P, lc, bar);
}

// ---------------------------------------------------------------------------
// The smallest levels on one thread-block cluster (16 CTAs where the device
// schedules clusters that large, else 8). A pass of such a level is a few
// hundred to a few thousand points: on the whole grid it costs a grid
// barrier (an atomic and a poll through L2, about 1.4 us) and L2 round
// trips for z, several times its arithmetic. Here each level's z and r are
// spread over the cluster's shared memory (distributed shared memory: any
// CTA reads and writes any CTA's slice), and the passes are separated by the
// cluster's hardware barrier. Each CTA updates the points of its own
// z-planes, at most one per thread (the host admits only levels whose
// colours have at most 256 points in any CTA's planes). The values still
// come from global memory, copied into shared memory two passes ahead.
// The arithmetic, and its order, is that of colour_pass's plane-by-plane
// form (one chain in slot order), residual_restrict and prolong; a neighbour
// outside the grid is clamped per coordinate instead of by linear index,
// which reads another point but multiplies it by the slot's 0.
// All CTAs take the same steps (the loop bounds are the plan's), so every
// cluster barrier is reached by all of them; a barrier of the hardware,
// not a poll of memory, it needs no time limit.
// ---------------------------------------------------------------------------
constexpr int CT = 256;  // threads per CTA of the cluster kernel

struct ClusterLevel {
  int32_t nx, ny, nz;
  uint32_t lp;     // a CTA holds 2^lp consecutive z-planes of each distributed array
  uint32_t slice;  // points per CTA: 2^lp nx ny
  uint32_t z, r;   // byte offsets of the level's z and r slices in each CTA's shared memory
  ColourStarts cs;
  const double* valc;
  const double* diag;
};

struct ClusterPlan {
  int32_t first, levels, ctas;  // levels first..levels-1, on `ctas` CTAs
  uint32_t vbuf;                // byte offset of the value buffers in shared memory
  uint32_t pts, info;           // byte offsets of the point and pass tables
  ClusterLevel L[8];
  const double* r_in;  // level first's right-hand side
  double* z_out;       // level first's solution
};

// Start of colour `colour`'s value block of level L.
__device__ __forceinline__ int64_t colour_start(const ClusterLevel& L, int colour) {
  int64_t start = 0;  // L.cs.s[colour] without a dynamic index into the parameter
#pragma unroll
  for (int c = 0; c < 8; ++c)
    if (c == colour) start = L.cs.s[c];
  return start;
}

namespace dsm {
__device__ __forceinline__ uint32_t rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// All threads of the cluster: writes before it (to any CTA's shared memory)
// are seen by reads after it.
__device__ __forceinline__ void sync() {
  __syncwarp();
  asm volatile(
      "barrier.cluster.arrive.release.aligned;\n\t"
      "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// The two halves of sync(), for work in between that touches nothing other
// threads read before the wait.
__device__ __forceinline__ void arrive() {
  __syncwarp();
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void wait() {
  __syncwarp();
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// The cluster-window address of byte `local` of CTA `rank`'s shared memory.
__device__ __forceinline__ uint32_t map(uint32_t local, uint32_t rank) {
  uint32_t a;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"(local), "r"(rank));
  return a;
}
// Loads and stores are volatile, so they keep their order with the cluster
// barrier.
__device__ __forceinline__ double ld(uint32_t a) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ void st(uint32_t a, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(a), "d"(v) : "memory");
}
}  // namespace dsm

// Each thread's point of every pass, found once per launch: for the
// cluster's level index lr (level first + lr) and colour c, entry
// (8 lr + c) CT + t of the point table holds the coordinates of thread t's
// point, x | y << 10 | z << 20 (coordinates below 1024, checked by the host),
// or NO_POINT. A CTA updates the points of its own z-planes (so the pass
// writes only its own shared memory), one per thread: those of colour c are
// a run [k0, k1) of the colour's points, at most CT long (checked by the
// host). Entry 8 lr + c of the pass table holds the run's first value offset
// (the colour block's start plus k0) and n_c.
constexpr uint32_t NO_POINT = 0x80000000u;

struct PassInfo {
  uint32_t kbase, n;
};

struct ClusterTables {
  const uint32_t* pt;    // the point table
  const PassInfo* info;  // the pass table
  __device__ __forceinline__ uint32_t point(int lr, int c) const {
    return pt[(lr * 8 + c) * CT + threadIdx.x];
  }
};

__device__ __forceinline__ void unpack(uint32_t p, uint32_t& x, uint32_t& y, uint32_t& z) {
  x = p & 1023u;
  y = (p >> 10) & 1023u;
  z = (p >> 20) & 1023u;
}

// A point's stencil neighbourhood in a level's distributed arrays, with each
// coordinate clamped to the grid (where a neighbour is outside the grid its
// value is 0: which point is read there does not change the sum). Byte
// addresses in the cluster window: pr[dz + 1][dy + 1] is the start of row
// y + dy of plane z + dz of the z array, in the CTA holding that plane, and
// col[dx + 1] the offset of column x + dx. The r array sits at the same
// offsets plus (r - z).
struct Hood {
  uint32_t pr[3][3], col[3];
  __device__ __forceinline__ Hood(const ClusterLevel& L, uint32_t base, uint32_t x, uint32_t y,
                                  uint32_t z) {
    const uint32_t nx = L.nx, ny = L.ny, nz = L.nz, pmask = (1u << L.lp) - 1;
    const uint32_t pb = nx * ny * 8;
    col[0] = (x > 0 ? x - 1 : 0) * 8;
    col[1] = x * 8;
    col[2] = min(x + 1, nx - 1) * 8;
    const uint32_t row[3] = {(y > 0 ? y - 1 : 0) * nx * 8, y * nx * 8, min(y + 1, ny - 1) * nx * 8};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const uint32_t zq = q == 0 ? (z > 0 ? z - 1 : 0) : (q == 1 ? z : min(z + 1, nz - 1));
      const uint32_t plane = dsm::map(base + L.z + (zq & pmask) * pb, zq >> L.lp);
#pragma unroll
      for (int a = 0; a < 3; ++a) pr[q][a] = plane + row[a];
    }
  }
  template <int ND>
  __device__ __forceinline__ uint32_t at(int d) const {
    return pr[slot_dz(ND, d) + 1][slot_dy(ND, d) + 1] + col[slot_dx(ND, d) + 1];
  }
};

// Shared-memory address of point (x, y, z), one of this CTA's own, in the
// slice at byte `off`.
__device__ __forceinline__ uint32_t own_at(const ClusterLevel& L, uint32_t base, uint32_t off,
                                           uint32_t x, uint32_t y, uint32_t z) {
  return base + off + (((z & ((1u << L.lp) - 1)) * (uint32_t)L.ny + y) * (uint32_t)L.nx + x) * 8;
}

// Address of point (x, y, z) of the distributed array at byte `off`.
__device__ __forceinline__ uint32_t cluster_at(const ClusterLevel& L, uint32_t base, uint32_t off,
                                               uint32_t x, uint32_t y, uint32_t z) {
  const uint32_t local =
      base + off + (((z & ((1u << L.lp) - 1)) * (uint32_t)L.ny + y) * (uint32_t)L.nx + x) * 8;
  return dsm::map(local, z >> L.lp);
}

// The values of a pass do not depend on z: while a pass computes, each
// thread copies the values of its point of the next pass into its own slots
// of a shared-memory buffer (slot d of thread t at d CT + t), with
// asynchronous copies that it waits for itself before that pass. Two buffers
// alternate.
__device__ __forceinline__ void cp_async8(uint32_t dst, const double* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(PENDING) : "memory");
}

template <int ND, uint32_t LIVE>
__device__ __forceinline__ void prefetch_pass(const ClusterLevel& L, uint32_t buf,
                                              const ClusterTables& T, int lr, int colour) {
  constexpr int D0 = ND / 2;
  if (!(T.point(lr, colour) & NO_POINT)) {
    const PassInfo pi = T.info[lr * 8 + colour];
    const double* vc = L.valc + pi.kbase + threadIdx.x;
#pragma unroll
    for (int d = 0; d < ND; ++d)
      if (d == D0 || ((LIVE >> d) & 1)) cp_async8(buf + (d * CT + threadIdx.x) * 8, vc + d * pi.n);
  }
  cp_async_commit();
}

// One colour pass of level L: z_i = (r_i - sum_{j != i} a_ij z_j) / a_ii,
// the slots outside LIVE skipped; the values from the thread's slots of the
// buffer vb.
template <int ND, uint32_t LIVE>
__device__ __forceinline__ void cluster_pass(const ClusterLevel& L, uint32_t base, const double* vb,
                                             const ClusterTables& T, int lr, int colour) {
  constexpr int D0 = ND / 2;
  const uint32_t p = T.point(lr, colour);
  if (p & NO_POINT) return;
  double v[ND], zz[ND];
#pragma unroll
  for (int d = 0; d < ND; ++d)
    if (d == D0 || ((LIVE >> d) & 1)) v[d] = vb[d * CT + threadIdx.x];
  uint32_t x, y, z;
  unpack(p, x, y, z);
  const Hood h(L, base, x, y, z);
#pragma unroll
  for (int d = 0; d < ND; ++d)
    if (d != D0 && ((LIVE >> d) & 1)) zz[d] = dsm::ld(h.at<ND>(d));
  double* zs = reinterpret_cast<double*>(__cvta_shared_to_generic(own_at(L, base, L.z, x, y, z)));
  double acc = zs[(L.r - L.z) / 8];  // r_i, from the r slice
#pragma unroll
  for (int d = 0; d < ND; ++d)
    if (d != D0 && ((LIVE >> d) & 1)) acc = fma(-v[d], zz[d], acc);
  *zs = acc * v[D0];
}

// The pass (or its prefetch) of a step of a sweep, with its slot set fixed at
// compile time: all slots, or a zero-start forward pass's.
template <int ND, bool PREFETCH>
__device__ __forceinline__ void sweep_step(const ClusterLevel& L, uint32_t base, uint32_t buf,
                                           const ClusterTables& T, int lr, int step, bool zero) {
  constexpr uint32_t ALL = (1u << ND) - 1;
  const int colour = step < 8 ? step : 14 - step;
  const double* vb = reinterpret_cast<const double*>(__cvta_shared_to_generic(buf));
#define DM_STEP(MASK)                                              \
  do {                                                             \
    if constexpr (PREFETCH)                                        \
      prefetch_pass<ND, (MASK)>(L, buf, T, lr, colour);            \
    else                                                           \
      cluster_pass<ND, (MASK)>(L, base, vb, T, lr, colour);        \
  } while (0)
  if (!(zero && step < 8)) {
    DM_STEP(ALL);
    return;
  }
  switch (colour) {
    case 0: DM_STEP(live_slots(ND, 0, true)); break;
    case 1: DM_STEP(live_slots(ND, 1, true)); break;
    case 2: DM_STEP(live_slots(ND, 2, true)); break;
    case 3: DM_STEP(live_slots(ND, 3, true)); break;
    case 4: DM_STEP(live_slots(ND, 4, true)); break;
    case 5: DM_STEP(live_slots(ND, 5, true)); break;
    case 6: DM_STEP(live_slots(ND, 6, true)); break;
    default: DM_STEP(live_slots(ND, 7, true)); break;
  }
#undef DM_STEP
}

// vbuf: byte offset of the two value buffers (ND x CT doubles each). The
// copies run two passes ahead: after pass s has read buffer s & 1 and
// arrived at the cluster barrier, the thread starts the copies for pass
// s + 2 into that buffer (its own slots), then waits at the barrier. Every
// step commits one copy group, so waiting for all but the latest group
// leaves the current pass's values complete.
template <int ND>
__device__ __forceinline__ void cluster_sweep(const ClusterLevel& L, uint32_t base, uint32_t vbuf,
                                              const ClusterTables& T, int lr, bool zero) {
  constexpr uint32_t BUF = ND * CT * 8;
  sweep_step<ND, true>(L, base, base + vbuf, T, lr, 0, zero);
  sweep_step<ND, true>(L, base, base + vbuf + BUF, T, lr, 1, zero);
  for (int step = 0; step < 15; ++step) {
    cp_async_wait<1>();
    sweep_step<ND, false>(L, base, base + vbuf + (step & 1) * BUF, T, lr, step, zero);
    dsm::arrive();
    if (step + 2 < 15)
      sweep_step<ND, true>(L, base, base + vbuf + (step & 1) * BUF, T, lr, step + 2, zero);
    else
      cp_async_commit();
    dsm::wait();
  }
  cp_async_wait<0>();
}

// Level C's right-hand side: (r - A z) of level F at its coarse points (the
// points of colour 7, F's level index lr).
template <int ND>
__device__ __forceinline__ void cluster_restrict(const ClusterLevel& F, const ClusterLevel& C,
                                                 uint32_t base, const ClusterTables& T, int lr) {
  constexpr int D0 = ND / 2;
  const uint32_t p = T.point(lr, 7);
  if (p & NO_POINT) return;
  uint32_t x, y, z;
  unpack(p, x, y, z);
  const PassInfo pi = T.info[lr * 8 + 7];
  const double* vc = F.valc + pi.kbase + threadIdx.x;
  const int64_t i = (int64_t)x + (int64_t)F.nx * ((int64_t)y + (int64_t)F.ny * z);
  double v[ND], zz[ND];
#pragma unroll
  for (int d = 0; d < ND; ++d) v[d] = d == D0 ? __ldg(F.diag + i) : __ldg(vc + d * pi.n);
  const Hood h(F, base, x, y, z);
#pragma unroll
  for (int d = 0; d < ND; ++d) zz[d] = dsm::ld(h.at<ND>(d));
  double acc = 0.0;
#pragma unroll
  for (int d = 0; d < ND; ++d) acc = fma(v[d], zz[d], acc);
  const double rf =
      *reinterpret_cast<const double*>(__cvta_shared_to_generic(own_at(F, base, F.r, x, y, z)));
  dsm::st(cluster_at(C, base, C.r, x >> 1, y >> 1, z >> 1), rf - acc);
}

// z_F += z_C at the coarse points of level F (level index lr).
__device__ __forceinline__ void cluster_prolong(const ClusterLevel& F, const ClusterLevel& C,
                                                uint32_t base, const ClusterTables& T, int lr) {
  const uint32_t p = T.point(lr, 7);
  if (p & NO_POINT) return;
  uint32_t x, y, z;
  unpack(p, x, y, z);
  double* zf = reinterpret_cast<double*>(__cvta_shared_to_generic(own_at(F, base, F.z, x, y, z)));
  *zf = *zf + dsm::ld(cluster_at(C, base, C.z, x >> 1, y >> 1, z >> 1));
}

// Levels first..levels-1 of a V-cycle: z = 0, level first's right-hand side
// from global memory, per level the zero-start sweep and the next level's
// right-hand side, then back up (prolongation and post-smoothing), and level
// first's solution to global memory. CTA q's slice of a level is its points
// [q slice, (q + 1) slice).
template <int ND>
__global__ void __launch_bounds__(CT, 1)
cluster_cycle_kernel(ClusterPlan P, const int32_t* __restrict__ skip) {
  if (skip && *skip) return;  // the same for every CTA
  extern __shared__ __align__(16) unsigned char cl_smem[];
  const uint32_t base = (uint32_t)__cvta_generic_to_shared(cl_smem);
  double* sm = reinterpret_cast<double*>(cl_smem);
  const uint32_t rk = dsm::rank();
  uint32_t* pt = reinterpret_cast<uint32_t*>(cl_smem + P.pts);
  PassInfo* info = reinterpret_cast<PassInfo*>(cl_smem + P.info);
  const ClusterTables T{pt, info};
  for (int l = P.first; l < P.levels; ++l) {
    const ClusterLevel& L = P.L[l];
    const int lr = l - P.first;
    for (uint32_t o = threadIdx.x; o < L.slice; o += CT) sm[L.z / 8 + o] = 0.0;
    for (int c = 0; c < 8; ++c) {
      const ColourGrid g(L.nx, L.ny, L.nz, 7 - c);
      const uint32_t n = (uint32_t)g.count(), plane = (uint32_t)(g.cx * g.cy);
      // the colour's half-grid planes h with 2 h + pz in this CTA's planes
      // [rk 2^lp, (rk + 1) 2^lp)
      const uint32_t z0 = rk << L.lp, z1 = (rk + 1) << L.lp, pz = (uint32_t)g.pz;
      const uint32_t h0 = min((uint32_t)g.cz, (z0 + 1 - pz) / 2);
      const uint32_t h1 = min((uint32_t)g.cz, (z1 + 1 - pz) / 2);
      const uint32_t k0 = h0 * plane, k = k0 + threadIdx.x;
      uint32_t packed = NO_POINT;
      if (k < h1 * plane) {
        uint32_t x, y, z;
        g.coords(k, x, y, z);
        packed = x | (y << 10) | (z << 20);
      }
      pt[(lr * 8 + c) * CT + threadIdx.x] = packed;
      if (threadIdx.x == 0) info[lr * 8 + c] = PassInfo{(uint32_t)colour_start(L, c) + k0, n};
    }
  }
  {
    const ClusterLevel& L = P.L[P.first];
    const int64_t N = (int64_t)L.nx * L.ny * L.nz;
    for (uint32_t o = threadIdx.x; o < L.slice; o += CT) {
      const int64_t i = (int64_t)rk * L.slice + o;
      sm[L.r / 8 + o] = i < N ? P.r_in[i] : 0.0;
    }
  }
  dsm::sync();
  for (int l = P.first; l < P.levels; ++l) {
    const int lr = l - P.first;
    cluster_sweep<ND>(P.L[l], base, P.vbuf, T, lr, true);
    if (l + 1 < P.levels) {
      cluster_restrict<ND>(P.L[l], P.L[l + 1], base, T, lr);
      dsm::sync();
    }
  }
  for (int l = P.levels - 2; l >= P.first; --l) {
    const int lr = l - P.first;
    cluster_prolong(P.L[l], P.L[l + 1], base, T, lr);
    dsm::sync();
    cluster_sweep<ND>(P.L[l], base, P.vbuf, T, lr, false);
  }
  {  // the last sweep ended with a cluster barrier: every z is in place
    const ClusterLevel& L = P.L[P.first];
    const int64_t N = (int64_t)L.nx * L.ny * L.nz;
    for (uint32_t o = threadIdx.x; o < L.slice; o += CT) {
      const int64_t i = (int64_t)rk * L.slice + o;
      if (i < N) P.z_out[i] = sm[L.z / 8 + o];
    }
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

MgLevel level_desc(const dynmat_mg_s* M, int l, const double* r, double* z) {
  MgLevel L{};
  const auto& d = M->dims[l];
  L.nx = d[0];
  L.ny = d[1];
  L.nz = d[2];
  L.offs = stencil_offsets(M, l);
  for (int c = 0; c < 8; ++c) L.cs.s[c] = M->cstart[l][c];
  L.valc = M->valc[l].as<double>();
  const dynmat_s* A = M->A[l];
  L.diag = A->dia.val.as<double>() + (int64_t)M->d0[l] * A->dia.ld;
  L.r = r;
  L.z = z;
  return L;
}

cudaLaunchConfig_t cooperative(unsigned grid, int bs, cudaStream_t s, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(bs);
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

// The barrier of launch site `site`: counts first (8 bytes per site), then
// the timeout flags (4 bytes per site).
GridBar site_bar(dynmat_mg_s* M, int site) {
  unsigned long long* counts = M->bar.as<unsigned long long>();
  unsigned* flags = reinterpret_cast<unsigned*>(counts + M->nbar);
  return GridBar{counts + site, flags + site};
}

// One symmetric sweep on level l; zero_start: z is 0 when it begins. reset:
// clear the site's barrier count first (a V-cycle clears every count once).
void symgs(dynmat_mg_s* M, int l, const double* r, double* z, const int32_t* skip,
           bool zero_start, bool reset, cudaStream_t s) {
  const auto& d = M->dims[l];
  // A colour of a coarse level is a few thousand points: blocks of 32 or 64
  // threads put it on more SMs (the FP64 pipe of each SM is narrow). The grid
  // stays within what is co-resident, which the cooperative launch checks.
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
  cudaLaunchAttribute attr[1];
  const cudaLaunchConfig_t cfg = cooperative(grid, bs, s, attr);
  MgLevel L = level_desc(M, l, r, z);
  const int site = 2 * l + (zero_start ? 1 : 0);
  GridBar bar = site_bar(M, site);
  if (reset) DM_CUDA(cudaMemsetAsync(bar.count, 0, sizeof(unsigned long long), s));
  void* args[] = {(void*)&L, (void*)&skip, (void*)&bar};
  DM_CUDA(cudaLaunchKernelExC(&cfg, fn, args));
}

// A cooperative launch of a coarse-cycle kernel over every SM (as many
// blocks per SM as are co-resident).
void launch_coarse(const void* fn, void** args, cudaStream_t s) {
  int per_sm = 0;
  DM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, T, 0));
  const unsigned grid = (unsigned)(std::max(per_sm, 1) * device().sms);
  cudaLaunchAttribute attr[1];
  const cudaLaunchConfig_t cfg = cooperative(grid, T, s, attr);
  DM_CUDA(cudaLaunchKernelExC(&cfg, fn, args));
}

const void* cluster_fn(int points) {
  return points == 27 ? (const void*)cluster_cycle_kernel<27> : (const void*)cluster_cycle_kernel<7>;
}

cudaLaunchConfig_t cluster_config(int ctas, size_t smem, cudaStream_t s, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(ctas);
  cfg.blockDim = dim3(CT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = ctas;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

constexpr size_t CLUSTER_SMEM = 200 * 1024;  // at most this much shared memory per CTA

// Picks the cluster of the coarse levels: 16 CTAs where the device
// schedules a cluster that large, else 8. Its first level is the first
// level l >= 1 whose colours have at most CT points in any CTA's planes and
// whose dimensions are below 1024 (the levels below it are smaller still),
// moved down while the cluster's shared memory would exceed CLUSTER_SMEM.
// None, or no such cluster schedulable: cl_ctas = 0.
void plan_cluster(dynmat_mg_s* M) {
  M->cl_ctas = 0;
  const void* fn = cluster_fn(M->points);
  for (int ctas : {16, 8}) {
    int first = M->levels;
    for (int l = M->levels - 1; l >= 1; --l) {
      const auto& d = M->dims[l];
      uint32_t k = 0;
      while (((int64_t)ctas << k) < d[2]) ++k;
      // a CTA's 2^k planes hold at most ceil(2^k / 2) planes of a colour
      int64_t most = 0;
      for (int c = 0; c < 8; ++c) {
        const ColourGrid g(d[0], d[1], d[2], c);
        most = std::max(most, g.cx * g.cy * ((((int64_t)1 << k) + 1) / 2));
      }
      if (most > CT || d[0] >= 1024 || d[1] >= 1024 || d[2] >= 1024) break;
      first = l;
    }
    for (; first < M->levels; ++first) {
      // per CTA: each level's z and r slices (2^lp whole z-planes, with
      // CTAs x 2^lp >= nz), the two value buffers, the point and pass tables
      std::vector<uint32_t> lp, zo, ro;
      size_t bytes = 0;
      for (int l = 0; l < M->levels; ++l) {
        uint32_t k = 0;
        const auto& d = M->dims[l];
        if (l >= first)
          while (((int64_t)ctas << k) < d[2]) ++k;
        const size_t slice = l >= first ? ((size_t)d[0] * d[1]) << k : 0;
        lp.push_back(k);
        zo.push_back((uint32_t)bytes);
        ro.push_back((uint32_t)(bytes + slice * 8));
        bytes += slice * 16;
      }
      const size_t nlev = (size_t)(M->levels - first);
      const size_t vbuf = (bytes + 15) / 16 * 16;
      const size_t pts = vbuf + (size_t)2 * M->points * CT * 8;
      const size_t info = pts + nlev * 8 * CT * 4;
      bytes = info + nlev * 8 * sizeof(PassInfo);
      if (bytes > CLUSTER_SMEM) continue;
      if (ctas > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                          cudaSuccess) {
        (void)cudaGetLastError();
        break;
      }
      // the kernel's limit, the same for every hierarchy (an attribute of the
      // function, not of the launch)
      if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)CLUSTER_SMEM) != cudaSuccess) {
        (void)cudaGetLastError();
        break;
      }
      cudaLaunchAttribute attr[1];
      const cudaLaunchConfig_t cfg = cluster_config(ctas, bytes, nullptr, attr);
      int fits = 0;
      if (cudaOccupancyMaxActiveClusters(&fits, fn, &cfg) != cudaSuccess || fits < 1) {
        (void)cudaGetLastError();
        break;
      }
      M->cl_ctas = ctas;
      M->cl_first = first;
      M->cl_smem = bytes;
      M->cl_vbuf = (uint32_t)vbuf;
      M->cl_pts = (uint32_t)pts;
      M->cl_info = (uint32_t)info;
      M->cl_lp = lp;
      M->cl_z = zo;
      M->cl_r = ro;
      return;
    }
  }
}

void vcycle(dynmat_mg_s* M, const double* r, double* z, const int32_t* skip, cudaStream_t s) {
  const auto& d = M->dims[0];
  // every launch of the V-cycle starts its barrier from a zero count, even
  // after an earlier launch gave up on a barrier
  DM_CUDA(cudaMemsetAsync(M->bar.p, 0, sizeof(unsigned long long) * M->nbar, s));
  DM_CUDA(cudaMemsetAsync(z, 0, d[0] * d[1] * d[2] * sizeof(double), s));
  symgs(M, 0, r, z, skip, true, false, s);
  if (M->levels == 1) return;
  MgPlan P{};
  P.levels = M->levels;
  P.L[0] = level_desc(M, 0, r, z);
  for (int l = 1; l < M->levels; ++l)
    P.L[l] = level_desc(M, l, M->r[l].as<double>(), M->z[l].as<double>());
  const bool p27 = M->points == 27;
  if (M->cl_ctas == 0) {
    GridBar bar = site_bar(M, 2 * M->levels);
    void* args[] = {(void*)&P, (void*)&skip, (void*)&bar};
    launch_coarse(p27 ? (const void*)coarse_cycle_kernel<27> : (const void*)coarse_cycle_kernel<7>,
                  args, s);
  } else {
    int lc = M->cl_first;
    GridBar down = site_bar(M, 2 * M->levels + 1), up = site_bar(M, 2 * M->levels + 2);
    void* dargs[] = {(void*)&P, (void*)&lc, (void*)&skip, (void*)&down};
    launch_coarse(p27 ? (const void*)coarse_down_kernel<27> : (const void*)coarse_down_kernel<7>,
                  dargs, s);
    ClusterPlan C{};
    C.first = lc;
    C.levels = M->levels;
    C.ctas = M->cl_ctas;
    C.vbuf = M->cl_vbuf;
    C.pts = M->cl_pts;
    C.info = M->cl_info;
    for (int l = lc; l < M->levels; ++l) {
      ClusterLevel& Q = C.L[l];
      const MgLevel& G = P.L[l];
      Q.nx = (int32_t)G.nx;
      Q.ny = (int32_t)G.ny;
      Q.nz = (int32_t)G.nz;
      Q.lp = M->cl_lp[l];
      Q.slice = (uint32_t)(G.nx * G.ny) << Q.lp;
      Q.z = M->cl_z[l];
      Q.r = M->cl_r[l];
      Q.cs = G.cs;
      Q.valc = G.valc;
      Q.diag = G.diag;
    }
    C.r_in = P.L[lc].r;
    C.z_out = P.L[lc].z;
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t cfg = cluster_config(M->cl_ctas, M->cl_smem, s, attr);
    void* cargs[] = {(void*)&C, (void*)&skip};
    DM_CUDA(cudaLaunchKernelExC(&cfg, cluster_fn(M->points), cargs));
    void* uargs[] = {(void*)&P, (void*)&lc, (void*)&skip, (void*)&up};
    launch_coarse(p27 ? (const void*)coarse_up_kernel<27> : (const void*)coarse_up_kernel<7>, uargs,
                  s);
  }
  symgs(M, 0, r, z, skip, false, false, s);
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
  vcycle(M, r, z, skip, s);
}

const dynmat_s* mg_matrix(const dynmat_mg_s* M) { return M->A[0]; }

// Blocking: DYNMAT_ERR_TIMEOUT (and a reset barrier) if a smoother's grid
// barrier timed out since the last check.
void mg_check_timeout(dynmat_mg_s* M, cudaStream_t s) {
  std::vector<unsigned> h((size_t)M->nbar, 0u);
  DM_CUDA(cudaMemcpyAsync(h.data(), site_bar(M, 0).timeout, h.size() * sizeof(unsigned),
                          cudaMemcpyDeviceToHost, s));
  DM_CUDA(cudaStreamSynchronize(s));
  bool timed_out = false;
  for (int k = 0; k < M->nbar; ++k) timed_out = timed_out || h[k] != 0;
  if (timed_out) {  // clear the flags (the counts are cleared before each launch)
    DM_CUDA(cudaMemsetAsync(site_bar(M, 0).timeout, 0, sizeof(unsigned) * M->nbar, s));
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
    DM_REQUIRE(nx * ny * nz < (1ll << 31), DYNMAT_ERR_INVALID_ARG,
               "grid %lld x %lld x %lld: at most 2^31 - 1 points", (long long)nx, (long long)ny,
               (long long)nz);
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
    // sweeps per (level, zero start), then the coarse cycle, its descent and
    // its ascent
    M->nbar = 2 * levels + 3;
    M->bar.alloc((size_t)12 * M->nbar, s);
    DM_CUDA(cudaMemsetAsync(M->bar.p, 0, (size_t)12 * M->nbar, s));
    DM_CUDA(cudaStreamSynchronize(s));
    plan_cluster(M.get());
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
    symgs(M, level, r, z, nullptr, false, true, (cudaStream_t)stream);
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
