// Integer primitives used by create and the conversions: exclusive scan,
// stable LSD radix sort of 64-bit keys, max-reduction. All results are
// deterministic (integer arithmetic, fixed partitioning).
#include "internal.cuh"

namespace dm {

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ int32_t warp_incl_scan(int32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int32_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Exclusive block scan of one value per thread; returns the thread's prefix
// and writes the block total to *total.
__device__ int32_t block_excl_scan(int32_t v, int32_t* total) {
  __shared__ int32_t warp_sums[SCAN_THREADS / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int32_t inc = warp_incl_scan(v);
  if (lane == 31) warp_sums[w] = inc;
  __syncthreads();
  if (w == 0) {
    int32_t s = lane < SCAN_THREADS / 32 ? warp_sums[lane] : 0;
    int32_t si = warp_incl_scan(s);
    if (lane < SCAN_THREADS / 32) warp_sums[lane] = si - s;
    if (lane == SCAN_THREADS / 32 - 1) *total = si;
  }
  __syncthreads();
  int32_t r = inc - v + warp_sums[w];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(SCAN_THREADS)
scan_local_kernel(const int32_t* __restrict__ in, int32_t* __restrict__ out, int64_t n,
                  int32_t* __restrict__ block_sums) {
  __shared__ int32_t total;
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  int32_t v[SCAN_ITEMS];
  int32_t s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    int64_t i = base + k;
    v[k] = i < n ? in[i] : 0;
    s += v[k];
  }
  int32_t pre = block_excl_scan(s, &total);
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    int64_t i = base + k;
    if (i < n) out[i] = pre;
    pre += v[k];
  }
  if (threadIdx.x == 0 && block_sums) block_sums[blockIdx.x] = total;
}

__global__ void scan_add_kernel(int32_t* __restrict__ out, int64_t n,
                                const int32_t* __restrict__ offs) {
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  const int32_t o = offs[blockIdx.x];
  for (int k = threadIdx.x; k < SCAN_TILE; k += blockDim.x) {
    int64_t i = base + k;
    if (i < n) out[i] += o;
  }
}

__global__ void max_kernel(const int32_t* __restrict__ in, int64_t n, int32_t* __restrict__ res) {
  int32_t m = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    m = max(m, in[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(res, m);
}

// ---------------------------------------------------------------------------
// Radix sort: 8-bit digits, tiles of 4096 keys per block (staged in shared
// memory by the scatter).
// ---------------------------------------------------------------------------
constexpr int RS_THREADS = 256;
constexpr int RS_ROUNDS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;
constexpr int RS_WARPS = RS_THREADS / 32;

__global__ void __launch_bounds__(RS_THREADS)
rs_hist_kernel(const uint64_t* __restrict__ keys, int64_t n, int shift,
               int32_t* __restrict__ counts, int64_t nb) {
  __shared__ int32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int k = threadIdx.x; k < RS_TILE; k += RS_THREADS) {
    int64_t i = base + k;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255], 1);
  }
  __syncthreads();
  counts[(int64_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter of one tile. Warp w takes the tile's keys
// [w RS_PER_WARP, (w + 1) RS_PER_WARP), 16 per lane, all loaded at once into
// registers (their values are read when the keys are placed). In round q it ranks its 32 keys of round q (index order: round,
// then lane) by a warp match against its own running digit counts (no block
// barrier). One block-wide pass then turns the per-warp counts into each
// warp's first position per digit (digit-major, warps in order), and every
// key goes to shared memory at its warp's position plus its rank: the tile
// in digit order, stable. It then goes out in runs of equal digits (about
// 16 keys per run for 8-bit digits), each to consecutive positions of its
// digit's bucket: coalesced stores, where writing each key straight to its
// bucket scattered a warp's stores over up to 32 buckets. Dynamic shared
// memory: RS_TILE keys, then RS_TILE payloads (P: 4 or 8 bytes).
constexpr int RS_PER_WARP = RS_TILE / RS_WARPS;
constexpr int RS_KPL = RS_PER_WARP / 32;  // keys per lane

template <class P>
__global__ void __launch_bounds__(RS_THREADS, 3)  // 3 blocks per SM, as shared memory allows
rs_scatter_kernel(const uint64_t* __restrict__ kin, const P* __restrict__ vin,
                  uint64_t* __restrict__ kout, P* __restrict__ vout, int64_t n, int shift,
                  const int32_t* __restrict__ offsets, int64_t nb) {
  extern __shared__ __align__(16) unsigned char rs_smem[];
  uint64_t* sk = reinterpret_cast<uint64_t*>(rs_smem);
  P* sv = reinterpret_cast<P*>(sk + RS_TILE);
  __shared__ int32_t gbase[256];
  __shared__ int32_t toff[256];            // first tile position of each digit
  __shared__ int32_t wpos[RS_WARPS][256];  // per warp: its count, then its first position
  __shared__ int32_t unused_total;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  gbase[t] = offsets[(int64_t)t * nb + blockIdx.x];
#pragma unroll
  for (int k = 0; k < RS_WARPS; ++k) wpos[k][t] = 0;
  const unsigned lt_mask = (1u << lane) - 1u;
  // keys of this tile left from the warp's first one (<= 0: none)
  const int64_t left = n - ((int64_t)blockIdx.x * RS_TILE + (int64_t)w * RS_PER_WARP);
  const int wn = (int)(left < RS_PER_WARP ? (left > 0 ? left : 0) : RS_PER_WARP);
  const uint64_t* kw = kin + (int64_t)blockIdx.x * RS_TILE + w * RS_PER_WARP;
  const P* vw = vin + (int64_t)blockIdx.x * RS_TILE + w * RS_PER_WARP;
  uint64_t key[RS_KPL];
#pragma unroll
  for (int q = 0; q < RS_KPL; ++q) {
    const int j = 32 * q + lane;
    key[q] = j < wn ? kw[j] : 0;
  }
  __syncthreads();  // wpos cleared
  uint16_t rank[RS_KPL];
#pragma unroll
  for (int q = 0; q < RS_KPL; ++q) {
    const bool valid = 32 * q + lane < wn;
    const int d = valid ? (int)((key[q] >> shift) & 255) : 256;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int before = valid ? wpos[w][d] : 0;
    __syncwarp();
    if (valid && (peers & lt_mask) == 0) wpos[w][d] = before + __popc(peers);
    __syncwarp();
    rank[q] = (uint16_t)(before + __popc(peers & lt_mask));
  }
  __syncthreads();
  {  // thread t = digit t: the warps' first positions, after the earlier digits
    int32_t c[RS_WARPS], tot = 0;
#pragma unroll
    for (int k = 0; k < RS_WARPS; ++k) {
      c[k] = wpos[k][t];
      tot += c[k];
    }
    int32_t p = block_excl_scan(tot, &unused_total);
    toff[t] = p;
#pragma unroll
    for (int k = 0; k < RS_WARPS; ++k) {
      wpos[k][t] = p;
      p += c[k];
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < RS_KPL; ++q) {
    if (32 * q + lane < wn) {
      const int d = (int)((key[q] >> shift) & 255);
      const int pos = wpos[w][d] + rank[q];
      sk[pos] = key[q];
      sv[pos] = vw[32 * q + lane];  // the values are read only here
    }
  }
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
  const int tile_n = (int)(n - base < RS_TILE ? n - base : RS_TILE);
  for (int j = t; j < tile_n; j += RS_THREADS) {
    const uint64_t k = sk[j];
    const int d = (int)((k >> shift) & 255);
    const int64_t pos = (int64_t)gbase[d] + (j - toff[d]);
    kout[pos] = k;
    vout[pos] = sv[j];
  }
}

template <class P>
constexpr size_t rs_smem() { return (size_t)RS_TILE * (8 + sizeof(P)); }

}  // namespace

void exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, int64_t* total,
                        cudaStream_t s) {
  if (n <= 0) {
    if (total) *total = 0;
    return;
  }
  const int64_t nb = cdiv(n, SCAN_TILE);
  if (nb == 1) {
    scan_local_kernel<<<1, SCAN_THREADS, 0, s>>>(in, out, n, nullptr);
    DM_CHECK_LAUNCH();
  } else {
    DBuf sums((size_t)nb * 4, s), offs((size_t)nb * 4, s);
    scan_local_kernel<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, out, n, sums.as<int32_t>());
    DM_CHECK_LAUNCH();
    exclusive_scan_i32(sums.as<int32_t>(), offs.as<int32_t>(), nb, nullptr, s);
    scan_add_kernel<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(out, n, offs.as<int32_t>());
    DM_CHECK_LAUNCH();
  }
  if (total) {
    int32_t a = 0, b = 0;
    DM_CUDA(cudaMemcpyAsync(&a, out + (n - 1), 4, cudaMemcpyDeviceToHost, s));
    DM_CUDA(cudaMemcpyAsync(&b, in + (n - 1), 4, cudaMemcpyDeviceToHost, s));
    DM_CUDA(cudaStreamSynchronize(s));
    *total = (int64_t)a + b;
  }
}

int64_t reduce_max_i32(const int32_t* in, int64_t n, cudaStream_t s) {
  if (n <= 0) return 0;
  DBuf r(4, s);
  DM_CUDA(cudaMemsetAsync(r.p, 0, 4, s));
  int blocks = (int)std::min<int64_t>(cdiv(n, 256), (int64_t)device().sms * 8);
  max_kernel<<<blocks, 256, 0, s>>>(in, n, r.as<int32_t>());
  DM_CHECK_LAUNCH();
  int32_t h = 0;
  DM_CUDA(cudaMemcpyAsync(&h, r.p, 4, cudaMemcpyDeviceToHost, s));
  DM_CUDA(cudaStreamSynchronize(s));
  return h;
}

namespace {

template <class P>
void radix_sort_keys(uint64_t* keys, P* vals, int64_t n, int bits, cudaStream_t s) {
  if (n <= 1 || bits <= 0) return;
  constexpr size_t RS_SMEM = rs_smem<P>();
  const int64_t nb = cdiv(n, RS_TILE);
  // the staged tile is over the default 48 KB (an attribute of the function
  // on the current device)
  DM_CUDA(cudaFuncSetAttribute(rs_scatter_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)RS_SMEM));
  DBuf k2((size_t)n * 8, s), v2((size_t)n * sizeof(P), s);
  DBuf counts((size_t)nb * 256 * 4, s), offs((size_t)nb * 256 * 4, s);
  uint64_t *ka = keys, *kb = k2.as<uint64_t>();
  P *va = vals, *vb = v2.as<P>();
  const int passes = (bits + 7) / 8;
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    rs_hist_kernel<<<(unsigned)nb, RS_THREADS, 0, s>>>(ka, n, shift, counts.as<int32_t>(), nb);
    DM_CHECK_LAUNCH();
    exclusive_scan_i32(counts.as<int32_t>(), offs.as<int32_t>(), nb * 256, nullptr, s);
    rs_scatter_kernel<P><<<(unsigned)nb, RS_THREADS, RS_SMEM, s>>>(ka, va, kb, vb, n, shift,
                                                                   offs.as<int32_t>(), nb);
    DM_CHECK_LAUNCH();
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (ka != keys) {
    DM_CUDA(cudaMemcpyAsync(keys, ka, (size_t)n * 8, cudaMemcpyDeviceToDevice, s));
    DM_CUDA(cudaMemcpyAsync(vals, va, (size_t)n * sizeof(P), cudaMemcpyDeviceToDevice, s));
  }
  // Temporaries are freed stream-ordered; the copies above precede the frees.
}

}  // namespace

void radix_sort_u64(uint64_t* keys, int32_t* vals, int64_t n, int bits, cudaStream_t s) {
  radix_sort_keys(keys, vals, n, bits, s);
}
void radix_sort_u64(uint64_t* keys, uint64_t* vals, int64_t n, int bits, cudaStream_t s) {
  radix_sort_keys(keys, vals, n, bits, s);
}

}  // namespace dm
