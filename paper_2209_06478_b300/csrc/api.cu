// The C ABI of dynmat: errors, memory, create / destroy / inspect, the
// in-place format switch (§III-A activate, §III-B convert) and the SpMV
// entry points (§III-D multiply).
#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <memory>
#include <mutex>
#include <unordered_map>
#include <vector>

#include <sys/mman.h>

#include "device.cuh"
#include "internal.cuh"

namespace dm {

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------
static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}
void clear_error() { g_err[0] = 0; }

// ---------------------------------------------------------------------------
// Memory
// ---------------------------------------------------------------------------
static dynmat_alloc_fn g_alloc = nullptr;
static dynmat_free_fn g_free = nullptr;
static void* g_alloc_ctx = nullptr;
static std::atomic<int64_t> g_in_use{0};
static std::atomic<int64_t> g_limit{0};
double g_pad_limit = 16.0;
// host memory from dynmat_host_alloc: start -> mapped length
static std::mutex g_host_mu;
static std::unordered_map<void*, size_t> g_host;

// The library's own stream-ordered pool on each device, created on first
// use. Freed blocks stay cached in it (release threshold at the maximum),
// so the arrays of a format conversion (hundreds of MB at 128^3) are reused
// from one conversion to the next. The device's default pool returns
// memory at every synchronisation, and mapping it again cost milliseconds
// per conversion. The cache goes back to the device when a handle is
// destroyed, or when an allocation fails (then it is retried once). The byte
// cap and dynmat_memory_in_use count allocations, not cached bytes.
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64] = {};

static cudaMemPool_t device_pool() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pool[dev] = pool;
  }
  return g_pool[dev];
}

// Returns the pool's cached (free) memory to the device once the work on
// `s` has finished.
void trim_device_pool(cudaStream_t s) {
  if (g_alloc) return;
  cudaMemPool_t pool = device_pool();
  if (!pool) return;
  cudaStreamSynchronize(s);
  cudaMemPoolTrimTo(pool, 0);
}

static void* pool_alloc(size_t bytes, cudaStream_t s) {
  void* p = nullptr;
  cudaMemPool_t pool = device_pool();
  cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, bytes, pool, s) : cudaMallocAsync(&p, bytes, s);
  if (e == cudaSuccess) return p;
  cudaGetLastError();
  if (pool) {  // the cache may hold the memory: give it back and retry once
    trim_device_pool(s);
    if (cudaMallocFromPoolAsync(&p, bytes, pool, s) == cudaSuccess) return p;
    cudaGetLastError();
  }
  return nullptr;
}

void* dev_alloc(size_t bytes, cudaStream_t s) {
  const int64_t lim = g_limit.load();
  const int64_t now = g_in_use.fetch_add((int64_t)bytes) + (int64_t)bytes;
  if (lim > 0 && now > lim) {
    g_in_use.fetch_sub((int64_t)bytes);
    set_error("allocation of %zu bytes exceeds the memory limit (%lld of %lld bytes in use)",
              bytes, (long long)(now - (int64_t)bytes), (long long)lim);
    throw Fail{DYNMAT_ERR_OOM};
  }
  void* p = g_alloc ? g_alloc(bytes, (void*)s, g_alloc_ctx) : pool_alloc(bytes, s);
  if (!p) {
    g_in_use.fetch_sub((int64_t)bytes);
    set_error("device allocation of %zu bytes failed", bytes);
    throw Fail{DYNMAT_ERR_OOM};
  }
  return p;
}

void dev_free(void* p, size_t bytes, cudaStream_t s) {
  if (!p) return;
  if (g_alloc) {
    if (g_free) g_free(p, bytes, (void*)s, g_alloc_ctx);
  } else {
    cudaFreeAsync(p, s);
  }
  g_in_use.fetch_sub((int64_t)bytes);
}

const Dev& device() {
  static std::mutex mu;
  static Dev devs[64];
  int id = 0;
  if (cudaGetDevice(&id) != cudaSuccess) id = 0;
  if (id < 0 || id >= 64) id = 0;
  std::lock_guard<std::mutex> lk(mu);
  Dev& d = devs[id];
  if (d.id != id) {
    int sms = 0, l2 = 0;
    DM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, id));
    DM_CUDA(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, id));
    d.sms = sms;
    d.l2_bytes = l2;
    d.id = id;
  }
  return d;
}

int64_t handle_bytes(const dynmat_s* A) {
  int64_t b = 0;
  for (const DBuf* p : {&A->coo.row, &A->coo.col, &A->coo.val, &A->csr.rowptr, &A->csr.col,
                        &A->csr.val, &A->dia.offsets, &A->dia.val, &A->ell.col, &A->ell.val,
                        &A->seg.chunk_row, &A->seg.carry, &A->seg.unit_start, &A->stage_x,
                        &A->stage_y, &A->cg_work})
    b += (int64_t)p->bytes;
  if (A->shadow32) b += handle_bytes(A->shadow32);
  return b;
}

void free_format(dynmat_s* A, cudaStream_t s) {
  ++A->gen;
  for (DBuf* p : {&A->coo.row, &A->coo.col, &A->coo.val, &A->csr.rowptr, &A->csr.col,
                  &A->csr.val, &A->dia.offsets, &A->dia.val, &A->ell.col, &A->ell.val,
                  &A->seg.chunk_row, &A->seg.carry, &A->seg.unit_start}) {
    p->s = s;
    p->release();
  }
  A->coo.nnz = A->csr.nnz = 0;
  A->dia.ndiag = A->dia.ld = 0;
  A->ell.K = A->ell.ld = 0;
  A->seg.nchunks = 0;
}

void destroy_handle(dynmat_s* A, cudaStream_t s) {
  if (!A) return;
  if (A->shadow32) destroy_handle(A->shadow32, s);
  A->shadow32 = nullptr;
  free_format(A, s);
  for (DBuf* p : {&A->stage_x, &A->stage_y, &A->cg_work}) {
    p->s = s;
    p->release();
  }
  for (cudaStream_t& q : A->pipe_s)
    if (q) {
      cudaStreamSynchronize(q);
      cudaStreamDestroy(q);
      q = nullptr;
    }
  for (cudaEvent_t& e : A->pipe_ev)
    if (e) {
      cudaEventDestroy(e);
      e = nullptr;
    }
  delete A;
}

// ---------------------------------------------------------------------------
// Create: validate, sort by (row, col) when needed, reject duplicates.
// ---------------------------------------------------------------------------
namespace {

constexpr int T = 256;

enum : int { F_RANGE = 1, F_UNSORTED = 2, F_DUP = 4, F_INEXACT = 8 };

// Flags of one entry (r, c) and its successor (r2, c2) in the array:
// F_RANGE for an index outside the matrix; for two in-range entries,
// F_UNSORTED when (r2, c2) comes before (r, c) and F_DUP when they are equal
// (row-major order compared lexicographically, no 64-bit keys).
__device__ __forceinline__ int coo_pair_flags(int32_t r, int32_t c, int32_t r2, int32_t c2,
                                              bool has_next, int64_t nrows, int64_t ncols) {
  if (r < 0 || r >= nrows || c < 0 || c >= ncols) return F_RANGE;
  if (!has_next || r2 < 0 || r2 >= nrows || c2 < 0 || c2 >= ncols) return 0;
  if (r2 < r || (r2 == r && c2 < c)) return F_UNSORTED;
  return (r2 == r && c2 == c) ? F_DUP : 0;
}

// Range, order and duplicate check of a COO. VEC: four entries per thread
// from 16-byte loads of row and col (both 16-byte aligned; the arrays' tail
// padding covers the last group); the entry after a thread's four is the
// next lane's first, or a plain load for the last lane of the warp.
template <bool VEC>
__global__ void check_coo_kernel(const int32_t* __restrict__ row, const int32_t* __restrict__ col,
                                 int64_t nnz, int64_t nrows, int64_t ncols, int* __restrict__ flags) {
  int f = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (VEC) {
    const int lane = threadIdx.x & 31;
    const int64_t ng = (nnz + 3) / 4;
    // every lane of a warp runs the same number of passes (for the shuffles)
    const int64_t t0 = t - lane;
    for (int64_t g0 = t0; g0 < ng; g0 += stride) {
      const int64_t g = g0 + lane;
      int4 r = make_int4(0, 0, 0, 0), c = make_int4(0, 0, 0, 0);
      if (g < ng) {
        r = __ldcs(reinterpret_cast<const int4*>(row) + g);
        c = __ldcs(reinterpret_cast<const int4*>(col) + g);
      }
      int32_t rn = __shfl_down_sync(0xffffffffu, r.x, 1);
      int32_t cn = __shfl_down_sync(0xffffffffu, c.x, 1);
      const int64_t e = 4 * g;
      if (lane == 31 && e + 4 < nnz) {
        rn = row[e + 4];
        cn = col[e + 4];
      }
      if (g < ng) {
        f |= coo_pair_flags(r.x, c.x, r.y, c.y, e + 1 < nnz, nrows, ncols);
        if (e + 1 < nnz) f |= coo_pair_flags(r.y, c.y, r.z, c.z, e + 2 < nnz, nrows, ncols);
        if (e + 2 < nnz) f |= coo_pair_flags(r.z, c.z, r.w, c.w, e + 3 < nnz, nrows, ncols);
        if (e + 3 < nnz) f |= coo_pair_flags(r.w, c.w, rn, cn, e + 4 < nnz, nrows, ncols);
      }
    }
  } else {
    for (int64_t e = t; e < nnz; e += stride) {
      const bool nx = e + 1 < nnz;
      f |= coo_pair_flags(row[e], col[e], nx ? row[e + 1] : 0, nx ? col[e + 1] : 0, nx, nrows,
                          ncols);
    }
  }
  f = __reduce_or_sync(0xffffffffu, f);
  if ((threadIdx.x & 31) == 0 && f) atomicOr(flags, f);
}

// Sort keys (row << cbits) | col, cbits the bit width of ncols - 1: they
// order entries by (row, col) as row * ncols + col does, and unkey_kernel
// takes row and col back with a shift and a mask. (The division by ncols that
// the product form needs is an emulated 64-bit sequence: that kernel took
// 296 us at 55.7M entries, against 193 us with the shift.) The key can be one
// bit wider than the product's, one more radix pass where that crosses a
// multiple of 8 bits.
__global__ void make_keys_kernel(const int32_t* __restrict__ row, const int32_t* __restrict__ col,
                                 int64_t nnz, int cbits, uint64_t* __restrict__ key) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nnz) return;
  key[e] = ((uint64_t)row[e] << cbits) | (uint64_t)col[e];
}

// Sorted keys back to rows and columns; equal neighbours are duplicates.
__global__ void unkey_kernel(const uint64_t* __restrict__ key, int64_t nnz, int cbits,
                             int32_t* __restrict__ row, int32_t* __restrict__ col,
                             int* __restrict__ flags) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nnz) return;
  const uint64_t k = key[e];
  row[e] = (int32_t)(k >> cbits);
  col[e] = (int32_t)(k & ((1ull << cbits) - 1));
  if (e + 1 < nnz && key[e + 1] == k) atomicOr(flags, F_DUP);
}

// A value (NaN excepted) that FP32 does not hold exactly, decided on the
// bits: a conversion to float and back would take two instructions on the
// FP64 pipe, which on B300 retires 2 per clock per SM (the kernel ran at
// 0.16 of HBM that way). With E the unbiased exponent: zero and infinity
// are exact; E > 127 overflows; -126 <= E <= 127 is a normal float, exact
// when the 29 low fraction bits are zero; -149 <= E < -126 is a float
// subnormal, exact when the fraction bits below 2^-149 (the low -97 - E of
// them) are zero; smaller nonzero values are not exact.
__device__ __forceinline__ bool inexact_f32(double a) {
  const uint64_t u = (uint64_t)__double_as_longlong(a);
  const int e = (int)((u >> 52) & 0x7ff);
  const uint64_t frac = u & 0xfffffffffffffull;
  if (e == 0x7ff) return false;  // infinity is exact; NaN does not count
  if (e == 0) return frac != 0;  // zero exact; FP64 subnormals are below 2^-149
  const int E = e - 1023;
  if (E > 127) return true;
  if (E >= -126) return (frac & 0x1fffffffull) != 0;
  if (E >= -149) return (frac & ((1ull << (-97 - E)) - 1)) != 0;
  return true;
}

// Any value (NaN excepted) that FP32 does not hold exactly. 16-byte loads
// with two in flight per thread when v is 16-byte aligned.
__global__ void exact_f32_kernel(const double* __restrict__ v, int64_t n, int* __restrict__ flags) {
  bool bad = false;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t tail = 0;
  if (((uintptr_t)v & 15u) == 0) {
    const int64_t np = n / 2;
    const double2* v2 = reinterpret_cast<const double2*>(v);
    int64_t k = t;
    for (; k + stride < np; k += 2 * stride) {
      const double2 a = __ldcs(v2 + k), b = __ldcs(v2 + k + stride);
      bad |= inexact_f32(a.x) | inexact_f32(a.y) | inexact_f32(b.x) | inexact_f32(b.y);
    }
    for (; k < np; k += stride) {
      const double2 a = __ldcs(v2 + k);
      bad |= inexact_f32(a.x) | inexact_f32(a.y);
    }
    tail = 2 * np;
  }
  for (int64_t i = tail + t; i < n; i += stride) bad |= inexact_f32(v[i]);
  const int f = __reduce_or_sync(0xffffffffu, bad ? F_INEXACT : 0);
  if ((threadIdx.x & 31) == 0 && f) atomicOr(flags, f);
}

unsigned small_grid(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(n, T), (int64_t)device().sms * 16));
}

int read_flags(DBuf& f, cudaStream_t s) {
  int h = 0;
  DM_CUDA(cudaMemcpyAsync(&h, f.p, 4, cudaMemcpyDeviceToHost, s));
  DM_CUDA(cudaStreamSynchronize(s));
  return h;
}

}  // namespace

int values_exact_in_f32(const void* val, int64_t n, dynmat_dtype dt, cudaStream_t s) {
  if (dt == DYNMAT_F32 || n == 0) return 1;
  DBuf f(4, s);
  DM_CUDA(cudaMemsetAsync(f.p, 0, 4, s));
  exact_f32_kernel<<<small_grid(n), T, 0, s>>>((const double*)val, n, f.as<int>());
  DM_CHECK_LAUNCH();
  return (read_flags(f, s) & F_INEXACT) ? 0 : 1;
}

static void create_impl(dynmat_t* out, int64_t nrows, int64_t ncols, int64_t nnz,
                        const int32_t* row, const int32_t* col, const void* val,
                        dynmat_dtype vdt, int on_dev, cudaStream_t s) {
  DM_REQUIRE(out, DYNMAT_ERR_INVALID_ARG, "out is NULL");
  DM_REQUIRE(nrows >= 0 && ncols >= 0 && nnz >= 0, DYNMAT_ERR_INVALID_ARG,
             "negative size (nrows %lld, ncols %lld, nnz %lld)", (long long)nrows,
             (long long)ncols, (long long)nnz);
  DM_REQUIRE(nrows < INT32_MAX && ncols < INT32_MAX && nnz < INT32_MAX, DYNMAT_ERR_INVALID_ARG,
             "sizes must be below 2^31 - 1");
  DM_REQUIRE(vdt == DYNMAT_F64 || vdt == DYNMAT_F32, DYNMAT_ERR_INVALID_ARG, "bad value dtype");
  DM_REQUIRE(nnz == 0 || (row && col && val), DYNMAT_ERR_INVALID_ARG, "null input array");
  DM_REQUIRE(nnz == 0 || (nrows > 0 && ncols > 0), DYNMAT_ERR_INDEX_RANGE,
             "entries given for an empty matrix");
  device();
  const size_t vb = vsize(vdt);
  auto A = std::make_unique<dynmat_s>();
  A->nrows = nrows;
  A->ncols = ncols;
  A->vdt = vdt;
  A->fmt = DYNMAT_COO;
  Coo& C = A->coo;
  C.nnz = nnz;
  C.row.alloc(nnz * 4, s);
  C.col.alloc(nnz * 4, s);
  C.val.alloc(nnz * vb, s);
  if (nnz) {
    const cudaMemcpyKind k = on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    DM_CUDA(cudaMemcpyAsync(C.row.p, row, nnz * 4, k, s));
    DM_CUDA(cudaMemcpyAsync(C.col.p, col, nnz * 4, k, s));
    DM_CUDA(cudaMemcpyAsync(C.val.p, val, nnz * vb, k, s));
    DBuf flags(4, s);
    DM_CUDA(cudaMemsetAsync(flags.p, 0, 4, s));
    if (((uintptr_t)C.row.p | (uintptr_t)C.col.p) & 15u)
      check_coo_kernel<false><<<small_grid(nnz), T, 0, s>>>(
          C.row.as<int32_t>(), C.col.as<int32_t>(), nnz, nrows, ncols, flags.as<int>());
    else
      check_coo_kernel<true><<<small_grid(cdiv(nnz, 4)), T, 0, s>>>(
          C.row.as<int32_t>(), C.col.as<int32_t>(), nnz, nrows, ncols, flags.as<int>());
    DM_CHECK_LAUNCH();
    int f = read_flags(flags, s);
    DM_REQUIRE(!(f & F_RANGE), DYNMAT_ERR_INDEX_RANGE, "row or column index out of range");
    if (f & F_UNSORTED) {
      // The values travel with the keys as the sort's payload (raw 32- or
      // 64-bit words). Sorting a permutation instead and gathering the
      // values by it afterwards took 1.19 ms of random 8-byte reads at
      // 55.7M entries, more than the payload's extra bytes in the passes.
      DBuf key(nnz * 8, s);
      // bit widths of the largest row and column index (0 for one row or column)
      auto width = [](int64_t n) { return n > 1 ? 64 - __builtin_clzll((uint64_t)(n - 1)) : 0; };
      const int cbits = width(ncols), bits = std::max(1, width(nrows) + cbits);
      make_keys_kernel<<<(unsigned)cdiv(nnz, T), T, 0, s>>>(C.row.as<int32_t>(),
                                                              C.col.as<int32_t>(), nnz, cbits,
                                                              key.as<uint64_t>());
      DM_CHECK_LAUNCH();
      if (vb == 8)
        radix_sort_u64(key.as<uint64_t>(), C.val.as<uint64_t>(), nnz, bits, s);
      else
        radix_sort_u64(key.as<uint64_t>(), C.val.as<int32_t>(), nnz, bits, s);
      DM_CUDA(cudaMemsetAsync(flags.p, 0, 4, s));
      unkey_kernel<<<(unsigned)cdiv(nnz, T), T, 0, s>>>(key.as<uint64_t>(), nnz, cbits,
                                                        C.row.as<int32_t>(), C.col.as<int32_t>(),
                                                        flags.as<int>());
      DM_CHECK_LAUNCH();
      f = read_flags(flags, s);
    }
    DM_REQUIRE(!(f & F_DUP), DYNMAT_ERR_DUPLICATE, "two entries at the same (row, col)");
  }
  A->nnz = nnz;
  A->values_exact_f32 = values_exact_in_f32(C.val.p, nnz, vdt, s);
  prepare_spmv(A.get(), s);
  DM_CUDA(cudaStreamSynchronize(s));
  *out = A.release();
}

// Converts in place; on failure A is untouched.
void convert_impl(dynmat_s* A, dynmat_format fmt, dynmat_dtype vdt, cudaStream_t s) {
  DM_REQUIRE(A, DYNMAT_ERR_INVALID_ARG, "null handle");
  DM_REQUIRE(fmt >= DYNMAT_COO && fmt <= DYNMAT_HYB, DYNMAT_ERR_INVALID_ARG, "bad format %d",
             (int)fmt);
  DM_REQUIRE(vdt == DYNMAT_F64 || vdt == DYNMAT_F32, DYNMAT_ERR_INVALID_ARG, "bad value dtype");
  if (A->fmt == fmt && A->vdt == vdt) return;
  Coo tmp;
  const Coo* src = &A->coo;
  if (A->fmt != DYNMAT_COO) {
    to_coo(A, tmp, s);
    src = &tmp;
  }
  auto T2 = std::make_unique<dynmat_s>();
  T2->nrows = A->nrows;
  T2->ncols = A->ncols;
  T2->vdt = A->vdt;
  build_from_coo(T2.get(), *src, fmt, vdt, s);
  const int exact = (vdt == DYNMAT_F32 || A->vdt == DYNMAT_F32) ? 1 : A->values_exact_f32;
  free_format(A, s);
  A->coo = std::move(T2->coo);
  A->csr = std::move(T2->csr);
  A->dia = std::move(T2->dia);
  A->ell = std::move(T2->ell);
  A->fmt = fmt;
  A->vdt = vdt;
  A->nnz = T2->nnz;
  A->values_exact_f32 = exact;
  A->plan.forced = 0;
  if (A->shadow32) {
    destroy_handle(A->shadow32, s);
    A->shadow32 = nullptr;
  }
  A->cg_work.s = s;
  A->cg_work.release();
  A->cg_work_bytes = 0;
  prepare_spmv(A, s);
  DM_CUDA(cudaStreamSynchronize(s));
}

}  // namespace dm

namespace dm {
namespace {
// dynmat_spmv_host for tile-based kernels (DIA, ELL, HYB without overflow,
// CSR variants 1-5, 7 and 8, COO variant 2), pipelined: x goes up in pieces on one
// stream; the product runs in as many row chunks, alternating between two
// streams, each chunk waiting only for the pieces of x its rows read (for DIA
// up to its last row + the largest offset, for the others up to the largest
// column stored in its rows); each chunk's y comes down on a fourth stream as soon
// as it is done. The upload of x, the products and the download of y overlap
// (the host link carries both directions at once). About 4 MiB of x and y
// per piece, 2 to PIPE_MAX pieces. (Chunks in one-pass tiles, with twice the
// blocks, and 2 MiB pieces both measured slower.)
constexpr size_t PIPE_PIECE_BYTES = (size_t)4 << 20;

// out[c] = the largest column stored in ELL rows [c * chunk_rows, (c + 1) *
// chunk_rows), for c < gridDim.x (out zeroed by the caller; padding is -1).
// Block (c, b) takes rows of chunk c with stride gridDim.y * blockDim.x.
__global__ void ell_chunk_maxcol_kernel(const int32_t* __restrict__ col, int64_t K, int64_t ld,
                                        int64_t N, int64_t chunk_rows, int32_t* __restrict__ out) {
  const int64_t r0 = blockIdx.x * chunk_rows, r1 = min(N, r0 + chunk_rows);
  int32_t m = -1;
  for (int64_t i = r0 + (int64_t)blockIdx.y * blockDim.x + threadIdx.x; i < r1;
       i += (int64_t)gridDim.y * blockDim.x)
    for (int64_t k = 0; k < K; ++k) m = max(m, __ldcs(col + k * ld + i));
  for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ int32_t wm[32];
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = max(m, wm[w]);
    atomicMax(out + blockIdx.x, m);
  }
}

// out[c] = the largest column among entries [e[c], e[c + 1]) of col (out
// zeroed by the caller), for c < gridDim.x: the row chunks of a CSR or COO
// matrix are contiguous entry ranges. Block (c, b) strides its chunk.
struct EntryBounds {
  int64_t e[PIPE_MAX + 1];
};
__global__ void range_maxcol_kernel(const int32_t* __restrict__ col,
                                    const __grid_constant__ EntryBounds eb,
                                    int32_t* __restrict__ out) {
  const int64_t e1 = eb.e[blockIdx.x + 1];
  int32_t m = -1;
  for (int64_t e = eb.e[blockIdx.x] + (int64_t)blockIdx.y * blockDim.x + threadIdx.x; e < e1;
       e += (int64_t)gridDim.y * blockDim.x)
    m = max(m, __ldcs(col + e));
  for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ int32_t wm[32];
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = max(m, wm[w]);
    atomicMax(out + blockIdx.x, m);
  }
}

struct PipeShape {
  int n = 0;       // pieces of x = row chunks = pieces of y
  int64_t xc = 0;  // x elements per piece
  int64_t tc = 0;  // plan tiles per row chunk
};

PipeShape pipe_shape(const dynmat_s* A, size_t vb) {
  PipeShape sh;
  const Plan& P = A->plan;
  const int64_t N = A->nrows, M = A->ncols;
  const size_t bytes = (size_t)(N + M) * vb;
  if (!has_row_ranges(A)) return sh;
  if (bytes < 2 * PIPE_PIECE_BYTES || M == 0) return sh;
  int n = (int)std::min<size_t>(PIPE_MAX, bytes / PIPE_PIECE_BYTES);
  n = (int)std::min<int64_t>(n, P.ntiles / 2);
  if (n < 2) return sh;
  sh.n = n;
  sh.xc = round_up(cdiv(M, n), 32);
  sh.tc = cdiv(P.ntiles, n);
  return sh;
}

// The x piece each row chunk waits for (the piece of its last x read).
void pipe_needs(dynmat_s* A, const PipeShape& sh, int32_t* need, cudaStream_t s) {
  const Plan& P = A->plan;
  const int64_t N = A->nrows, M = A->ncols;
  if (A->fmt == DYNMAT_DIA) {
    const int64_t reach = std::max<int64_t>(A->dia.off_max, 0);
    for (int c = 0; c < sh.n; ++c) {
      const int64_t r1 = std::min<int64_t>(N, std::min<int64_t>(P.ntiles, (c + 1) * sh.tc) *
                                                  P.tile_rows);
      need[c] = (int32_t)(std::max<int64_t>(0, std::min<int64_t>(M - 1, r1 - 1 + reach)) / sh.xc);
    }
    return;
  }
  if (A->pipe_need_gen != A->gen || A->pipe_need_n != sh.n) {  // measured once per plan
    DBuf m((size_t)sh.n * 4, s);
    DM_CUDA(cudaMemsetAsync(m.p, 0, (size_t)sh.n * 4, s));
    const int64_t chunk_rows = sh.tc * P.tile_rows;
    const unsigned slices = (unsigned)std::max<int64_t>(1, std::min<int64_t>(64, cdiv(chunk_rows, 256)));
    if (A->fmt == DYNMAT_ELL || A->fmt == DYNMAT_HYB) {
      ell_chunk_maxcol_kernel<<<dim3((unsigned)sh.n, slices), 256, 0, s>>>(
          A->ell.col.as<int32_t>(), A->ell.K, A->ell.ld, N, chunk_rows, m.as<int32_t>());
    } else {
      // CSR: the row pointer at each chunk boundary; COO (stream plan): the
      // first entry of the boundary's base of rows (a tile is one base)
      const int32_t* ptr = A->fmt == DYNMAT_CSR ? A->csr.rowptr.as<int32_t>()
                                                : A->seg.unit_start.as<int32_t>();
      int32_t at[PIPE_MAX + 1];
      for (int c = 0; c <= sh.n; ++c) {
        const int64_t t = std::min<int64_t>(P.ntiles, c * sh.tc);
        const int64_t k = A->fmt == DYNMAT_CSR ? std::min<int64_t>(N, t * P.tile_rows) : t;
        DM_CUDA(cudaMemcpyAsync(at + c, ptr + k, 4, cudaMemcpyDeviceToHost, s));
      }
      DM_CUDA(cudaStreamSynchronize(s));
      EntryBounds eb;
      for (int c = 0; c <= sh.n; ++c) eb.e[c] = at[c];
      const int32_t* col = A->fmt == DYNMAT_CSR ? A->csr.col.as<int32_t>() : A->coo.col.as<int32_t>();
      range_maxcol_kernel<<<dim3((unsigned)sh.n, slices), 256, 0, s>>>(col, eb, m.as<int32_t>());
    }
    DM_CHECK_LAUNCH();
    int32_t maxcol[PIPE_MAX];
    DM_CUDA(cudaMemcpyAsync(maxcol, m.p, (size_t)sh.n * 4, cudaMemcpyDeviceToHost, s));
    DM_CUDA(cudaStreamSynchronize(s));
    for (int c = 0; c < sh.n; ++c)
      A->pipe_need[c] = (int32_t)(std::min<int64_t>(M - 1, std::max(0, maxcol[c])) / sh.xc);
    A->pipe_need_gen = A->gen;
    A->pipe_need_n = sh.n;
  }
  for (int c = 0; c < sh.n; ++c) need[c] = A->pipe_need[c];
}

// Returns false when the pipeline does not apply (the caller then copies,
// multiplies and copies back on s). Blocking.
bool spmv_host_pipelined(dynmat_s* A, const void* x_host, void* y_host, dynmat_dtype vdt,
                         cudaStream_t s) {
  const size_t vb = vsize(vdt);
  const PipeShape sh = pipe_shape(A, vb);
  if (sh.n == 0) return false;
  for (cudaStream_t& q : A->pipe_s)
    if (!q) DM_CUDA(cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking));
  for (cudaEvent_t& e : A->pipe_ev)
    if (!e) DM_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  int32_t need[PIPE_MAX];
  pipe_needs(A, sh, need, s);
  const Plan& P = A->plan;
  const int64_t N = A->nrows, M = A->ncols;
  cudaStream_t s_in = A->pipe_s[0], s_out = A->pipe_s[3];
  cudaStream_t s_cmp[2] = {A->pipe_s[1], A->pipe_s[2]};
  cudaEvent_t* ex = A->pipe_ev;                 // x piece j uploaded
  cudaEvent_t* ec = A->pipe_ev + PIPE_MAX;      // row chunk c computed
  cudaEvent_t entry = A->pipe_ev[2 * PIPE_MAX];
  // after whatever the caller queued on s
  DM_CUDA(cudaEventRecord(entry, s));
  for (cudaStream_t q : A->pipe_s) DM_CUDA(cudaStreamWaitEvent(q, entry, 0));
  char* dx = (char*)A->stage_x.p;
  char* dy = (char*)A->stage_y.p;
  for (int j = 0; j < sh.n; ++j) {
    const int64_t lo = std::min<int64_t>(M, j * sh.xc), hi = std::min<int64_t>(M, (j + 1) * sh.xc);
    if (hi > lo)
      DM_CUDA(cudaMemcpyAsync(dx + lo * vb, (const char*)x_host + lo * vb, (hi - lo) * vb,
                              cudaMemcpyHostToDevice, s_in));
    DM_CUDA(cudaEventRecord(ex[j], s_in));
  }
  for (int c = 0; c < sh.n; ++c) {
    const int64_t t0 = c * sh.tc, t1 = std::min<int64_t>(P.ntiles, (c + 1) * sh.tc);
    if (t0 >= t1) break;
    const int64_t r0 = t0 * P.tile_rows, r1 = std::min<int64_t>(N, t1 * P.tile_rows);
    cudaStream_t q = s_cmp[c & 1];
    DM_CUDA(cudaStreamWaitEvent(q, ex[need[c]], 0));
    spmv_rows(A, dx, dy, vdt, r0, r1, q);
    DM_CUDA(cudaEventRecord(ec[c], q));
    DM_CUDA(cudaStreamWaitEvent(s_out, ec[c], 0));
    DM_CUDA(cudaMemcpyAsync((char*)y_host + r0 * vb, dy + r0 * vb, (r1 - r0) * vb,
                            cudaMemcpyDeviceToHost, s_out));
  }
  // every upload has ended too (a piece no chunk waited for may still be
  // reading the caller's x)
  DM_CUDA(cudaStreamSynchronize(s_in));
  DM_CUDA(cudaStreamSynchronize(s_out));
  return true;
}
}  // namespace
}  // namespace dm

using namespace dm;

extern "C" {

const char* dynmat_last_error(void) { return g_err; }

const char* dynmat_status_string(dynmat_status st) {
  switch (st) {
    case DYNMAT_OK: return "ok";
    case DYNMAT_ERR_INVALID_ARG: return "invalid argument";
    case DYNMAT_ERR_INDEX_RANGE: return "index out of range";
    case DYNMAT_ERR_DUPLICATE: return "duplicate entry";
    case DYNMAT_ERR_OOM: return "out of memory";
    case DYNMAT_ERR_FORMAT_TOO_LARGE: return "format too large";
    case DYNMAT_ERR_CUDA: return "CUDA error";
    case DYNMAT_ERR_BREAKDOWN: return "CG breakdown";
    case DYNMAT_ERR_NOT_CONVERGED: return "not converged";
    case DYNMAT_ERR_TIMEOUT: return "timeout";
  }
  return "unknown status";
}

dynmat_status dynmat_set_allocator(dynmat_alloc_fn alloc, dynmat_free_fn free_fn, void* ctx) {
  return guard([&] {
    DM_REQUIRE((alloc == nullptr) == (free_fn == nullptr), DYNMAT_ERR_INVALID_ARG,
               "give both allocator functions or neither");
    g_alloc = alloc;
    g_free = free_fn;
    g_alloc_ctx = ctx;
  });
}

dynmat_status dynmat_set_memory_limit(int64_t bytes) {
  return guard([&] {
    DM_REQUIRE(bytes >= 0, DYNMAT_ERR_INVALID_ARG, "negative limit");
    g_limit.store(bytes);
  });
}

int64_t dynmat_memory_in_use(void) { return g_in_use.load(); }

dynmat_status dynmat_host_alloc(int64_t bytes, void** out) {
  return guard([&] {
    DM_REQUIRE(out, DYNMAT_ERR_INVALID_ARG, "null output pointer");
    *out = nullptr;
    DM_REQUIRE(bytes > 0, DYNMAT_ERR_INVALID_ARG, "host allocation of %lld bytes",
               (long long)bytes);
    const size_t huge = (size_t)2 << 20;
    const size_t len = (size_t)round_up(bytes, (int64_t)huge);
    // map one huge page more than needed and trim both ends to a 2 MiB boundary
    void* raw = mmap(nullptr, len + huge, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
    DM_REQUIRE(raw != MAP_FAILED, DYNMAT_ERR_OOM, "mmap of %zu bytes failed", len + huge);
    char* lo = (char*)raw;
    char* p = lo + ((huge - (uintptr_t)lo % huge) % huge);
    if (p > lo) munmap(lo, p - lo);
    if (lo + len + huge > p + len) munmap(p + len, lo + len + huge - (p + len));
    madvise(p, len, MADV_HUGEPAGE);  // advice only: a kernel without THP ignores it
    const cudaError_t e = cudaHostRegister(p, len, cudaHostRegisterDefault);
    if (e != cudaSuccess) {
      cudaGetLastError();
      munmap(p, len);
      set_error("cudaHostRegister of %zu bytes: %s", len, cudaGetErrorString(e));
      throw Fail{DYNMAT_ERR_CUDA};
    }
    {
      std::lock_guard<std::mutex> g(g_host_mu);
      g_host[p] = len;
    }
    *out = p;
  });
}

dynmat_status dynmat_host_free(void* ptr) {
  return guard([&] {
    if (!ptr) return;
    size_t len = 0;
    {
      std::lock_guard<std::mutex> g(g_host_mu);
      auto it = g_host.find(ptr);
      DM_REQUIRE(it != g_host.end(), DYNMAT_ERR_INVALID_ARG,
                 "pointer %p was not returned by dynmat_host_alloc", ptr);
      len = it->second;
      g_host.erase(it);
    }
    const cudaError_t e = cudaHostUnregister(ptr);
    munmap(ptr, len);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("cudaHostUnregister: %s", cudaGetErrorString(e));
      throw Fail{DYNMAT_ERR_CUDA};
    }
  });
}

dynmat_status dynmat_set_pad_limit(double ratio) {
  return guard([&] {
    DM_REQUIRE(ratio > 0, DYNMAT_ERR_INVALID_ARG, "pad limit must be positive");
    g_pad_limit = ratio;
  });
}

dynmat_status dynmat_create(dynmat_t* out, int64_t nrows, int64_t ncols, int64_t nnz,
                            const int32_t* row, const int32_t* col, const void* val,
                            dynmat_dtype vdtype, int inputs_on_device, dynmat_stream_t stream) {
  return guard([&] {
    create_impl(out, nrows, ncols, nnz, row, col, val, vdtype, inputs_on_device,
                (cudaStream_t)stream);
  });
}

dynmat_status dynmat_destroy(dynmat_t A, dynmat_stream_t stream) {
  return guard([&] {
    destroy_handle(A, (cudaStream_t)stream);
    trim_device_pool((cudaStream_t)stream);
  });
}

dynmat_status dynmat_get_info(dynmat_t A, dynmat_info* o) {
  return guard([&] {
    DM_REQUIRE(A && o, DYNMAT_ERR_INVALID_ARG, "null argument");
    memset(o, 0, sizeof *o);
    o->format = A->fmt;
    o->vdtype = A->vdt;
    o->nrows = A->nrows;
    o->ncols = A->ncols;
    o->nnz = A->nnz;
    o->ndiag = A->fmt == DYNMAT_DIA ? A->dia.ndiag : 0;
    o->ell_width = (A->fmt == DYNMAT_ELL || A->fmt == DYNMAT_HYB) ? A->ell.K : 0;
    o->hyb_coo_nnz = A->fmt == DYNMAT_HYB ? A->coo.nnz : 0;
    o->ld = A->fmt == DYNMAT_DIA ? A->dia.ld
            : (A->fmt == DYNMAT_ELL || A->fmt == DYNMAT_HYB) ? A->ell.ld : 0;
    o->bytes = handle_bytes(A);
    o->values_exact_in_f32 = A->values_exact_f32;
    o->spmv_variant = A->plan.variant;
  });
}

dynmat_status dynmat_copy_out(dynmat_t A, dynmat_array which, void* dst, int64_t dst_bytes,
                              int dst_on_device, dynmat_stream_t stream) {
  return guard([&] {
    DM_REQUIRE(A && dst, DYNMAT_ERR_INVALID_ARG, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t vb = vsize(A->vdt), N = A->nrows;
    const void* src = nullptr;
    int64_t bytes = -1;
    const bool hyb = A->fmt == DYNMAT_HYB, ell = A->fmt == DYNMAT_ELL || hyb;
    switch (which) {
      case DYNMAT_ARR_ROW:
        if (A->fmt == DYNMAT_COO || hyb) { src = A->coo.row.p; bytes = A->coo.nnz * 4; }
        break;
      case DYNMAT_ARR_COL:
        if (A->fmt == DYNMAT_COO) { src = A->coo.col.p; bytes = A->coo.nnz * 4; }
        if (A->fmt == DYNMAT_CSR) { src = A->csr.col.p; bytes = A->csr.nnz * 4; }
        if (ell) { src = A->ell.col.p; bytes = A->ell.K * A->ell.ld * 4; }
        break;
      case DYNMAT_ARR_VAL:
        if (A->fmt == DYNMAT_COO) { src = A->coo.val.p; bytes = A->coo.nnz * vb; }
        if (A->fmt == DYNMAT_CSR) { src = A->csr.val.p; bytes = A->csr.nnz * vb; }
        if (A->fmt == DYNMAT_DIA) { src = A->dia.val.p; bytes = A->dia.ndiag * A->dia.ld * vb; }
        if (ell) { src = A->ell.val.p; bytes = A->ell.K * A->ell.ld * vb; }
        break;
      case DYNMAT_ARR_ROWPTR:
        if (A->fmt == DYNMAT_CSR) { src = A->csr.rowptr.p; bytes = (N + 1) * 4; }
        break;
      case DYNMAT_ARR_OFFSETS:
        if (A->fmt == DYNMAT_DIA) { src = A->dia.offsets.p; bytes = A->dia.ndiag * 4; }
        break;
      case DYNMAT_ARR_HYB_COL:
        if (hyb) { src = A->coo.col.p; bytes = A->coo.nnz * 4; }
        break;
      case DYNMAT_ARR_HYB_VAL:
        if (hyb) { src = A->coo.val.p; bytes = A->coo.nnz * vb; }
        break;
    }
    DM_REQUIRE(bytes >= 0, DYNMAT_ERR_INVALID_ARG, "array %d does not exist in format %d",
               (int)which, (int)A->fmt);
    DM_REQUIRE(dst_bytes >= bytes, DYNMAT_ERR_INVALID_ARG,
               "destination holds %lld bytes, array needs %lld", (long long)dst_bytes,
               (long long)bytes);
    if (bytes)
      DM_CUDA(cudaMemcpyAsync(dst, src, bytes,
                              dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    DM_CUDA(cudaStreamSynchronize(s));
  });
}

dynmat_status dynmat_convert(dynmat_t A, dynmat_format fmt, dynmat_dtype vdtype,
                             dynmat_stream_t stream) {
  return guard([&] { convert_impl(A, fmt, vdtype, (cudaStream_t)stream); });
}

dynmat_status dynmat_spmv(dynmat_t A, const void* x, void* y, dynmat_dtype vec_dtype,
                          dynmat_stream_t stream) {
  return guard([&] {
    DM_REQUIRE(A && (A->nrows == 0 || (x && y)), DYNMAT_ERR_INVALID_ARG, "null argument");
    DM_REQUIRE(vec_dtype == DYNMAT_F64 || vec_dtype == DYNMAT_F32, DYNMAT_ERR_INVALID_ARG,
               "bad vector dtype");
    spmv(A, x, y, vec_dtype, (cudaStream_t)stream);
  });
}

dynmat_status dynmat_spmv_host(dynmat_t A, const void* x_host, void* y_host,
                               dynmat_dtype vec_dtype, dynmat_stream_t stream) {
  return guard([&] {
    DM_REQUIRE(A && (A->nrows == 0 || (x_host && y_host)), DYNMAT_ERR_INVALID_ARG,
               "null argument");
    DM_REQUIRE(vec_dtype == DYNMAT_F64 || vec_dtype == DYNMAT_F32, DYNMAT_ERR_INVALID_ARG,
               "bad vector dtype");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t vb = vsize(vec_dtype);
    const size_t xb = (size_t)A->ncols * vb, yb = (size_t)A->nrows * vb;
    if (A->stage_x.bytes < DBuf::padded(xb)) A->stage_x.alloc(xb, s);
    if (A->stage_y.bytes < DBuf::padded(yb)) A->stage_y.alloc(yb, s);
    if (spmv_host_pipelined(A, x_host, y_host, vec_dtype, s)) {
      check_wait_timeout(s);
      return;
    }
    if (xb) DM_CUDA(cudaMemcpyAsync(A->stage_x.p, x_host, xb, cudaMemcpyHostToDevice, s));
    spmv(A, A->stage_x.p, A->stage_y.p, vec_dtype, s);
    if (yb) DM_CUDA(cudaMemcpyAsync(y_host, A->stage_y.p, yb, cudaMemcpyDeviceToHost, s));
    check_wait_timeout(s);
  });
}

dynmat_status dynmat_set_variant(dynmat_t A, int32_t variant) {
  return guard([&] {
    DM_REQUIRE(A, DYNMAT_ERR_INVALID_ARG, "null handle");
    DM_REQUIRE(variant >= 0 && variant <= variant_max(A->fmt), DYNMAT_ERR_INVALID_ARG,
               "format %d has no kernel variant %d", (int)A->fmt, variant);
    A->plan.forced = variant;
    cudaStream_t s = nullptr;
    prepare_spmv(A, s);
    DM_CUDA(cudaStreamSynchronize(s));
  });
}

}  // extern "C"
