// Internal declarations of the dynmat library (sm_103a). Not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <cstring>
#include <string>

#include "dynmat.h"

namespace dm {

// ---------------------------------------------------------------------------
// Errors: every ABI entry sets a thread-local message and returns a status.
// ---------------------------------------------------------------------------
void set_error(const char* fmt, ...);
void clear_error();

struct Fail {
  dynmat_status st;
};

#define DM_CUDA(call)                                                               \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      ::dm::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),       \
                      __FILE__, __LINE__);                                          \
      throw ::dm::Fail{DYNMAT_ERR_CUDA};                                            \
    }                                                                               \
  } while (0)

#define DM_CHECK_LAUNCH() DM_CUDA(cudaGetLastError())

#define DM_REQUIRE(cond, status, ...)                                               \
  do {                                                                              \
    if (!(cond)) {                                                                  \
      ::dm::set_error(__VA_ARGS__);                                                 \
      throw ::dm::Fail{status};                                                     \
    }                                                                               \
  } while (0)

// Wraps an ABI body: Fail -> its status, anything else -> CUDA/INVALID.
template <class F>
dynmat_status guard(F&& f) {
  try {
    clear_error();
    f();
    return DYNMAT_OK;
  } catch (const Fail& e) {
    return e.st;
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return DYNMAT_ERR_OOM;
  } catch (...) {
    set_error("unexpected host exception");
    return DYNMAT_ERR_INVALID_ARG;
  }
}

// ---------------------------------------------------------------------------
// Device memory through the pluggable allocator, with a byte cap.
// ---------------------------------------------------------------------------
void* dev_alloc(size_t bytes, cudaStream_t s);  // throws Fail{OOM}
void dev_free(void* p, size_t bytes, cudaStream_t s);

// Owning device buffer (move-only). Sizes are padded to 256 bytes plus a
// 256-byte tail so that vector loads that round a range out to 16 bytes stay
// inside the allocation.
struct DBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaStream_t s = nullptr;
  DBuf() = default;
  DBuf(size_t n, cudaStream_t st) { alloc(n, st); }
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept : p(o.p), bytes(o.bytes), s(o.s) { o.p = nullptr; o.bytes = 0; }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) {
      release();
      p = o.p; bytes = o.bytes; s = o.s;
      o.p = nullptr; o.bytes = 0;
    }
    return *this;
  }
  ~DBuf() { release(); }
  static size_t padded(size_t n) { return ((n + 255) / 256) * 256 + 256; }
  void alloc(size_t n, cudaStream_t st) {
    release();
    s = st;
    bytes = padded(n);
    p = dev_alloc(bytes, st);
  }
  void release() {
    if (p) dev_free(p, bytes, s);
    p = nullptr;
    bytes = 0;
  }
  template <class T> T* as() const { return reinterpret_cast<T*>(p); }
};

// ---------------------------------------------------------------------------
// Device facts sized once per process.
// ---------------------------------------------------------------------------
struct Dev {
  int id = -1;
  int sms = 148;
  int l2_bytes = 0;
};
const Dev& device();

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int64_t round_up(int64_t a, int64_t b) { return cdiv(a, b) * b; }
inline size_t vsize(int dt) { return dt == DYNMAT_F64 ? 8 : 4; }

// Leading dimension of slot-major / diagonal-major arrays: a multiple of 32
// elements, so every diagonal or slot row starts 128-byte aligned (F32) or
// 256-byte aligned (F64).
inline int64_t lead_dim(int64_t n) { return round_up(n > 0 ? n : 1, 32); }

// ---------------------------------------------------------------------------
// The dynamic matrix (§III-A): one active concrete format (State pattern).
// ---------------------------------------------------------------------------
struct Coo {
  int64_t nnz = 0;
  int64_t maxlen = 0;  // longest row (host copy, set by the SpMV plan)
  DBuf row, col, val;
};

struct Csr {
  int64_t nnz = 0;
  int64_t maxlen = 0;    // longest row (host copy, set by the SpMV plan)
  double mean_dist = 0;  // mean |col - row| over sampled rows (set by the SpMV plan)
  DBuf rowptr, col, val;
};

struct Dia {
  int64_t ndiag = 0, ld = 0;
  int32_t off_min = 0, off_max = 0;  // first and last offset (host copies)
  int64_t main_diag = -1;            // index of offset 0 (host copy); -1 if not stored
  DBuf offsets, val;
};

struct Ell {
  int64_t K = 0, ld = 0;
  DBuf col, val;
};

// Work buffers of the segmented (COO / CSR-merge / HYB-overflow) SpMV.
struct SegPlan {
  int64_t nchunks = 0;
  DBuf chunk_row;   // CSR-merge: row of each chunk's first entry (nchunks + 1)
  DBuf carry;       // per-chunk carry records
  DBuf unit_start;  // COO stream kernel: first entry of each base of rows (nbases + 1)
};

struct dynmat_impl;  // fwd
}  // namespace dm

// Launch plan of the active format's SpMV (the tuner's "tile shape").
namespace dm {
// DIA diagonals grouped into runs of consecutive offsets (at most
// DIA_RUN_LEN long, at most DIA_RUNS runs): run r covers offsets
// start[r] .. start[r] + len[r] - 1. n = 0: no grouping (too many runs).
constexpr int DIA_RUNS = 48, DIA_RUN_LEN = 4;
struct DiaRuns {
  int32_t n = 0;
  int32_t start[DIA_RUNS];
  int32_t len[DIA_RUNS];
};

// Most pieces of the host-buffer product's copy/compute pipeline.
constexpr int PIPE_MAX = 16;

struct Plan {
  int32_t variant = 0;      // CSR: 1..5 vector (2^variant lanes), 6 merge, 7 stream; COO: 1 segmented, 2 stream
  int32_t forced = 0;       // variant set by the user / tuner (0 = automatic)
  int64_t tile_rows = 0;    // rows per tile of the row-based kernels
  int64_t ntiles = 0;       // tiles (= partial sums of a fused dot product)
  int32_t stream_cap = 0;   // CSR stream kernel: entries staged in shared memory per pass
  DiaRuns runs;             // DIA variant 6: the offsets as runs
};
}  // namespace dm

struct dynmat_s {
  int64_t nrows = 0, ncols = 0, nnz = 0;
  dynmat_format fmt = DYNMAT_COO;
  dynmat_dtype vdt = DYNMAT_F64;
  int values_exact_f32 = 0;
  dm::Plan plan;
  dm::Coo coo;            // COO, and the COO part of HYB
  dm::Csr csr;
  dm::Dia dia;
  dm::Ell ell;            // ELL, and the ELL part of HYB
  dm::SegPlan seg;        // plan of the segmented kernels for the active format
  // Staging for dynmat_spmv_host, and its copy/compute pipeline (streams
  // and per-chunk events, created on first use).
  dm::DBuf stage_x, stage_y;
  cudaStream_t pipe_s[4] = {};                    // copies in, products (two), copies out
  cudaEvent_t pipe_ev[2 * dm::PIPE_MAX + 1] = {};  // x pieces, products, entry
  // ELL: per row chunk of the pipeline, the x piece holding its largest column
  int32_t pipe_need[dm::PIPE_MAX] = {};
  uint64_t pipe_need_gen = 0;  // plan generation it was measured at
  int32_t pipe_need_n = 0;     // chunks it was measured for
  // Bumped whenever the active format or its launch plan changes.
  uint64_t gen = 1;
  // Product scratch of dynmat_spmv_acc (nrows of the vector type).
  dm::DBuf acc_tmp;
  // FP32 copy used by the mixed-precision inner solve of an F64 matrix.
  dynmat_s* shadow32 = nullptr;
  // CG work space (allocated on the first solve, reused).
  dm::DBuf cg_work;
  size_t cg_work_bytes = 0;
};

namespace dm {

int64_t handle_bytes(const dynmat_s* A);
void free_format(dynmat_s* A, cudaStream_t s);  // releases the active format's arrays

// Scan / sort / reduction primitives (sort.cu).
// Exclusive scan of n int32 counts into out (int32), returning the total.
// Blocking only when `total` is requested.
void exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, int64_t* total,
                        cudaStream_t s);
// Stable LSD radix sort of 64-bit keys with a 32- or 64-bit payload, on the
// low `bits` bits. keys/vals are sorted in place (uses temporaries).
void radix_sort_u64(uint64_t* keys, int32_t* vals, int64_t n, int bits, cudaStream_t s);
void radix_sort_u64(uint64_t* keys, uint64_t* vals, int64_t n, int bits, cudaStream_t s);
// Kernel variants of a format run 1..variant_max(f) (0: automatic).
int variant_max(dynmat_format f);
// max over n int32 values (blocking), 0 for n == 0.
int64_t reduce_max_i32(const int32_t* in, int64_t n, cudaStream_t s);

// Conversions (convert.cu). Each builds the target from a canonical COO
// (row, col, val in the handle's value type).
void build_from_coo(dynmat_s* A, const Coo& src, dynmat_format fmt, dynmat_dtype vdt,
                    cudaStream_t s);
void to_coo(const dynmat_s* A, Coo& out, cudaStream_t s);
int64_t hyb_width(const int32_t* rowptr, int64_t N, int64_t maxlen, int64_t vb, cudaStream_t s);
void destroy_handle(dynmat_s* A, cudaStream_t s);
// 1 if every value of val[0..n) is exactly representable in FP32 (blocking).
int values_exact_in_f32(const void* val, int64_t n, dynmat_dtype dt, cudaStream_t s);
void convert_impl(dynmat_s* A, dynmat_format fmt, dynmat_dtype vdt, cudaStream_t s);
void csr_rowptr_from_rows(const int32_t* row, int64_t nnz, int64_t nrows, int32_t* rowptr,
                          cudaStream_t s);
// flag[col[e] - row[e] + nrows - 1] = 1 for every entry e (flag zeroed by
// the caller, nrows + ncols - 1 of them): the distinct offsets of a COO.
void mark_offsets(const int32_t* row, const int32_t* col, int64_t nnz, int64_t nrows,
                  int32_t* flag, cudaStream_t s);

// SpMV dispatch (spmv.cu). spmv_dot also forms the dot product x.y with the
// fixed tile partition of the plan (fused where the format allows).
struct DotSpec;
void spmv(const dynmat_s* A, const void* x, void* y, dynmat_dtype vdt_vec, cudaStream_t s);
// HPCG's multigrid preconditioner (hpcg.cu): z = M^{-1} r, one V-cycle;
// every kernel returns at once while *skip != 0 (skip may be NULL).
void mg_vcycle(dynmat_mg_s* M, const double* r, double* z, const int32_t* skip, cudaStream_t s);
void mg_check_timeout(dynmat_mg_s* M, cudaStream_t s);
const dynmat_s* mg_matrix(const dynmat_mg_s* M);  // the finest level
// Whether the active kernel runs row ranges: DIA, ELL, HYB without a COO
// overflow, CSR variants 1-5 and 7, COO variant 2 (tile-based kernels).
bool has_row_ranges(const dynmat_s* A);
// Rows [r0, r1) of y = A x for a matrix with has_row_ranges (r0 a multiple
// of the plan's tile_rows; the same bits as spmv gives those rows).
void spmv_rows(const dynmat_s* A, const void* x, void* y, dynmat_dtype vdt_vec, int64_t r0,
               int64_t r1, cudaStream_t s);
// Blocking: DYNMAT_ERR_TIMEOUT if a bounded device wait ran out since the last check.
void check_wait_timeout(cudaStream_t s);
// y += A x in one pass where the format's kernel accumulates (COO, CSR merge);
// false (nothing launched) otherwise.
bool spmv_accumulate(const dynmat_s* A, const void* x, void* y, dynmat_dtype vdt_vec,
                     cudaStream_t s);
void spmv_dot(const dynmat_s* A, const void* x, void* y, dynmat_dtype vdt_vec,
              const DotSpec* dot, cudaStream_t s);
void spmv_skip(const dynmat_s* A, const void* x, void* y, dynmat_dtype vdt_vec,
               const DotSpec* dot, const int32_t* skip, cudaStream_t s);
void dot_tiles(const dynmat_s* A, const void* a, const void* b, dynmat_dtype vdt_vec,
               const DotSpec& dot, cudaStream_t s);
void prepare_spmv(dynmat_s* A, cudaStream_t s);  // plans / work buffers
int auto_variant(const dynmat_s* A);

// Features (select.cu).
void compute_features(const dynmat_s* A, int32_t guard, dynmat_features* f, cudaStream_t s);

}  // namespace dm
