/*
 * dynmat — dynamic sparse matrices on one B300 GPU (sm_103a).
 *
 * A C ABI for the method of "Exploiting dynamic sparse matrices for
 * performance portable linear algebra operations" (arXiv 2209.06478): a sparse
 * matrix whose storage format is switched at run time (§III-A, the
 * DynamicMatrix and its activate()), element-wise conversion between formats
 * through COO (§III-B), one `multiply` interface over every format (§III-D),
 * and the CG solve of HPCG with the preconditioner disabled (§II-B, §IV-B).
 *
 * Conventions for every call:
 *  - Return value: DYNMAT_OK or an error status; no C++ exception crosses
 *    this boundary. dynmat_last_error() gives a message for the last failure
 *    on the calling thread.
 *  - Indices are int32 (row, column, CSR row pointer, DIA offset); sizes are
 *    int64. A matrix has at most 2^31 - 1 rows, columns and stored entries.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream). Calls that only launch work return before the GPU is done;
 *    calls documented as blocking synchronise `stream` themselves.
 *  - A handle may be used from one stream at a time. Vectors passed to a
 *    call (x, y, b) are caller-owned device buffers that the library aliases
 *    for the duration of the call only (§IV-A "unmanaged" containers).
 *  - Device memory owned by a handle comes from the allocator set with
 *    dynmat_set_allocator (default: the library's own stream-ordered memory
 *    pool on the device, cudaMallocFromPoolAsync / cudaFreeAsync on the
 *    call's stream). The default pool keeps freed memory cached for reuse
 *    (format conversions reuse their temporaries); dynmat_destroy gives the
 *    cache back to the device, and so does an allocation that fails before
 *    it is retried.
 */
#ifndef DYNMAT_H
#define DYNMAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dynmat_s* dynmat_t;
typedef void* dynmat_stream_t; /* cudaStream_t */

/* The concrete formats a dynamic matrix can hold (§III-A; ELL and HYB from
 * §VI). Layouts, all in device memory, nrows = N:
 *  COO: row[nnz], col[nnz], val[nnz]; sorted by (row, col), no duplicates.
 *  CSR: rowptr[N+1], col[nnz], val[nnz]; columns ascending in each row.
 *  DIA: offsets[ndiag] ascending (offset = col - row); val[ndiag * ld] with
 *       val[d*ld + i] = a(i, i + offsets[d]), 0 where the entry is absent or
 *       outside the matrix; ld = N rounded up to a multiple of 32.
 *  ELL: width K = longest row; col[K*ld], val[K*ld] slot-major: slot k of
 *       row i holds the row's k-th entry in column order, padding col = -1
 *       and val = 0; ld as for DIA.
 *  HYB: an ELL part of width K_h plus a COO part (sorted by (row, col)) with
 *       each row's entries beyond the first K_h. K_h minimises the modelled
 *       bytes (4+v) k N + (8+v) sum_i max(0, len_i - k), v = value bytes,
 *       ties to the smaller k. */
typedef enum {
  DYNMAT_COO = 0,
  DYNMAT_CSR = 1,
  DYNMAT_DIA = 2,
  DYNMAT_ELL = 3,
  DYNMAT_HYB = 4
} dynmat_format;

/* Value type of the stored matrix or of a vector. */
typedef enum { DYNMAT_F64 = 0, DYNMAT_F32 = 1 } dynmat_dtype;

typedef enum {
  DYNMAT_OK = 0,
  DYNMAT_ERR_INVALID_ARG = 1,      /* null pointer, negative size, bad enum, ... */
  DYNMAT_ERR_INDEX_RANGE = 2,      /* a row or column index outside the matrix */
  DYNMAT_ERR_DUPLICATE = 3,        /* two entries at the same (row, col) */
  DYNMAT_ERR_OOM = 4,              /* allocation failed or over the memory limit */
  DYNMAT_ERR_FORMAT_TOO_LARGE = 5, /* padded format over the padding limit */
  DYNMAT_ERR_CUDA = 6,             /* a CUDA runtime call failed */
  DYNMAT_ERR_BREAKDOWN = 7,        /* CG: p.Ap <= 0 (matrix not SPD) */
  DYNMAT_ERR_NOT_CONVERGED = 8,    /* CG: iteration limit reached */
  DYNMAT_ERR_TIMEOUT = 9           /* a bounded device-side wait ran out */
} dynmat_status;

/* ---------------------------------------------------------------------- */
/* Memory                                                                  */
/* ---------------------------------------------------------------------- */

/* Device allocator used for everything a handle owns. `alloc` returns NULL on
 * failure; both receive the stream of the call that allocates or frees and
 * the `ctx` given here. Passing NULL for both restores the default (the
 * library's caching pool, see above). Set it before creating handles: memory
 * is always freed through the allocator that provided it. Not thread-safe
 * against concurrent calls. */
typedef void* (*dynmat_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*dynmat_free_fn)(void* ptr, size_t bytes, void* stream, void* ctx);
dynmat_status dynmat_set_allocator(dynmat_alloc_fn alloc, dynmat_free_fn free_fn, void* ctx);

/* A process-wide cap on device bytes held by the library (handles and their
 * work buffers); 0 = no cap. An allocation that would exceed it fails with
 * DYNMAT_ERR_OOM. Used by admission control under an HBM budget. */
dynmat_status dynmat_set_memory_limit(int64_t bytes);
/* Device bytes the library holds right now. */
int64_t dynmat_memory_in_use(void);

/* Padded formats (DIA, ELL) whose modelled bytes exceed `ratio` times the CSR
 * bytes of the same matrix are refused by dynmat_convert with
 * DYNMAT_ERR_FORMAT_TOO_LARGE (§V-E: DIA padding on irregular matrices runs
 * out of memory). Default 16. */
dynmat_status dynmat_set_pad_limit(double ratio);

/* Page-locked host memory for the host-buffer calls (dynmat_spmv_host).
 * Returns in *out `bytes` (> 0) of zeroed host memory that starts on a
 * 2 MiB boundary, is advised for transparent huge pages and is registered
 * with CUDA (cudaHostRegister), so copies to and from it run at the host
 * link's rate. Memory pinned in 4 KB pages copies more slowly, and
 * increasingly so as the host's free memory fragments, so the rate of
 * ordinary pinned buffers depends on when in a process they are allocated.
 * The caller owns the memory until dynmat_host_free. Not counted by
 * dynmat_memory_in_use. Errors: INVALID_ARG (bytes <= 0, out NULL), OOM
 * (the mapping failed), CUDA (the registration failed). */
dynmat_status dynmat_host_alloc(int64_t bytes, void** out);
/* Unregisters and unmaps memory returned by dynmat_host_alloc. NULL is a
 * no-op; any other pointer not returned by dynmat_host_alloc (or already
 * freed) fails with INVALID_ARG and is left alone. */
dynmat_status dynmat_host_free(void* ptr);

/* ---------------------------------------------------------------------- */
/* Create, inspect, destroy                                                */
/* ---------------------------------------------------------------------- */

/* Builds a dynamic matrix from COO triplets by element-wise conversion
 * (§IV-A step 1, §IV-B "Problem Optimization setup").
 *  nrows, ncols, nnz: matrix shape and entry count (>= 0, < 2^31).
 *  row, col: int32[nnz]; val: nnz values of type `vdtype`. In device memory
 *    if inputs_on_device != 0, else in host memory. Any order; they are
 *    copied, never retained or modified.
 *  On success *out receives a new handle in COO format (canonical order).
 *  Errors: INVALID_ARG, INDEX_RANGE (checked first), DUPLICATE, OOM, CUDA;
 *  *out is left untouched on failure. Blocking. */
dynmat_status dynmat_create(dynmat_t* out, int64_t nrows, int64_t ncols, int64_t nnz,
                            const int32_t* row, const int32_t* col, const void* val,
                            dynmat_dtype vdtype, int inputs_on_device, dynmat_stream_t stream);

/* Builds the HPCG problem matrix directly on the device (§II-B: Poisson on a
 * regular nx x ny x nz grid). points = 27: a(i,i) = 26 and a(i,j) = -1 for
 * the in-grid neighbours in the 3x3x3 box; points = 7: a(i,i) = 6 and -1 for
 * the six face neighbours. Row i = ix + nx*(iy + ny*iz). The result equals,
 * bit for bit, dynmat_create on the same triplets followed by
 * dynmat_convert(fmt, vdtype). Errors: INVALID_ARG (sizes, points, more
 * than 2^31 - 1 entries), OOM, CUDA. Blocking. */
dynmat_status dynmat_create_stencil(dynmat_t* out, int64_t nx, int64_t ny, int64_t nz,
                                    int32_t points, dynmat_format fmt, dynmat_dtype vdtype,
                                    dynmat_stream_t stream);

/* Frees the handle and everything it owns. Blocking: with the default
 * allocator it waits for `stream`, then returns the memory pool's cached
 * bytes to the device. */
dynmat_status dynmat_destroy(dynmat_t A, dynmat_stream_t stream);

typedef struct {
  int32_t format;      /* dynmat_format */
  int32_t vdtype;      /* dynmat_dtype of the stored values */
  int64_t nrows, ncols;
  int64_t nnz;         /* stored entries (explicit zeros included) */
  int64_t ndiag;       /* DIA: number of diagonals */
  int64_t ell_width;   /* ELL: K; HYB: K_h */
  int64_t hyb_coo_nnz; /* HYB: entries in the COO part */
  int64_t ld;          /* DIA / ELL / HYB-ELL leading dimension */
  int64_t bytes;       /* device bytes owned by the handle */
  int32_t values_exact_in_f32; /* 1 if every value is exactly representable in FP32 */
  int32_t spmv_variant;        /* kernel variant the tuner picked (see dynmat_set_variant) */
} dynmat_info;

dynmat_status dynmat_get_info(dynmat_t A, dynmat_info* out);

/* Arrays of the active format, for dynmat_copy_out. */
typedef enum {
  DYNMAT_ARR_ROW = 0,      /* COO row / HYB COO-part row (int32) */
  DYNMAT_ARR_COL = 1,      /* COO, CSR col; ELL / HYB-ELL col (int32) */
  DYNMAT_ARR_VAL = 2,      /* COO, CSR, DIA, ELL / HYB-ELL values */
  DYNMAT_ARR_ROWPTR = 3,   /* CSR row pointers (int32, N+1) */
  DYNMAT_ARR_OFFSETS = 4,  /* DIA offsets (int32) */
  DYNMAT_ARR_HYB_COL = 5,  /* HYB COO-part col (int32) */
  DYNMAT_ARR_HYB_VAL = 6   /* HYB COO-part values */
} dynmat_array;

/* Copies one array of the active format (deep copy, §III-B) into `dst`
 * (host memory if dst_on_device == 0). `dst_bytes` must be at least the
 * array's size: count x element size, where count is nnz, N+1, ndiag,
 * ndiag*ld, K*ld or hyb_coo_nnz as the layout above gives. Blocking. */
dynmat_status dynmat_copy_out(dynmat_t A, dynmat_array which, void* dst, int64_t dst_bytes,
                              int dst_on_device, dynmat_stream_t stream);

/* ---------------------------------------------------------------------- */
/* Format switching (§III-A activate(), §III-B convert, §IV-B)             */
/* ---------------------------------------------------------------------- */

/* Converts A in place to `fmt` with values of type `vdtype`, going through
 * COO (§III-B proxy policy: active format -> COO -> fmt). The result equals,
 * bit for bit, the canonical layout above. DIA drops stored zeros (it cannot
 * tell them from padding); every other format keeps them. Converting F64
 * values to F32 rounds to nearest.
 * Errors: INVALID_ARG, FORMAT_TOO_LARGE (see dynmat_set_pad_limit), OOM,
 * CUDA. On failure A is unchanged and still valid. Blocking. */
dynmat_status dynmat_convert(dynmat_t A, dynmat_format fmt, dynmat_dtype vdtype,
                             dynmat_stream_t stream);

/* Integer features of A's COO view and the modelled bytes per format
 * (v = value bytes of A, indices 4 bytes):
 *   COO (8+v) nnz; CSR (4+v) nnz + 4 (N+1); DIA v ndiag N + 4 ndiag;
 *   ELL (4+v) maxlen N; HYB (4+v) K_h N + (8+v) overflow. */
typedef struct {
  int64_t nrows, ncols, nnz;
  int64_t ndiag;     /* distinct diagonals holding an entry */
  int64_t maxlen;    /* longest row */
  int64_t hyb_k;     /* K_h */
  int64_t hyb_over;  /* entries beyond K_h */
  int64_t bytes[5];  /* modelled bytes indexed by dynmat_format */
  int32_t choice;    /* the deterministic rule's format */
  int32_t guard;     /* padding guard used */
} dynmat_features;

/* Selection modes. FEATURES: a deterministic rule on the features — padded
 * formats (DIA, ELL) over `guard` (3) times the CSR bytes are excluded, the
 * smallest modelled bytes win, ties in the order DIA, ELL, CSR, HYB, COO.
 * PROFILE: §V-E's auto-tuner — converts a copy of A to each admissible
 * format, times its SpMV on the GPU and returns the fastest (A itself is not
 * changed). Neither mode converts A. */
enum { DYNMAT_SELECT_FEATURES = 0, DYNMAT_SELECT_PROFILE = 1 };

dynmat_status dynmat_features_get(dynmat_t A, int32_t guard, dynmat_features* out,
                                  dynmat_stream_t stream);
dynmat_status dynmat_select_format(dynmat_t A, int mode, dynmat_format* out,
                                   dynmat_stream_t stream);

/* The per-matrix auto-tuner (§V-E, run online): profiles like
 * DYNMAT_SELECT_PROFILE, including the kernel variants of CSR (lanes per
 * row, nnz-balanced), then converts A to the fastest format and fixes that
 * variant. Either output pointer may be NULL. Blocking. */
dynmat_status dynmat_autotune(dynmat_t A, dynmat_format* fmt_out, int32_t* variant_out,
                              dynmat_stream_t stream);

/* Keeps A's format and times each kernel variant of it (see
 * dynmat_set_variant) on a zero vector, 5 runs after 2 warm-ups, median;
 * fixes the fastest, where the automatic variant is kept unless another is
 * at least 2% faster. `variant_out` may be NULL. Blocking. */
dynmat_status dynmat_tune_variant(dynmat_t A, int32_t* variant_out, dynmat_stream_t stream);

/* ---------------------------------------------------------------------- */
/* multiply (§III-D): y = A x                                              */
/* ---------------------------------------------------------------------- */

/* y[i] = sum_j a(i, j) x[j] over the stored entries, dispatched on the
 * active format. x: ncols device values, y: nrows device values, both of
 * type `vec_dtype`; y must not overlap x. Value/vector combinations:
 * F64 values with F64 vectors (FP64 sums), F32 values with F32 vectors
 * (FP32 sums), F32 values with F64 vectors (FP64 sums). Every row's sum has
 * exactly one writer, so the result is deterministic run to run.
 * Asynchronous on `stream`. Errors: INVALID_ARG, CUDA. The CSR stream
 * kernel (CSR variants 7 and 8, COO variant 2) bounds every wait of its copy
 * pipeline; if one ever
 * ran out, its y is invalid and the next blocking call (dynmat_spmv_host,
 * cg_solve, pcg_solve) returns DYNMAT_ERR_TIMEOUT. */
dynmat_status dynmat_spmv(dynmat_t A, const void* x, void* y, dynmat_dtype vec_dtype,
                          dynmat_stream_t stream);

/* The same product with x and y in HOST memory: copies x to the device,
 * runs the product and copies y back, after the work already queued on
 * `stream`, and returns once y is on the host; the results have the bits
 * dynmat_spmv gives. Staging buffers are owned by the handle and reused.
 * Above 8 MiB of x and y, on the tile-based kernels (DIA, ELL, HYB without
 * a COO overflow, CSR variants 1-5, 7 and 8, COO variant 2), the copies and the
 * product overlap: x goes up
 * in pieces on a stream of the handle, the product runs in row chunks on two
 * more, each waiting only for the pieces of x its rows read, and each
 * chunk's y comes down on a fourth. Host memory from dynmat_host_alloc copies
 * fastest; pageable memory works, without the overlap of the copies. */
dynmat_status dynmat_spmv_host(dynmat_t A, const void* x_host, void* y_host,
                               dynmat_dtype vec_dtype, dynmat_stream_t stream);

/* COO product that allocates no device memory. The paper has no
 * counterpart: this call is for callers that cannot allocate at the time
 * they multiply — processes whose device allocator is disabled or
 * budget-locked while a solver runs (every byte is accounted to someone
 * else), and latency-bound loops or hosts that forbid cudaMalloc on the hot
 * path because it can synchronise the device or fail under memory pressure.
 *  y[i] = sum over the entries e with row[e] == i of val[e] * x[col[e]],
 *  FP64 values, vectors and sums — the same kernel and the same results as
 *  dynmat_spmv on a COO handle.
 *  row, col, val: nnz entries in device memory, canonical COO (sorted by
 *    (row, col), no duplicates, indices in range — not checked here; the
 *    arrays of a COO handle copied out with dynmat_copy_out qualify), each
 *    starting on a 16-byte boundary. x: device, at least max(col)+1 values;
 *    y: device, nrows values, not overlapping x. Caller-owned; nothing is
 *    retained.
 *  Work space: a fixed 4 MiB array compiled into the library (held on every
 *    GPU that loads it until the process exits), enough for
 *    DYNMAT_NOALLOC_MAX_NNZ entries; larger nnz is refused with
 *    DYNMAT_ERR_INVALID_ARG before anything runs. The array is shared by
 *    every call in the process, so calls whose work overlaps on the GPU
 *    (different streams, or host threads) race and give wrong results:
 *    order them on one stream. It keeps the last call's contents; nothing
 *    in it needs clearing between calls.
 *  The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before capturing a stream into a graph. The address is kept for the
 *    life of the process: after cudaDeviceReset, or any other reset of the
 *    device's primary context, it is stale, and this entry point must not
 *    be called again in that process.
 *  Asynchronous on `stream`; errors: INVALID_ARG, CUDA. */
#define DYNMAT_NOALLOC_MAX_NNZ 16777216LL
dynmat_status dynmat_spmv_coo_noalloc(int64_t nrows, int64_t nnz, const int32_t* row,
                                      const int32_t* col, const double* val, const double* x,
                                      double* y, dynmat_stream_t stream);

/* Kernel variant for the active format, as picked by the tuner
 * (0 = automatic). CSR: 1..5 = vector kernel with 2,4,8,16,32 lanes per row,
 * 6 = nnz-balanced (merge) kernel, 7 = stream kernel (a block's 256 rows'
 * contiguous entries copied to shared memory by TMA, two threads per row),
 * 8 = as 7 with 64-row bases (a smaller staging ring, several blocks per
 * SM: faster where neighbouring rows read nearby x, as in banded matrices;
 * slower on random columns). Automatic: the stream kernel when the mean row
 * length is at least 4 and the longest row is at most 2 x mean + 32
 * entries, else 6; of the stream kernels 8 when the mean |col - row| over
 * 4096 sampled rows is at most min(N / 32, 65536), else 7. DIA (row counts for
 * FP64; FP32 doubles them): 1 = two rows per thread, 2 = four rows per
 * thread, 3 = two rows per thread with half-size tiles (more resident
 * blocks), 4 = as 3 with two multiply-add chains per row, 5 = four rows
 * with two chains per row, 6 = as 1 with the diagonals in runs of
 * consecutive offsets (FP64 values and vectors, x 16-byte aligned; else 1;
 * on large matrices one-pass tiles over every resident block),
 * 7 = a block takes 32 rows at a time and its 8 warps split the diagonals,
 * the partial sums added in warp order (small matrices); automatic: 7 when
 * 3's tiles would number fewer than two per SM, else 3 when 1's would, else
 * 6 for FP64 values, else 1. COO: 1 = segmented kernel (nnz-balanced, warp
 * scan), 2 = stream kernel (as CSR 7, 128-row bases, rows found by binary
 * search in the staged row indices); automatic by the CSR rule. ELL and HYB
 * (its ELL part): 1 = a thread per two rows (FP64; four for FP32), slots in
 * order; 2 = a block takes 32 rows at a time and its 8 warps split the
 * slots, the partial sums added in warp order (for small matrices);
 * automatic: 2 when 1's 1024-row tiles (FP64) would number fewer than two per
 * SM, else 1. */
dynmat_status dynmat_set_variant(dynmat_t A, int32_t variant);

/* Diagonal extraction (§III-D): diag[i] = a(i, i) for i < min(nrows, ncols),
 * 0 where (i, i) is not stored (DIA: the offset-0 diagonal, 0 if it is
 * absent). diag: device array of the matrix's value type. Blocking. */
dynmat_status dynmat_diagonal(dynmat_t A, void* diag, dynmat_stream_t stream);

/* Diagonal update in the active format (§III-D; §IV-B: HPCG's CG test
 * exaggerates the diagonal and restores it): every stored (i, i) entry
 * becomes diag[i] (device array of the matrix's value type); the structure is
 * unchanged. Every i < min(nrows, ncols) must have its (i, i) entry stored
 * (DIA: the offset-0 diagonal must exist, all its slots count as stored),
 * else INVALID_ARG and nothing changes. Blocking. */
dynmat_status dynmat_set_diagonal(dynmat_t A, const void* diag, dynmat_stream_t stream);

/* y += A x (y is read and updated; x, y as for dynmat_spmv). Rows without
 * entries keep their y. The COO and CSR stream kernels and the segmented
 * COO / CSR-merge kernels add in one pass; other kernels go through a
 * scratch vector the handle keeps (nrows values). Asynchronous. */
dynmat_status dynmat_spmv_acc(dynmat_t A, const void* x, void* y, dynmat_dtype vec_dtype,
                              dynmat_stream_t stream);

/* ---------------------------------------------------------------------- */
/* Local / remote split of a partitioned matrix (§IV-B, §V-E)             */
/* ---------------------------------------------------------------------- */

/* dst[k] = src[idx[k]] for k < n (device arrays; idx int32 indices into src).
 * On one device this is the halo exchange of a partitioned product. */
dynmat_status dynmat_gather(const void* src, const int32_t* idx, int64_t n, void* dst,
                            dynmat_dtype vec_dtype, dynmat_stream_t stream);

/* One process's product of a partitioned matrix whose rows are split into a
 * square local part and a rectangular remote part, each a dynamic matrix in
 * its own format (§IV-B: the remote part makes the local system matrix
 * irregular; §V-E: Morpheus / Ghost / multi-format versions):
 *   x_ext = x_src[halo]        (n_ext halo values; x_ext is caller scratch)
 *   y     = A_loc x_loc + A_rem x_ext
 * A_loc: n x n. A_rem: n x n_ext, or NULL when the process has no remote
 * columns (then halo, x_src and x_ext are not read). halo: device int32
 * indices into x_src. All vectors are device arrays of vec_dtype; y must not
 * alias the inputs. Asynchronous; INVALID_ARG on mismatched shapes. */
dynmat_status dynmat_split_spmv(dynmat_t A_loc, dynmat_t A_rem, const int32_t* halo, int64_t n_ext,
                                const void* x_src, const void* x_loc, void* x_ext, void* y,
                                dynmat_dtype vec_dtype, dynmat_stream_t stream);

/* ---------------------------------------------------------------------- */
/* Conjugate gradient (§II-B, §IV-B: HPCG's CG, preconditioner disabled)   */
/* ---------------------------------------------------------------------- */

typedef enum { CG_FP64 = 0, CG_MIXED = 1, CG_MIXED_RELIABLE = 2 } cg_precision;

typedef struct {
  double tol;            /* FP64: stop when ||r|| / ||r_0|| <= tol; MIXED*: ||b - A x|| / ||b|| */
  int32_t max_iters;     /* FP64, MIXED_RELIABLE: iterations; MIXED: inner iterations per step */
  int32_t precision;     /* cg_precision */
  double inner_tol;      /* MIXED: inner FP32 relative residual target (e.g. 1e-5) */
  int32_t max_outer;     /* MIXED: refinement steps (e.g. 30) */
  int32_t check_every;   /* iterations between host checks of the device-side status */
  double delta;          /* MIXED_RELIABLE: fold when the recursive residual fell below
                            delta x its value at the last fold (0 = default 0.1) */
} cg_opts;

typedef struct {
  int32_t status;            /* dynmat_status of the solve */
  int32_t iterations;        /* CG iterations (MIXED: inner iterations in total) */
  int32_t outer_iterations;  /* MIXED: refinement steps; MIXED_RELIABLE: folds */
  double rel_residual;       /* FP64: recursive ||r_k|| / ||r_0||; MIXED*: last FP64 ||r||/||b|| */
  double true_rel_residual;  /* ||b - A x|| / ||b|| recomputed in FP64 at the end */
} cg_result;

/* Solves A x = b. b: nrows FP64 device values; x: nrows FP64 device values,
 * the starting guess on entry (FP64) and the solution on return. A must be
 * square.
 * FP64: textbook CG — r = b - A x; p = r; each iteration q = A p,
 * alpha = r.r / p.q, x += alpha p, r -= alpha q, beta = r'.r' / r.r,
 * p = r + beta p; dot products are reduced in a fixed order (deterministic).
 * MIXED: iterative refinement from x = 0 — r = b - A x in FP64 with FP64
 * sums; inner CG in FP32 (FP32 values and vectors, FP32 SpMV sums, dot
 * products summed in FP64, alpha and beta formed in FP64) on A d = r,
 * restarted for every refinement; x += d in FP64; stops when
 * ||r|| / ||b|| <= tol.
 * MIXED_RELIABLE: from x = 0, one FP32 CG of the same kind on A x = b whose
 * FP32 correction is folded into the FP64 x — x += d, r = b - A x in FP64,
 * r32 = (float) r — whenever its recursive residual has dropped below delta
 * times its value at the last fold, or meets tol, or at max_iters; the
 * search direction continues across folds (no restart), so the iteration
 * count stays close to FP64 CG's while each iteration moves FP32 data.
 * Converged when an FP64 residual after a fold meets tol.
 * If A holds F64 values the FP32 work uses an FP32 copy that the handle
 * keeps until the next conversion, and the FP64 residuals use A's F64
 * values. Blocking. The call returns DYNMAT_OK when the solve ran;
 * `res->status` says whether it converged (OK, BREAKDOWN, NOT_CONVERGED). */
dynmat_status cg_solve(dynmat_t A, const double* b, double* x, const cg_opts* opts,
                       cg_result* res, dynmat_stream_t stream);

/* ---------------------------------------------------------------------- */
/* HPCG's preconditioned CG (§II-B: symmetric Gauss-Seidel inside          */
/* multigrid; the paper's runs disable it, §IV-B)                          */
/* ---------------------------------------------------------------------- */

/* The multigrid hierarchy of HPCG's problem: level l is the `points`-point
 * stencil (7 or 27) on the nx/2^l x ny/2^l x nz/2^l grid, each a dynamic
 * matrix in DIA with FP64 values, built on the device. nx, ny, nz must
 * divide by 2^(levels-1), and the coarsest grid must keep every diagonal of
 * the stencil (at least 3 points per dimension for 27 points, 2 for 7),
 * and the finest grid has at most 2^31 - 1 points; levels 1..8. Coarse
 * point (i, j, k) is fine point (2i, 2j, 2k). Each level
 * also keeps its values in colour order for the smoother (twice the DIA
 * values in all). Blocking; INVALID_ARG, OOM, CUDA. */
typedef struct dynmat_mg_s* dynmat_mg_t;
dynmat_status dynmat_mg_create(dynmat_mg_t* out, int64_t nx, int64_t ny, int64_t nz,
                               int32_t points, int32_t levels, dynmat_stream_t stream);
dynmat_status dynmat_mg_destroy(dynmat_mg_t M, dynmat_stream_t stream);

/* Level `level`'s matrix (borrowed: owned by M, valid until it is destroyed;
 * do not convert it) and, if dims != NULL, its grid (3 values). */
dynmat_status dynmat_mg_level(dynmat_mg_t M, int32_t level, dynmat_t* A, int64_t* dims);

/* One symmetric Gauss-Seidel sweep on level `level`, z updated in place
 * (device FP64 vectors of the level's size). Rows are taken colour by colour,
 * colour(i) = 7 - ((ix & 1) + 2 (iy & 1) + 4 (iz & 1)), forward colours 0..7
 * then backward 7..0; no two stencil neighbours share a colour, so a
 * colour's rows update in parallel: z_i = (r_i - sum_{j != i} a_ij z_j) /
 * a_ii, the sum in column order; the division is a multiplication by 1/a_ii,
 * computed once per level (within one rounding of the quotient). The coarse
 * grid's points are colour 7: the last colour of a sweep has zero residual,
 * which injection would hand to the coarse grid. One cooperative launch per
 * sweep, its colours separated by a bounded grid barrier whose count is
 * cleared before each launch; a barrier that timed out (never expected)
 * leaves a flag that the next pcg_solve reports as DYNMAT_ERR_TIMEOUT, and
 * later launches are not affected by it. Asynchronous. */
dynmat_status dynmat_mg_symgs(dynmat_mg_t M, int32_t level, const double* r, double* z,
                              dynmat_stream_t stream);

/* z = M^{-1} r: one V-cycle (level 0 vectors). On level l: z = 0; the
 * coarsest level is one sweep; otherwise a sweep, t = r - A_l z, the coarse
 * right-hand side t at the coarse points (injection), the coarse V-cycle,
 * z += the coarse z at the coarse points (injection), a sweep. The
 * preconditioner is symmetric positive definite. Launches: a sweep of level
 * 0, everything below level 0 in one cooperative launch, a sweep of level 0
 * (sweeps that start from z = 0 skip the products with neighbours still at
 * 0; the residual is formed only at the coarse points). Where the smallest
 * levels are small enough (at most 256 points of a colour per CTA of a
 * thread-block cluster, dimensions below 1024), they run on one cluster of
 * 16 CTAs (8 where the device schedules no cluster of 16): z and r in the
 * cluster's distributed shared memory, the colour passes separated by the
 * cluster's hardware barrier. The part below level 0 is then three launches:
 * the levels above the cluster's on the grid down to it, the cluster, and
 * back up on the grid. Asynchronous. */
dynmat_status dynmat_mg_apply(dynmat_mg_t M, const double* r, double* z, dynmat_stream_t stream);

/* Preconditioned CG on level 0 of M with one V-cycle as the preconditioner
 * (textbook PCG): per iteration q = A p and p.q, x += alpha p, r -= alpha q
 * and r.r (stop when ||r|| / ||r_0|| <= tol), z = M^{-1} r, r.z, p = z +
 * beta p. opts: tol, max_iters, check_every (iterations per CUDA graph);
 * precision must be CG_FP64. b, x as for cg_solve (x in: x0, out: solution).
 * Blocking; BREAKDOWN, NOT_CONVERGED as for cg_solve. */
dynmat_status pcg_solve(dynmat_mg_t M, const double* b, double* x, const cg_opts* opts,
                        cg_result* res, dynmat_stream_t stream);

/* ---------------------------------------------------------------------- */
/* Batches: many matrices in one persistent launch                         */
/* ---------------------------------------------------------------------- */

/* A batch has `max_slots` slots; each slot holds one matrix (a dynmat_t the
 * caller keeps alive and does not convert while it sits in the batch) in
 * DIA, ELL or CSR format with its own tile shape. Every phase over the batch
 * is one persistent kernel launch (a grid of resident blocks on every SM)
 * that takes row tiles of all slots from a device work list; launches are
 * replayed from CUDA graphs. Not thread-safe; one stream at a time. */
typedef struct dynmat_batch_s* dynmat_batch_t;

/* Tile shape of one matrix (the tuner's per-matrix choice, extending
 * §V-E's per-process format choice to the kernel's work decomposition):
 *  lanes: how a CSR row block is summed. 0 (the default): segmented; every
 *    lane sums a fixed run of 8 consecutive entries (each warp a contiguous
 *    range of runs), rows crossing runs being completed by a segmented scan
 *    over the lanes and rows crossing warps after one block barrier, so any
 *    mix of row lengths is balanced. 2, 4, 8, 16 or
 *    32: that many lanes per row, and a row longer than nnz_per_tile gets a
 *    tile of its own, reduced by a whole thread block;
 *  rows_per_tile: DIA / ELL rows per tile (a multiple of 1024);
 *  nnz_per_tile: CSR entries per row block (>= 256; default 16384). */
typedef struct {
  int32_t lanes;
  int32_t rows_per_tile;
  int32_t nnz_per_tile;
} dynmat_tile_shape;

dynmat_status dynmat_batch_create(dynmat_batch_t* out, int32_t max_slots, dynmat_stream_t stream);
dynmat_status dynmat_batch_destroy(dynmat_batch_t B, dynmat_stream_t stream);

/* Puts A (DIA, ELL or CSR) in `slot` for dynmat_batch_spmv with its vectors:
 * x (ncols) and y (nrows) device values of A's value type. shape NULL picks
 * a default from the row lengths; A NULL empties the slot. INVALID_ARG for
 * another format, or a CSR matrix of more than 2^31 - 65 entries. */
dynmat_status dynmat_batch_set(dynmat_batch_t B, int32_t slot, dynmat_t A,
                               const dynmat_tile_shape* shape, const void* x, void* y,
                               dynmat_stream_t stream);

/* y = A x for every matrix set in the batch, as one persistent launch
 * (a CUDA graph after the first call). Each row is summed by one thread
 * group in a fixed order: deterministic. Asynchronous. */
dynmat_status dynmat_batch_spmv(dynmat_batch_t B, dynmat_stream_t stream);

/* Per-matrix auto-tuner of a batch slot (§V-E's profiling tuner, run
 * online): times the slot's matrix in the batch kernel for every admissible
 * format (DIA and ELL within 3 x the CSR bytes, in 1024-row tiles; CSR in
 * several tile shapes, in that order), converts the matrix to the fastest
 * and keeps that shape; a later format must beat the best so far by 3%
 * (timing noise must not flip near-ties). The matrix is
 * timed as copies that together fill the GPU (about 4M rows), each with its
 * own x, y and matrix arrays (temporary device memory: the copies' vectors
 * and up to 2 GB of matrix clones). Blocking. */
dynmat_status dynmat_batch_autotune(dynmat_batch_t B, int32_t slot, dynmat_format* fmt_out,
                                    dynmat_tile_shape* shape_out, dynmat_stream_t stream);

/* The same tuner for a matrix outside any batch, e.g. when a server first
 * meets a matrix (the online tuning the paper leaves as future work, §VII):
 * converts A to the format that is fastest in the batch kernel and returns
 * the tile shape to pass to dynmat_batch_set / cg_batch_admit. effort 0: a
 * short probe of the format only, each in its default tile shape, copies of
 * about 1M rows; 1: the full sweep of dynmat_batch_autotune. Blocking. */
dynmat_status dynmat_batch_tune_matrix(dynmat_t A, int32_t effort, dynmat_format* fmt_out,
                                       dynmat_tile_shape* shape_out, dynmat_stream_t stream);

/* CG solves over a batch (the serving loop's primitives). A slot admitted
 * with cg_batch_admit runs CG on A x = b: b and x are caller-owned FP64
 * device vectors (x: start on entry for FP64, overwritten with 0 first for
 * MIXED; the solution when the slot finishes). FP64 needs F64 or F32
 * values; MIXED needs A with F32 values (exact values of the problem) and
 * runs FP32 inner CG iterations in the batch with FP64 residuals and
 * corrections between them, as cg_solve does. Each slot keeps its own
 * tiles, partial sums and scalars, so its iterates are bit-identical
 * whatever other slots share the batch. Work vectors are allocated at
 * admission (DYNMAT_ERR_OOM leaves the batch unchanged) and freed at
 * retirement. */
dynmat_status cg_batch_admit(dynmat_batch_t B, int32_t slot, dynmat_t A, const double* b,
                             double* x, const cg_opts* opts, const dynmat_tile_shape* shape,
                             dynmat_stream_t stream);

/* Advances every running slot by `iterations` CG iterations (one graph
 * launch of persistent SpMV+dot, update+dot and direction kernels per
 * iteration), then finishes outer refinement steps of MIXED slots whose
 * inner solve ended. done_flags (host, max_slots entries, may be NULL): 1
 * for slots whose solve is over. n_active (may be NULL): slots still
 * running. Blocking. */
dynmat_status cg_batch_step(dynmat_batch_t B, int32_t iterations, int32_t* done_flags,
                            int32_t* n_active, dynmat_stream_t stream);

/* Leaves running CG slot `slot` out of the following cg_batch_step calls
 * (paused = 1) or takes it back (paused = 0), so that a server can give the
 * GPU to some requests first (shortest remaining work). A paused slot's
 * state does not move; its iterates are the same bits as without the pause,
 * only later. No effect on a slot whose solve is over. Not in the paper: an
 * addition of the continuous-batching server. Errors: INVALID_ARG (no CG
 * solve in the slot, paused not 0 or 1). */
dynmat_status cg_batch_pause(dynmat_batch_t B, int32_t slot, int32_t paused,
                             dynmat_stream_t stream);

/* Result of a slot; res->status is -1 while it still runs. For a finished
 * slot the true relative residual is recomputed in FP64. Blocking. */
dynmat_status cg_batch_result(dynmat_batch_t B, int32_t slot, cg_result* res,
                              dynmat_stream_t stream);

/* Frees the slot's work vectors and empties it. */
dynmat_status cg_batch_retire(dynmat_batch_t B, int32_t slot, dynmat_stream_t stream);

/* ---------------------------------------------------------------------- */
/* Errors                                                                  */
/* ---------------------------------------------------------------------- */

/* Self-test of the bounded waits the kernels rely on (the stream kernels'
 * mbarrier waits, the smoother's grid barrier): runs a tiny kernel whose
 * wait nothing can satisfy, with a limit of `cycles` SM clock cycles
 * (at most 2^33). which = 0: a grid barrier in a two-block cooperative
 * launch whose second block leaves without arriving; which = 1: an
 * mbarrier that expects two arrivals and gets one. *timed_out = 1 when the
 * wait gave up and reported it (the expected outcome); the kernel returns
 * either way and the context stays usable. Blocking. */
dynmat_status dynmat_selftest_wait_timeout(int32_t which, int64_t cycles, int32_t* timed_out,
                                           dynmat_stream_t stream);

const char* dynmat_last_error(void);
const char* dynmat_status_string(dynmat_status s);

#ifdef __cplusplus
}
#endif

#endif /* DYNMAT_H */
