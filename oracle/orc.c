/*
 * CPU oracle for the dynamic sparse matrix method (arXiv 2209.06478).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow, single-threaded
 * FP64 statement of what the GPU path must compute. Only the tests, the
 * smoke check and the benchmark's CPU-baseline leg may load it. It shares
 * no code, header, table or helper with the CUDA library and includes none
 * of its headers; the two meet only through the seeded inputs of `synth`.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -shared -fPIC
 * (no FMA contraction, so every sum is rounded in the order written).
 * The same source built once more with -fopenmp (liborc_omp.so) is the
 * multi-core CPU baseline, standing for the paper's OpenMP backend (§III-D,
 * measured on CPU nodes in §V-D): the row loops of the CSR, DIA and ELL
 * products are split across threads. Each row's sum stays sequential and is
 * written by one thread, so both builds give bit-identical products; without
 * -fopenmp the pragmas are ignored.
 *
 * What each part follows:
 *  - COO, CSR (§II-A): three arrays; CSR compresses rows into pointers.
 *    Canonical order (our reading; §II-A leaves COO unordered and CSR
 *    columns unordered): entries sorted by (row, col).
 *  - DIA (§II-A): one column of coefficients per stored diagonal plus an
 *    offset array; stored here diagonal-major, val[d*nrows + i] =
 *    a(i, i + off[d]), zero where the entry is absent or outside the matrix.
 *  - ELL and HYB (§VI names them; ELL + COO overflow): slot-major arrays of
 *    width K, padding col = -1 / val = 0; HYB keeps each row's first K_h
 *    entries in ELL and the rest in COO.
 *  - Convert (§III-B): every conversion goes to COO and from COO.
 *  - multiply / SpMV (§III-D): y = A x summed per row in the natural order
 *    of the format.
 *  - Format selection (§V-E, "naive auto-tuner"; §IV-B picks the format at
 *    run time): a deterministic byte-model rule, our own reading.
 *  - CG (§II-B, §IV-B): HPCG's CG with the preconditioner disabled, i.e.
 *    textbook Hestenes-Stiefel CG.
 *  - Mixed-precision iterative refinement: FP32 inner CG, FP64 residual and
 *    update (not in the paper; the workload definition adds it).
 *
 * Parity pins: every function here is checked in tests/test_oracle_pins.py
 * against brute-force dense products, exact rational sums, the stencil's
 * closed forms (row sums, eigenpairs, spectrum-based CG bound), hand-written
 * golden arrays and round-trip identities.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Status values (same meaning as the library's, defined independently). */
enum {
  ORC_OK = 0,
  ORC_ERR_INVALID_ARG = 1,
  ORC_ERR_INDEX_RANGE = 2,
  ORC_ERR_DUPLICATE = 3,
  ORC_ERR_OOM = 4,
  ORC_ERR_FORMAT_TOO_LARGE = 5,
  ORC_ERR_BREAKDOWN = 7,
  ORC_ERR_NOT_CONVERGED = 8
};

enum { ORC_COO = 0, ORC_CSR = 1, ORC_DIA = 2, ORC_ELL = 3, ORC_HYB = 4 };

/* ------------------------------------------------------------------------ */
/* Canonical COO (§II-A; duplicates rejected, sorted by (row, col))          */
/* ------------------------------------------------------------------------ */

typedef struct {
  int64_t key;
  int64_t pos;
} orc_kp;

static int cmp_kp(const void* a, const void* b) {
  const orc_kp* x = (const orc_kp*)a;
  const orc_kp* y = (const orc_kp*)b;
  if (x->key < y->key) return -1;
  if (x->key > y->key) return 1;
  return 0;
}

/* Validates indices, sorts by (row, col) and rejects duplicate positions.
 * Index-range errors take precedence over duplicates. Output arrays may be
 * NULL to validate only. */
int orc_coo_canonical(int64_t nrows, int64_t ncols, int64_t nnz, const int32_t* row,
                      const int32_t* col, const double* val, int32_t* orow, int32_t* ocol,
                      double* oval) {
  if (nrows < 0 || ncols < 0 || nnz < 0) return ORC_ERR_INVALID_ARG;
  for (int64_t e = 0; e < nnz; ++e)
    if (row[e] < 0 || row[e] >= nrows || col[e] < 0 || col[e] >= ncols) return ORC_ERR_INDEX_RANGE;
  orc_kp* kp = (orc_kp*)malloc(sizeof(orc_kp) * (size_t)(nnz > 0 ? nnz : 1));
  if (!kp) return ORC_ERR_OOM;
  int sorted = 1;
  for (int64_t e = 0; e < nnz; ++e) {
    kp[e].key = (int64_t)row[e] * ncols + (int64_t)col[e];
    kp[e].pos = e;
    if (e > 0 && kp[e].key < kp[e - 1].key) sorted = 0;
  }
  if (!sorted) qsort(kp, (size_t)nnz, sizeof(orc_kp), cmp_kp);
  for (int64_t e = 1; e < nnz; ++e)
    if (kp[e].key == kp[e - 1].key) {
      free(kp);
      return ORC_ERR_DUPLICATE;
    }
  if (orow)
    for (int64_t e = 0; e < nnz; ++e) {
      orow[e] = row[kp[e].pos];
      ocol[e] = col[kp[e].pos];
      oval[e] = val[kp[e].pos];
    }
  free(kp);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* CSR <-> COO (§II-A, §III-B)                                               */
/* ------------------------------------------------------------------------ */

/* rowptr[i] = number of entries in rows < i; col/val are the COO arrays. */
void orc_coo_to_csr(int64_t nrows, int64_t nnz, const int32_t* row, int32_t* rowptr) {
  for (int64_t i = 0; i <= nrows; ++i) rowptr[i] = 0;
  for (int64_t e = 0; e < nnz; ++e) rowptr[row[e] + 1] += 1;
  for (int64_t i = 0; i < nrows; ++i) rowptr[i + 1] += rowptr[i];
}

void orc_csr_to_coo(int64_t nrows, const int32_t* rowptr, int32_t* row) {
  for (int64_t i = 0; i < nrows; ++i)
    for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e) row[e] = (int32_t)i;
}

/* ------------------------------------------------------------------------ */
/* DIA <-> COO (§II-A, §III-B)                                               */
/* ------------------------------------------------------------------------ */

/* Number of distinct diagonals (j - i) holding at least one stored entry. */
int64_t orc_dia_ndiag(int64_t nrows, int64_t ncols, int64_t nnz, const int32_t* row,
                      const int32_t* col) {
  int64_t span = nrows + ncols - 1;
  if (span <= 0) return 0;
  unsigned char* seen = (unsigned char*)calloc((size_t)span, 1);
  int64_t nd = 0;
  for (int64_t e = 0; e < nnz; ++e) {
    int64_t k = (int64_t)col[e] - (int64_t)row[e] + (nrows - 1);
    if (!seen[k]) {
      seen[k] = 1;
      ++nd;
    }
  }
  free(seen);
  return nd;
}

/* offsets[ndiag] ascending; dval[d*nrows + i] = a(i, i + offsets[d]) or 0. */
void orc_coo_to_dia(int64_t nrows, int64_t ncols, int64_t nnz, const int32_t* row,
                    const int32_t* col, const double* val, int32_t* offsets, double* dval) {
  int64_t span = nrows + ncols - 1;
  int64_t* slot = (int64_t*)malloc(sizeof(int64_t) * (size_t)(span > 0 ? span : 1));
  for (int64_t k = 0; k < span; ++k) slot[k] = -1;
  for (int64_t e = 0; e < nnz; ++e) slot[(int64_t)col[e] - row[e] + (nrows - 1)] = 0;
  int64_t nd = 0;
  for (int64_t k = 0; k < span; ++k)
    if (slot[k] == 0) {
      slot[k] = nd;
      offsets[nd] = (int32_t)(k - (nrows - 1));
      ++nd;
    }
  for (int64_t s = 0; s < nd * nrows; ++s) dval[s] = 0.0;
  for (int64_t e = 0; e < nnz; ++e) {
    int64_t d = slot[(int64_t)col[e] - row[e] + (nrows - 1)];
    dval[d * nrows + row[e]] = val[e];
  }
  free(slot);
}

/* Emits, row by row and within a row by ascending offset (= ascending column),
 * the slots that lie inside the matrix and hold a value other than zero
 * (+0.0 and -0.0 both count as padding). Returns the count; the output
 * arrays may be NULL to count only. */
int64_t orc_dia_to_coo(int64_t nrows, int64_t ncols, int64_t ndiag, const int32_t* offsets,
                       const double* dval, int32_t* orow, int32_t* ocol, double* oval) {
  int64_t m = 0;
  for (int64_t i = 0; i < nrows; ++i)
    for (int64_t d = 0; d < ndiag; ++d) {
      int64_t j = i + offsets[d];
      if (j < 0 || j >= ncols) continue;
      double v = dval[d * nrows + i];
      if (v == 0.0) continue;
      if (orow) {
        orow[m] = (int32_t)i;
        ocol[m] = (int32_t)j;
        oval[m] = v;
      }
      ++m;
    }
  return m;
}

/* ------------------------------------------------------------------------ */
/* ELL and HYB <-> COO (§VI: ELL; HYB = ELL + COO)                           */
/* ------------------------------------------------------------------------ */

int64_t orc_max_row_length(int64_t nrows, int64_t nnz, const int32_t* row) {
  int64_t* len = (int64_t*)calloc((size_t)(nrows > 0 ? nrows : 1), sizeof(int64_t));
  int64_t mx = 0;
  for (int64_t e = 0; e < nnz; ++e) len[row[e]] += 1;
  for (int64_t i = 0; i < nrows; ++i)
    if (len[i] > mx) mx = len[i];
  free(len);
  return mx;
}

/* Slot k of row i holds the row's k-th entry in column order:
 * ecol[k*nrows + i], eval[k*nrows + i]; padding col = -1, val = 0. */
void orc_coo_to_ell(int64_t nrows, int64_t nnz, const int32_t* row, const int32_t* col,
                    const double* val, int64_t K, int32_t* ecol, double* eval) {
  for (int64_t s = 0; s < K * nrows; ++s) {
    ecol[s] = -1;
    eval[s] = 0.0;
  }
  int64_t* fill = (int64_t*)calloc((size_t)(nrows > 0 ? nrows : 1), sizeof(int64_t));
  for (int64_t e = 0; e < nnz; ++e) {
    int64_t i = row[e];
    int64_t k = fill[i]++;
    ecol[k * nrows + i] = col[e];
    eval[k * nrows + i] = val[e];
  }
  free(fill);
}

int64_t orc_ell_to_coo(int64_t nrows, int64_t K, const int32_t* ecol, const double* eval,
                       int32_t* orow, int32_t* ocol, double* oval) {
  int64_t m = 0;
  for (int64_t i = 0; i < nrows; ++i)
    for (int64_t k = 0; k < K; ++k) {
      int32_t c = ecol[k * nrows + i];
      if (c < 0) continue;
      if (orow) {
        orow[m] = (int32_t)i;
        ocol[m] = c;
        oval[m] = eval[k * nrows + i];
      }
      ++m;
    }
  return m;
}

/* HYB width (our rule; the paper gives none): the k in [0, maxlen] that
 * minimises the modelled bytes slot*k*nrows + over*sum_i max(0, len_i - k),
 * with slot = 4 + vbytes (ELL: index + value per padded slot) and
 * over = 8 + vbytes (COO: two indices + value per overflow entry); ties go
 * to the smaller k. `over_out` receives sum_i max(0, len_i - K_h). */
int64_t orc_hyb_width(int64_t nrows, int64_t nnz, const int32_t* row, int64_t vbytes,
                      int64_t* over_out) {
  int64_t* len = (int64_t*)calloc((size_t)(nrows > 0 ? nrows : 1), sizeof(int64_t));
  for (int64_t e = 0; e < nnz; ++e) len[row[e]] += 1;
  int64_t maxlen = 0;
  for (int64_t i = 0; i < nrows; ++i)
    if (len[i] > maxlen) maxlen = len[i];
  int64_t* cnt = (int64_t*)calloc((size_t)(maxlen + 1), sizeof(int64_t));
  for (int64_t i = 0; i < nrows; ++i) cnt[len[i]] += 1;
  int64_t best_k = 0, best_cost = -1, best_over = 0;
  for (int64_t k = 0; k <= maxlen; ++k) {
    int64_t over = 0;
    for (int64_t l = k + 1; l <= maxlen; ++l) over += (l - k) * cnt[l];
    int64_t cost = (4 + vbytes) * k * nrows + (8 + vbytes) * over;
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best_k = k;
      best_over = over;
    }
  }
  free(cnt);
  free(len);
  if (over_out) *over_out = best_over;
  return best_k;
}

/* ELL part: each row's first min(len, Kh) entries (slot-major as in ELL);
 * COO part: the remaining entries in (row, col) order. */
void orc_coo_to_hyb(int64_t nrows, int64_t nnz, const int32_t* row, const int32_t* col,
                    const double* val, int64_t Kh, int32_t* ecol, double* eval, int32_t* crow,
                    int32_t* ccol, double* cval) {
  for (int64_t s = 0; s < Kh * nrows; ++s) {
    ecol[s] = -1;
    eval[s] = 0.0;
  }
  int64_t* fill = (int64_t*)calloc((size_t)(nrows > 0 ? nrows : 1), sizeof(int64_t));
  int64_t m = 0;
  for (int64_t e = 0; e < nnz; ++e) {
    int64_t i = row[e];
    int64_t k = fill[i]++;
    if (k < Kh) {
      ecol[k * nrows + i] = col[e];
      eval[k * nrows + i] = val[e];
    } else {
      crow[m] = row[e];
      ccol[m] = col[e];
      cval[m] = val[e];
      ++m;
    }
  }
  free(fill);
}

/* Row by row: the ELL slots in slot order, then that row's COO entries. */
int64_t orc_hyb_to_coo(int64_t nrows, int64_t Kh, const int32_t* ecol, const double* eval,
                       int64_t ncoo, const int32_t* crow, const int32_t* ccol, const double* cval,
                       int32_t* orow, int32_t* ocol, double* oval) {
  int64_t m = 0, c = 0;
  for (int64_t i = 0; i < nrows; ++i) {
    for (int64_t k = 0; k < Kh; ++k) {
      int32_t cc = ecol[k * nrows + i];
      if (cc < 0) continue;
      if (orow) {
        orow[m] = (int32_t)i;
        ocol[m] = cc;
        oval[m] = eval[k * nrows + i];
      }
      ++m;
    }
    while (c < ncoo && crow[c] == i) {
      if (orow) {
        orow[m] = crow[c];
        ocol[m] = ccol[c];
        oval[m] = cval[c];
      }
      ++m;
      ++c;
    }
  }
  return m;
}

/* ------------------------------------------------------------------------ */
/* Features and the deterministic format rule (§IV-B run-time choice,        */
/* §V-E auto-tuner; the byte model and the guard are our reading)            */
/* ------------------------------------------------------------------------ */

typedef struct {
  int64_t nrows, ncols, nnz, ndiag, maxlen, hyb_k, hyb_over;
  int64_t bytes[5]; /* modelled bytes per format, indexed by ORC_COO..ORC_HYB */
  int64_t choice;   /* selected format */
} orc_features;

/* Modelled bytes of each format with `vbytes`-byte values and 4-byte indices:
 *   COO = (8 + v) nnz                CSR = (4 + v) nnz + 4 (nrows + 1)
 *   DIA = v ndiag nrows + 4 ndiag    ELL = (4 + v) maxlen nrows
 *   HYB = (4 + v) K_h nrows + (8 + v) overflow
 * A padded format (DIA, ELL) whose bytes exceed guard x CSR bytes is
 * excluded. The smallest remaining wins; ties go in the order
 * DIA, ELL, CSR, HYB, COO. All integer. */
void orc_features_select(int64_t nrows, int64_t ncols, int64_t nnz, const int32_t* row,
                         const int32_t* col, int64_t vbytes, int64_t guard, orc_features* f) {
  f->nrows = nrows;
  f->ncols = ncols;
  f->nnz = nnz;
  f->ndiag = orc_dia_ndiag(nrows, ncols, nnz, row, col);
  f->maxlen = orc_max_row_length(nrows, nnz, row);
  f->hyb_k = orc_hyb_width(nrows, nnz, row, vbytes, &f->hyb_over);
  int64_t v = vbytes;
  f->bytes[ORC_COO] = (8 + v) * nnz;
  f->bytes[ORC_CSR] = (4 + v) * nnz + 4 * (nrows + 1);
  f->bytes[ORC_DIA] = v * f->ndiag * nrows + 4 * f->ndiag;
  f->bytes[ORC_ELL] = (4 + v) * f->maxlen * nrows;
  f->bytes[ORC_HYB] = (4 + v) * f->hyb_k * nrows + (8 + v) * f->hyb_over;
  const int order[5] = {ORC_DIA, ORC_ELL, ORC_CSR, ORC_HYB, ORC_COO};
  int64_t best = -1;
  for (int t = 0; t < 5; ++t) {
    int fmt = order[t];
    if ((fmt == ORC_DIA || fmt == ORC_ELL) && f->bytes[fmt] > guard * f->bytes[ORC_CSR]) continue;
    if (best < 0 || f->bytes[fmt] < f->bytes[best]) best = fmt;
  }
  f->choice = best;
}

/* ------------------------------------------------------------------------ */
/* Diagonal extraction and update (§III-D: every container supports them;  */
/* §IV-B: HPCG's CG test modifies the matrix diagonal), on canonical COO    */
/* ------------------------------------------------------------------------ */

/* d[i] = a(i, i) for i < n = min(nrows, ncols); 0.0 where (i, i) is not
 * stored. Returns the number of stored diagonal entries. */
int64_t orc_diagonal(int64_t nrows, int64_t ncols, int64_t nnz, const int32_t* row,
                     const int32_t* col, const double* val, double* d) {
  const int64_t n = nrows < ncols ? nrows : ncols;
  int64_t found = 0;
  for (int64_t i = 0; i < n; ++i) d[i] = 0.0;
  for (int64_t e = 0; e < nnz; ++e)
    if (row[e] == col[e]) {
      d[row[e]] = val[e];
      ++found;
    }
  return found;
}

/* Sets every stored (i, i) entry to d[i] (the structure is unchanged).
 * Returns the number of entries set. */
int64_t orc_set_diagonal(int64_t nnz, const int32_t* row, const int32_t* col, double* val,
                         const double* d) {
  int64_t set = 0;
  for (int64_t e = 0; e < nnz; ++e)
    if (row[e] == col[e]) {
      val[e] = d[row[e]];
      ++set;
    }
  return set;
}

/* ------------------------------------------------------------------------ */
/* SpMV y = A x (§III-D "multiply"), one per format, FP64                    */
/* ------------------------------------------------------------------------ */

/* Threads the row loops below may use: 1 in the serial build. */
int64_t orc_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}


void orc_spmv_coo(int64_t nrows, int64_t nnz, const int32_t* row, const int32_t* col,
                  const double* val, const double* x, double* y) {
  for (int64_t i = 0; i < nrows; ++i) y[i] = 0.0;
  for (int64_t e = 0; e < nnz; ++e) y[row[e]] = y[row[e]] + val[e] * x[col[e]];
}

void orc_spmv_csr(int64_t nrows, const int32_t* rowptr, const int32_t* col, const double* val,
                  const double* x, double* y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < nrows; ++i) {
    double s = 0.0;
    for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e) s = s + val[e] * x[col[e]];
    y[i] = s;
  }
}

/* Over diagonals in ascending offset order, padded zeros included. */
void orc_spmv_dia(int64_t nrows, int64_t ncols, int64_t ndiag, const int32_t* offsets,
                  const double* dval, const double* x, double* y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < nrows; ++i) {
    double s = 0.0;
    for (int64_t d = 0; d < ndiag; ++d) {
      int64_t j = i + offsets[d];
      if (j >= 0 && j < ncols) s = s + dval[d * nrows + i] * x[j];
    }
    y[i] = s;
  }
}

void orc_spmv_ell(int64_t nrows, int64_t K, const int32_t* ecol, const double* eval,
                  const double* x, double* y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < nrows; ++i) {
    double s = 0.0;
    for (int64_t k = 0; k < K; ++k) {
      int32_t c = ecol[k * nrows + i];
      if (c >= 0) s = s + eval[k * nrows + i] * x[c];
    }
    y[i] = s;
  }
}

/* ELL slots, then the row's COO entries. */
void orc_spmv_hyb(int64_t nrows, int64_t Kh, const int32_t* ecol, const double* eval,
                  int64_t ncoo, const int32_t* crow, const int32_t* ccol, const double* cval,
                  const double* x, double* y) {
  orc_spmv_ell(nrows, Kh, ecol, eval, x, y);
  for (int64_t e = 0; e < ncoo; ++e) y[crow[e]] = y[crow[e]] + cval[e] * x[ccol[e]];
}

/* Reduced-precision product used by the mixed-precision inner solve:
 * float values, float x, float accumulation, entries in column order. */
void orc_spmv_csr_f32(int64_t nrows, const int32_t* rowptr, const int32_t* col, const float* val,
                      const float* x, float* y) {
  for (int64_t i = 0; i < nrows; ++i) {
    float s = 0.0f;
    for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e) s = s + val[e] * x[col[e]];
    y[i] = s;
  }
}

/* ------------------------------------------------------------------------ */
/* Conjugate gradient (§II-B HPCG; §IV-B: preconditioner disabled)           */
/* ------------------------------------------------------------------------ */

static double dot_seq(int64_t n, const double* a, const double* b) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s = s + a[i] * b[i];
  return s;
}

/* Textbook CG on A x = b (A in CSR), starting from the x passed in.
 *   r = b - A x; p = r; rho = r.r; stop at once if rho == 0.
 *   per iteration: q = A p; sigma = p.q (<= 0 -> breakdown);
 *   alpha = rho / sigma; x += alpha p; r -= alpha q; rho' = r.r;
 *   stop when sqrt(rho') / sqrt(rho_0) <= tol; beta = rho'/rho; p = r + beta p.
 * Outputs: iterations done, the recursive relative residual and the true one
 * ||b - A x|| / ||b|| (||r_0|| when b = 0 is impossible: rho_0 = 0 returns
 * early). `hist` (may be NULL) receives sqrt(rho_k)/sqrt(rho_0), k = 0..its. */
int orc_cg_csr(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val,
               const double* b, double* x, double tol, int64_t max_iters, int64_t* iters_out,
               double* relres_out, double* true_relres_out, double* hist) {
  double* r = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* p = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* q = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  int status = ORC_ERR_NOT_CONVERGED;
  int64_t k = 0;
  orc_spmv_csr(n, rowptr, col, val, x, q);
  for (int64_t i = 0; i < n; ++i) {
    r[i] = b[i] - q[i];
    p[i] = r[i];
  }
  double rho = dot_seq(n, r, r);
  double r0 = sqrt(rho);
  double rel = 0.0;
  if (hist) hist[0] = 1.0;
  if (r0 == 0.0) {
    status = ORC_OK;
  } else {
    rel = 1.0;
    for (k = 1; k <= max_iters; ++k) {
      orc_spmv_csr(n, rowptr, col, val, p, q);
      double sigma = dot_seq(n, p, q);
      if (!(sigma > 0.0)) {
        status = ORC_ERR_BREAKDOWN;
        --k;
        break;
      }
      double alpha = rho / sigma;
      for (int64_t i = 0; i < n; ++i) x[i] = x[i] + alpha * p[i];
      for (int64_t i = 0; i < n; ++i) r[i] = r[i] - alpha * q[i];
      double rho_new = dot_seq(n, r, r);
      rel = sqrt(rho_new) / r0;
      if (hist) hist[k] = rel;
      if (rel <= tol) {
        status = ORC_OK;
        break;
      }
      double beta = rho_new / rho;
      for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
      rho = rho_new;
    }
    if (k > max_iters) k = max_iters;
  }
  /* true residual */
  orc_spmv_csr(n, rowptr, col, val, x, q);
  double rr = 0.0, bb = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double t = b[i] - q[i];
    rr = rr + t * t;
    bb = bb + b[i] * b[i];
  }
  if (iters_out) *iters_out = k;
  if (relres_out) *relres_out = rel;
  if (true_relres_out) *true_relres_out = bb > 0.0 ? sqrt(rr) / sqrt(bb) : sqrt(rr);
  free(r);
  free(p);
  free(q);
  return status;
}

/* ------------------------------------------------------------------------ */
/* Mixed-precision iterative refinement (FP32 inner CG, FP64 outer)          */
/* ------------------------------------------------------------------------ */

static double dot_f32_in_f64(int64_t n, const float* a, const float* b) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s = s + (double)a[i] * (double)b[i];
  return s;
}

/* Outer loop, x = 0 in FP64:
 *   r = b - A x (FP64 values `val`, FP64 sums); stop when ||r||/||b|| <= tol;
 *   inner CG in FP32 on A d = (float) r from d = 0 with FP32 values
 *   (float) val, FP32 SpMV sums and FP32 vector updates; its dot products are
 *   summed in FP64 and alpha, beta are formed in FP64 and rounded to float
 *   for the updates; it stops when ||r_in|| / ||r_in,0|| <= inner_tol or after
 *   inner_max iterations (or on sigma <= 0);
 *   x += (double) d.
 * Returns NOT_CONVERGED after max_outer refinements. */
int orc_ir_mixed_csr(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                     const double* b, double* x, double tol, double inner_tol, int64_t inner_max,
                     int64_t max_outer, int64_t* outer_out, int64_t* inner_total_out,
                     double* true_relres_out) {
  size_t nn = (size_t)(n > 0 ? n : 1);
  int64_t nnz = rowptr[n];
  float* v32 = (float*)malloc(sizeof(float) * (size_t)(nnz > 0 ? nnz : 1));
  for (int64_t e = 0; e < nnz; ++e) v32[e] = (float)val[e];
  double* r = (double*)malloc(sizeof(double) * nn);
  double* ax = (double*)malloc(sizeof(double) * nn);
  float* rf = (float*)malloc(sizeof(float) * nn);
  float* d = (float*)malloc(sizeof(float) * nn);
  float* p = (float*)malloc(sizeof(float) * nn);
  float* q = (float*)malloc(sizeof(float) * nn);
  for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
  double bn = sqrt(dot_seq(n, b, b));
  int status = ORC_ERR_NOT_CONVERGED;
  int64_t outer = 0, inner_total = 0;
  double rel = 0.0;
  for (;;) {
    orc_spmv_csr(n, rowptr, col, val, x, ax);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - ax[i];
    double rn = sqrt(dot_seq(n, r, r));
    rel = bn > 0.0 ? rn / bn : rn;
    if (rel <= tol) {
      status = ORC_OK;
      break;
    }
    if (outer >= max_outer) break;
    ++outer;
    for (int64_t i = 0; i < n; ++i) {
      rf[i] = (float)r[i];
      d[i] = 0.0f;
      p[i] = rf[i];
    }
    double rho = dot_f32_in_f64(n, rf, rf);
    double r0 = sqrt(rho);
    for (int64_t k = 1; k <= inner_max && r0 > 0.0; ++k) {
      orc_spmv_csr_f32(n, rowptr, col, v32, p, q);
      double sigma = dot_f32_in_f64(n, p, q);
      if (!(sigma > 0.0)) break;
      float alpha = (float)(rho / sigma);
      for (int64_t i = 0; i < n; ++i) d[i] = d[i] + alpha * p[i];
      for (int64_t i = 0; i < n; ++i) rf[i] = rf[i] - alpha * q[i];
      double rho_new = dot_f32_in_f64(n, rf, rf);
      ++inner_total;
      if (sqrt(rho_new) / r0 <= inner_tol) break;
      float beta = (float)(rho_new / rho);
      for (int64_t i = 0; i < n; ++i) p[i] = rf[i] + beta * p[i];
      rho = rho_new;
    }
    for (int64_t i = 0; i < n; ++i) x[i] = x[i] + (double)d[i];
  }
  if (outer_out) *outer_out = outer;
  if (inner_total_out) *inner_total_out = inner_total;
  if (true_relres_out) *true_relres_out = rel;
  free(v32);
  free(r);
  free(ax);
  free(rf);
  free(d);
  free(p);
  free(q);
  return status;
}

/* Mixed precision with reliable updates: one FP32 CG (FP32 values, FP32
 * vectors and SpMV sums, dot products summed in FP64, alpha and beta formed in
 * FP64 and rounded to float for the updates) whose correction d is folded
 * into the FP64 solution, with the residual recomputed in FP64, whenever the
 * recursive residual has dropped by `delta` since the last fold, or looks
 * converged, or the iteration limit is reached. The search direction is kept
 * across folds (no restart).
 *   x = 0; r = b; bn = ||b||; r32 = (float) r; p = r32; d = 0;
 *   rho = r.r (FP64, of the FP64 residual); rmax = sqrt(rho)
 *   for k = 1..max_iters:
 *     q = A32 p; sigma = p.q; sigma <= 0 -> breakdown
 *     alpha = rho / sigma; d += alpha p; r32 -= alpha q; rho' = r32.r32
 *     if sqrt(rho') < delta rmax or sqrt(rho') <= tol bn or k == max_iters:
 *       x += (double) d; d = 0; r = b - A x (FP64 values and sums);
 *       r32 = (float) r; rho' = r.r (FP64); rmax = sqrt(rho')
 *       if sqrt(rho') <= tol bn: converged; else if k == max_iters: not converged
 *     beta = rho' / rho; p = r32 + beta p; rho = rho'
 * `iters_out` receives k, `folds_out` the number of folds. */
int orc_cg_reliable_csr(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                        const double* b, double* x, double tol, double delta, int64_t max_iters,
                        int64_t* iters_out, int64_t* folds_out, double* true_relres_out) {
  size_t nn = (size_t)(n > 0 ? n : 1);
  int64_t nnz = rowptr[n];
  float* v32 = (float*)malloc(sizeof(float) * (size_t)(nnz > 0 ? nnz : 1));
  for (int64_t e = 0; e < nnz; ++e) v32[e] = (float)val[e];
  double* r = (double*)malloc(sizeof(double) * nn);
  double* ax = (double*)malloc(sizeof(double) * nn);
  float* rf = (float*)malloc(sizeof(float) * nn);
  float* d = (float*)malloc(sizeof(float) * nn);
  float* p = (float*)malloc(sizeof(float) * nn);
  float* q = (float*)malloc(sizeof(float) * nn);
  for (int64_t i = 0; i < n; ++i) {
    x[i] = 0.0;
    r[i] = b[i];
    rf[i] = (float)r[i];
    p[i] = rf[i];
    d[i] = 0.0f;
  }
  double bn = sqrt(dot_seq(n, b, b));
  double rho = dot_seq(n, r, r);
  double rmax = sqrt(rho);
  double rel = bn > 0.0 ? rmax / bn : 0.0;
  int status = ORC_ERR_NOT_CONVERGED;
  int64_t k = 0, folds = 0;
  const int zero_rhs = rmax == 0.0;
  if (zero_rhs) status = ORC_OK;
  for (k = 1; !zero_rhs && k <= max_iters; ++k) {
    orc_spmv_csr_f32(n, rowptr, col, v32, p, q);
    double sigma = dot_f32_in_f64(n, p, q);
    if (!(sigma > 0.0)) {
      status = ORC_ERR_BREAKDOWN;
      break;
    }
    float alpha = (float)(rho / sigma);
    for (int64_t i = 0; i < n; ++i) d[i] = d[i] + alpha * p[i];
    for (int64_t i = 0; i < n; ++i) rf[i] = rf[i] - alpha * q[i];
    double rho_new = dot_f32_in_f64(n, rf, rf);
    double rn = sqrt(rho_new);
    if (rn < delta * rmax || rn <= tol * bn || k == max_iters) {
      for (int64_t i = 0; i < n; ++i) {
        x[i] = x[i] + (double)d[i];
        d[i] = 0.0f;
      }
      ++folds;
      orc_spmv_csr(n, rowptr, col, val, x, ax);
      for (int64_t i = 0; i < n; ++i) {
        r[i] = b[i] - ax[i];
        rf[i] = (float)r[i];
      }
      rho_new = dot_seq(n, r, r);
      rmax = sqrt(rho_new);
      rel = bn > 0.0 ? rmax / bn : rmax;
      if (rmax <= tol * bn) {
        status = ORC_OK;
        break;
      }
    }
    float beta = (float)(rho_new / rho);
    for (int64_t i = 0; i < n; ++i) p[i] = rf[i] + beta * p[i];
    rho = rho_new;
  }
  if (k > max_iters) k = max_iters;
  if (zero_rhs) k = 0;
  if (iters_out) *iters_out = (status == ORC_ERR_BREAKDOWN) ? k - 1 : k;
  if (folds_out) *folds_out = folds;
  if (true_relres_out) *true_relres_out = rel;
  free(v32);
  free(r);
  free(ax);
  free(rf);
  free(d);
  free(p);
  free(q);
  return status;
}

/* ------------------------------------------------------------------------ */
/* HPCG's preconditioned CG (§II-B: PCG with a symmetric Gauss-Seidel        */
/* smoother inside a multigrid preconditioner; the paper runs it with the    */
/* preconditioner disabled, §IV-B). Readings, as stated:                     */
/*  - grids: level l is an nx_l x ny_l x nz_l stencil grid (rows x fastest), */
/*    level l+1 has half the points in each dimension; coarse point          */
/*    (i, j, k) is fine point (2i, 2j, 2k);                                  */
/*  - symmetric Gauss-Seidel in colour order: colour(i) = 7 - ((ix & 1) +   */
/*    2 (iy & 1) + 4 (iz & 1)) (no two stencil neighbours share a colour);   */
/*    a forward pass takes colours 0..7, a backward pass 7..0, rows of a     */
/*    colour in increasing index (their order does not matter). The points  */
/*    with every coordinate even (the coarse grid's points) are colour 7:    */
/*    the last colour of a sweep has zero residual afterwards, and           */
/*    injection would then hand the coarse grid a zero right-hand side;      */
/*    z_i = (r_i - sum_{j != i} a_ij z_j) / a_ii, the sum in column order;   */
/*  - V-cycle on level l: z = 0; the coarsest level is one sweep; otherwise  */
/*    pre-smooth (one sweep), t = r - A z, coarse r = t at the coarse        */
/*    points (injection), the coarse V-cycle, z += coarse z at the coarse    */
/*    points, post-smooth (one sweep);                                       */
/*  - PCG: textbook preconditioned CG (Saad §9.2), stopping on the           */
/*    recursive residual ||r_k|| / ||r_0|| <= tol.                           */
/* ------------------------------------------------------------------------ */

typedef struct {
  int64_t nx, ny, nz;
  const int32_t* rowptr;
  const int32_t* col;
  const double* val;
} orc_level;

static void symgs_sweep(const orc_level* L, const double* r, double* z) {
  const int64_t n = L->nx * L->ny * L->nz;
  for (int pass = 0; pass < 2; ++pass)
    for (int cc = 0; cc < 8; ++cc) {
      const int c = pass == 0 ? cc : 7 - cc;
      for (int64_t i = 0; i < n; ++i) {
        const int64_t ix = i % L->nx, iy = (i / L->nx) % L->ny, iz = i / (L->nx * L->ny);
        if (7 - (int)((ix & 1) + 2 * (iy & 1) + 4 * (iz & 1)) != c) continue;
        double s = r[i], diag = 0.0;
        for (int32_t e = L->rowptr[i]; e < L->rowptr[i + 1]; ++e) {
          if (L->col[e] == i)
            diag = L->val[e];
          else
            s = s - L->val[e] * z[L->col[e]];
        }
        z[i] = s / diag;
      }
    }
}

/* One symmetric Gauss-Seidel sweep on level data (z updated in place). */
void orc_symgs(int64_t nx, int64_t ny, int64_t nz, const int32_t* rowptr, const int32_t* col,
               const double* val, const double* r, double* z) {
  orc_level L = {nx, ny, nz, rowptr, col, val};
  symgs_sweep(&L, r, z);
}

static void vcycle(const orc_level* lv, int64_t nlev, int64_t l, const double* r, double* z) {
  const orc_level* L = lv + l;
  const int64_t n = L->nx * L->ny * L->nz;
  for (int64_t i = 0; i < n; ++i) z[i] = 0.0;
  if (l == nlev - 1) {
    symgs_sweep(L, r, z);
    return;
  }
  const orc_level* C = lv + l + 1;
  const int64_t nc = C->nx * C->ny * C->nz;
  double* t = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* rc = (double*)malloc(sizeof(double) * (size_t)(nc > 0 ? nc : 1));
  double* zc = (double*)malloc(sizeof(double) * (size_t)(nc > 0 ? nc : 1));
  symgs_sweep(L, r, z);
  orc_spmv_csr(n, L->rowptr, L->col, L->val, z, t);
  for (int64_t i = 0; i < n; ++i) t[i] = r[i] - t[i];
  for (int64_t ic = 0; ic < nc; ++ic) {
    const int64_t cx = ic % C->nx, cy = (ic / C->nx) % C->ny, cz = ic / (C->nx * C->ny);
    rc[ic] = t[2 * cx + L->nx * (2 * cy + L->ny * 2 * cz)];
  }
  vcycle(lv, nlev, l + 1, rc, zc);
  for (int64_t ic = 0; ic < nc; ++ic) {
    const int64_t cx = ic % C->nx, cy = (ic / C->nx) % C->ny, cz = ic / (C->nx * C->ny);
    const int64_t f = 2 * cx + L->nx * (2 * cy + L->ny * 2 * cz);
    z[f] = z[f] + zc[ic];
  }
  symgs_sweep(L, r, z);
  free(t);
  free(rc);
  free(zc);
}

static void load_levels(orc_level* lv, int64_t nlev, const int64_t* dims,
                        const int32_t* const* rowptr, const int32_t* const* col,
                        const double* const* val) {
  for (int64_t l = 0; l < nlev; ++l) {
    lv[l].nx = dims[3 * l];
    lv[l].ny = dims[3 * l + 1];
    lv[l].nz = dims[3 * l + 2];
    lv[l].rowptr = rowptr[l];
    lv[l].col = col[l];
    lv[l].val = val[l];
  }
}

/* z = M^{-1} r: one V-cycle over nlev levels (nlev = 1: one sweep). */
void orc_mg_apply(int64_t nlev, const int64_t* dims, const int32_t* const* rowptr,
                  const int32_t* const* col, const double* const* val, const double* r, double* z) {
  orc_level lv[16];
  load_levels(lv, nlev, dims, rowptr, col, val);
  vcycle(lv, nlev, 0, r, z);
}

/* PCG on level 0 with the V-cycle as preconditioner; nlev = 0 takes M = I
 * (z = r), which reproduces orc_cg_csr. Same outputs as orc_cg_csr. */
int orc_pcg(int64_t nlev, const int64_t* dims, const int32_t* const* rowptr,
            const int32_t* const* col, const double* const* val, const double* b, double* x,
            double tol, int64_t max_iters, int64_t* iters_out, double* relres_out,
            double* true_relres_out, double* hist) {
  orc_level lv[16];
  const int64_t use = nlev > 0 ? nlev : 1;
  load_levels(lv, use, dims, rowptr, col, val);
  const orc_level* A = lv;
  const int64_t n = A->nx * A->ny * A->nz;
  const size_t sz = sizeof(double) * (size_t)(n > 0 ? n : 1);
  double *r = (double*)malloc(sz), *z = (double*)malloc(sz), *p = (double*)malloc(sz),
         *q = (double*)malloc(sz);
  int status = ORC_ERR_NOT_CONVERGED;
  int64_t k = 0;
  orc_spmv_csr(n, A->rowptr, A->col, A->val, x, q);
  for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
  double rr = dot_seq(n, r, r);
  const double r0 = sqrt(rr);
  double rel = 0.0;
  if (hist) hist[0] = 1.0;
  if (r0 == 0.0) {
    status = ORC_OK;
  } else {
    rel = 1.0;
    if (nlev > 0) vcycle(lv, nlev, 0, r, z); else for (int64_t i = 0; i < n; ++i) z[i] = r[i];
    for (int64_t i = 0; i < n; ++i) p[i] = z[i];
    double rz = dot_seq(n, r, z);
    for (k = 1; k <= max_iters; ++k) {
      orc_spmv_csr(n, A->rowptr, A->col, A->val, p, q);
      const double sigma = dot_seq(n, p, q);
      if (!(sigma > 0.0)) {
        status = ORC_ERR_BREAKDOWN;
        --k;
        break;
      }
      const double alpha = rz / sigma;
      for (int64_t i = 0; i < n; ++i) x[i] = x[i] + alpha * p[i];
      for (int64_t i = 0; i < n; ++i) r[i] = r[i] - alpha * q[i];
      rr = dot_seq(n, r, r);
      rel = sqrt(rr) / r0;
      if (hist) hist[k] = rel;
      if (rel <= tol) {
        status = ORC_OK;
        break;
      }
      if (nlev > 0) vcycle(lv, nlev, 0, r, z); else for (int64_t i = 0; i < n; ++i) z[i] = r[i];
      const double rz_new = dot_seq(n, r, z);
      const double beta = rz_new / rz;
      for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
      rz = rz_new;
    }
    if (k > max_iters) k = max_iters;
  }
  orc_spmv_csr(n, A->rowptr, A->col, A->val, x, q);
  double tr = 0.0, bb = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    const double t = b[i] - q[i];
    tr = tr + t * t;
    bb = bb + b[i] * b[i];
  }
  if (iters_out) *iters_out = k;
  if (relres_out) *relres_out = rel;
  if (true_relres_out) *true_relres_out = bb > 0.0 ? sqrt(tr) / sqrt(bb) : sqrt(tr);
  free(r);
  free(z);
  free(p);
  free(q);
  return status;
}
