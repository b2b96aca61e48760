/*
 * CPU oracle for the CSRC sparse matrix-vector product.
 *
 * TEST INFRASTRUCTURE ONLY. Tests, the smoke check and the benchmark's CPU
 * baseline call this code. The library's product path never does. It shares no
 * code, headers or tables with the CUDA library.
 *
 * Plain, single-threaded FP64 C, compiled with -O2 -ffp-contract=off so that no
 * multiply-add is fused: every operation is one IEEE-754 double rounding, and
 * the results are the same on x86-64 and AArch64. Indices are 0-based.
 *
 * Paper: Batista, Ainsworth Jr., Ribeiro, "Parallel structurally-symmetric
 * sparse matrix-vector products on multi-core processors" (arXiv:1003.0952).
 *
 * Pins (tests/test_oracle_*.py): dense brute force on small matrices, integer-valued
 * exactness, stencil closed forms, the transpose and bilinear identities,
 * Table 1 working sets, and partition/colouring invariants. Parity for the 9x9
 * example of Fig. 1 is unpinned because the figure is missing.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ------------------------------------------------------------------------- */
/* Section 2 (CSRC format). A = A_D + A_L + A_U. For every stored entry a_ij
 * with j < i, al holds a_ij and au holds its mirror a_ji at the same position.
 * ia(i) points at row i's first entry and ja holds the column of each A_L entry
 * (= the row of each A_U entry). ad holds the diagonal. The number of stored
 * pairs is k = (nnz - n)/2. */

/* Count the strictly-lower entries of a CSR matrix (the number of CSRC pairs). */
int64_t oracle_count_lower(int64_t n, const int64_t* row_ptr, const int32_t* col) {
  int64_t h = 0;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p)
      if (col[p] < i) ++h;
  return h;
}

/* Position of column c in row r of a sorted CSR row, or -1. */
static int64_t find_in_row(const int64_t* row_ptr, const int32_t* col, int64_t r, int64_t c) {
  int64_t lo = row_ptr[r], hi = row_ptr[r + 1] - 1;
  while (lo <= hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (col[mid] == c) return mid;
    if (col[mid] < c) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

/* Split a full CSR matrix (both triangles, strictly ascending columns per row)
 * into CSRC arrays (Section 2). ia has n+1 entries; ja, al, au have
 * oracle_count_lower() entries. A missing diagonal is stored as 0.
 * Returns 0 on success, 1 if some a_ij (j<i) has no mirror a_ji (pattern not
 * structurally symmetric), 2 if a column is out of range, 3 if a row's columns
 * are not strictly ascending. */
int oracle_csr_to_csrc(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                       int64_t* ia, int32_t* ja, double* al, double* au, double* ad) {
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
      if (col[p] < 0 || col[p] >= n) return 2;
      if (p > row_ptr[i] && col[p] <= col[p - 1]) return 3;
    }
  }
  int64_t k = 0;
  for (int64_t i = 0; i < n; ++i) {
    ia[i] = k;
    ad[i] = 0.0;
    for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
      int64_t j = col[p];
      if (j == i) {
        ad[i] = val[p];
      } else if (j < i) {
        int64_t q = find_in_row(row_ptr, col, j, i); /* the mirror a_ji */
        if (q < 0) return 1;
        ja[k] = (int32_t)j;
        al[k] = val[p];
        au[k] = val[q];
        ++k;
      } else {
        if (find_in_row(row_ptr, col, j, i) < 0) return 1; /* a_ij above the diagonal needs a_ji */
      }
    }
  }
  ia[n] = k;
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Fig. 2(a) and Section 2.2: the sequential CSRC product y = A x. Rows are
 * visited in ascending order. Row i's lower entries gather into t, and their
 * mirrors scatter au(k)*x(i) into y(ja(k)). Every ja(k) < i, so y(ja(k)) was
 * already assigned when row ja(k) finished, and no earlier row has written y(i)
 * when it is assigned. x and y have strides incx and incy (for one column of a
 * row-major block of vectors). */
void oracle_csrc_spmv(int64_t n, const int64_t* ia, const int32_t* ja, const double* al,
                      const double* au, const double* ad, const double* x, int64_t incx,
                      double* y, int64_t incy) {
  for (int64_t i = 0; i < n; ++i) {
    double xi = x[i * incx];
    double t = ad[i] * xi;
    for (int64_t k = ia[i]; k < ia[i + 1]; ++k) {
      int64_t j = ja[k];
      t = t + al[k] * x[j * incx];
      y[j * incy] = y[j * incy] + au[k] * xi;
    }
    y[i * incy] = t;
  }
}

/* Section 5: A^T x is the same product with the addresses of al and au swapped. */
void oracle_csrc_spmv_t(int64_t n, const int64_t* ia, const int32_t* ja, const double* al,
                        const double* au, const double* ad, const double* x, int64_t incx,
                        double* y, int64_t incy) {
  oracle_csrc_spmv(n, ia, ja, au, al, ad, x, incx, y, incy);
}

/* Section 2.1 and Fig. 2(b): a rectangular n-by-m matrix (m >= n) is A_S + A_R, with
 * A_S the n-by-n structurally symmetric part in CSRC and A_R the n-by-(m - n) rest in an
 * auxiliary CSR (iar, jar, ar; jar holds columns in [n, m)). Row i adds the auxiliary
 * CSR row to the sum t before it is assigned. x has m entries, y has n. */
void oracle_csrcr_spmv(int64_t n, const int64_t* ia, const int32_t* ja, const double* al,
                       const double* au, const double* ad, const int64_t* iar, const int32_t* jar,
                       const double* ar, const double* x, double* y) {
  for (int64_t i = 0; i < n; ++i) {
    double xi = x[i];
    double t = ad[i] * xi;
    for (int64_t k = ia[i]; k < ia[i + 1]; ++k) {
      int64_t j = ja[k];
      t = t + al[k] * x[j];
      y[j] = y[j] + au[k] * xi;
    }
    for (int64_t k = iar[i]; k < iar[i + 1]; ++k) t = t + ar[k] * x[jar[k]];
    y[i] = t;
  }
}

/* The transpose of the rectangular matrix, y = A^T x with x of n entries and y of m:
 * entries 0..n-1 are A_S^T x (Section 5: al and au swapped), entries n..m-1 are
 * A_R^T x, i.e. column c of A_R scattered by rows: y[c] += ar(k) x(i) for every
 * auxiliary entry (i, c), y[n..m-1] starting from zero. */
void oracle_csrcr_spmv_t(int64_t n, int64_t m, const int64_t* ia, const int32_t* ja, const double* al,
                         const double* au, const double* ad, const int64_t* iar, const int32_t* jar,
                         const double* ar, const double* x, double* y) {
  oracle_csrc_spmv(n, ia, ja, au, al, ad, x, 1, y, 1);
  for (int64_t c = n; c < m; ++c) y[c] = 0.0;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = iar[i]; k < iar[i + 1]; ++k) y[jar[k]] = y[jar[k]] + ar[k] * x[i];
}

/* Several right-hand sides: Y = A X (or A^T X), X and Y n-by-r row-major, one
 * Fig. 2(a) product per column. */
void oracle_csrc_spmm(int64_t n, const int64_t* ia, const int32_t* ja, const double* al,
                      const double* au, const double* ad, int64_t r, const double* X, double* Y,
                      int transpose) {
  for (int64_t c = 0; c < r; ++c) {
    if (transpose)
      oracle_csrc_spmv_t(n, ia, ja, al, au, ad, X + c, r, Y + c, r);
    else
      oracle_csrc_spmv(n, ia, ja, al, au, ad, X + c, r, Y + c, r);
  }
}

/* Section 1: the CSR product y_i = sum_p a(p) x(ja(p)) over row i. It is a second,
 * independent oracle that works on the original full matrix. */
void oracle_csr_spmv(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                     const double* x, int64_t incx, double* y, int64_t incy) {
  for (int64_t i = 0; i < n; ++i) {
    double t = 0.0;
    for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) t = t + val[p] * x[(int64_t)col[p] * incx];
    y[i * incy] = t;
  }
}

/* Selected rows of the CSR product (for sampled checks on very large matrices). */
void oracle_csr_spmv_rows(const int64_t* row_ptr, const int32_t* col, const double* val,
                          const double* x, int64_t nrows, const int64_t* rows, double* y) {
  for (int64_t s = 0; s < nrows; ++s) {
    int64_t i = rows[s];
    double t = 0.0;
    for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) t = t + val[p] * x[col[p]];
    y[s] = t;
  }
}

/* Error metric for every configuration: for each row,
 *   err_i = |y_i - yref_i| / sum_j |a_ij| |x_j|
 * using the original FP64 coefficients (the sum runs over column i of A for the
 * transpose). When the denominator is zero, err_i = |y_i - yref_i|.
 * Returns max_i err_i; a NaN anywhere returns NaN. */
double oracle_max_rel_err(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                          const double* x, int64_t incx, const double* y, const double* yref,
                          int64_t incy, int transpose) {
  double* den = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  if (!den) return -1.0;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
      if (transpose)
        den[col[p]] += fabs(val[p]) * fabs(x[i * incx]);
      else
        den[i] += fabs(val[p]) * fabs(x[(int64_t)col[p] * incx]);
    }
  double worst = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double d = fabs(y[i * incy] - yref[i * incy]);
    if (d != d) { worst = NAN; break; }
    double e = den[i] > 0.0 ? d / den[i] : d;
    if (e > worst) worst = e;
  }
  free(den);
  return worst;
}

/* ------------------------------------------------------------------------- */
/* Reduced-precision storage. Values are rounded once from FP64 to nearest, ties
 * to even: to FP32 by the C conversion (round-to-nearest-even under the default
 * rounding mode), and to BF16 directly (8 significant bits, the FP32 exponent
 * range), not through FP32, which would round twice. The oracle then evaluates
 * the product of the rounded matrix in FP64, so the storage error can be told
 * apart from the accumulation error. */
void oracle_round_f32(const double* in, double* out, int64_t m) {
  for (int64_t i = 0; i < m; ++i) out[i] = (double)(float)in[i];
}

static double round_bf16_one(double v) {
  if (v != v || v == 0.0 || isinf(v)) return v;
  int e;
  double f = frexp(v, &e); /* v = f * 2^e, 0.5 <= |f| < 1 */
  /* the spacing of 8-significant-bit numbers with exponent e is 2^(e-8); below
   * the normal range (2^-126) the spacing stays at the subnormal step 2^-133 */
  int qexp = e - 8;
  if (qexp < -133) qexp = -133;
  double scaled = ldexp(v, -qexp);
  double r = nearbyint(scaled); /* ties to even under the default rounding mode */
  double out = ldexp(r, qexp);
  if (fabs(out) > 3.3895313892515355e38) /* beyond the largest finite BF16 */
    out = v > 0 ? INFINITY : -INFINITY;
  (void)f;
  return out;
}

void oracle_round_bf16(const double* in, double* out, int64_t m) {
  for (int64_t i = 0; i < m; ++i) out[i] = round_bf16_one(in[i]);
}

/* ------------------------------------------------------------------------- */
/* Section 3.1: non-zero-guided partition into B contiguous row bands. The paper
 * balances the non-zeros per thread. Row i carries w_i = 1 + 2*(ia(i+1)-ia(i)):
 * its diagonal plus both entries of each stored pair, so the w_i sum to nnz.
 * With prefix sums P(r) = sum_{i<r} w_i, boundary b_t is the smallest r with
 * P(r)*B >= t*nnz, so b_0 = 0 and b_B = n. */
void oracle_partition(int64_t n, const int64_t* ia, int64_t nbands, int64_t* band_ptr) {
  int64_t nnz = n + 2 * ia[n];
  int64_t r = 0, P = 0; /* P = P(r) */
  band_ptr[0] = 0;
  for (int64_t t = 1; t <= nbands; ++t) {
    /* advance r until P(r)*B >= t*nnz (128-bit safe: n, nnz < 2^40 here) */
    while (r < n && (__int128)P * nbands < (__int128)t * nnz) {
      P += 1 + 2 * (ia[r + 1] - ia[r]);
      ++r;
    }
    band_ptr[t] = r;
  }
}

/* ------------------------------------------------------------------------- */
/* Section 3.2: colouring the conflict graph. Two rows u != v conflict when their
 * write sets overlap. W(i) = {i} U {ja(k) : k in row i} is the set of entries of
 * y that row i writes in Fig. 2(a). This is the exact write-conflict graph: it
 * holds the direct conflicts (v in ja of u) and the indirect ones (u and v both
 * scatter into some y(k)). Colours are assigned greedily in a given order, each
 * row taking the smallest colour not used by an already-coloured conflicting
 * row (the sequential method of Coleman and More cited in Section 3.2). */

/* SplitMix64 (Steele, Lea, Flood 2014): mix(z + 0x9E3779B97F4A7C15). */
static uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint64_t oracle_priority(uint64_t seed, int64_t i) { return splitmix64(seed ^ (uint64_t)i); }

typedef struct { uint64_t pri; int64_t row; } pri_row;
static int by_priority_desc(const void* a, const void* b) {
  const pri_row* x = (const pri_row*)a;
  const pri_row* y = (const pri_row*)b;
  if (x->pri != y->pri) return x->pri > y->pri ? -1 : 1;
  return x->row < y->row ? -1 : (x->row > y->row);
}

/* Rows in decreasing priority order (the order Jones-Plassmann colours in). */
int oracle_priority_order(int64_t n, uint64_t seed, int64_t* order) {
  pri_row* v = (pri_row*)malloc(sizeof(pri_row) * (size_t)(n > 0 ? n : 1));
  if (!v) return 1;
  for (int64_t i = 0; i < n; ++i) { v[i].pri = oracle_priority(seed, i); v[i].row = i; }
  qsort(v, (size_t)n, sizeof(pri_row), by_priority_desc);
  for (int64_t i = 0; i < n; ++i) order[i] = v[i].row;
  free(v);
  return 0;
}

/* Rows v > t that hold t in their ja (the A_U column of t), as a CSR structure. */
static int build_upper(int64_t n, const int64_t* ia, const int32_t* ja, int64_t** up_ptr_out,
                       int64_t** up_out) {
  int64_t h = ia[n];
  int64_t* up_ptr = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  int64_t* up = (int64_t*)malloc(sizeof(int64_t) * (size_t)(h > 0 ? h : 1));
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  if (!up_ptr || !up || !fill) { free(up_ptr); free(up); free(fill); return 1; }
  for (int64_t k = 0; k < h; ++k) up_ptr[ja[k] + 1]++;
  for (int64_t t = 0; t < n; ++t) up_ptr[t + 1] += up_ptr[t];
  for (int64_t t = 0; t < n; ++t) fill[t] = up_ptr[t];
  for (int64_t v = 0; v < n; ++v)
    for (int64_t k = ia[v]; k < ia[v + 1]; ++k) up[fill[ja[k]]++] = v;
  free(fill);
  *up_ptr_out = up_ptr;
  *up_out = up;
  return 0;
}

/* Greedy colouring of the write-conflict graph in the given order. Writes
 * colors[0..n) and returns the number of colours, or -1 on allocation failure. */
int64_t oracle_greedy_color(int64_t n, const int64_t* ia, const int32_t* ja, const int64_t* order,
                            int32_t* colors) {
  int64_t *up_ptr, *up;
  if (build_upper(n, ia, ja, &up_ptr, &up)) return -1;
  int64_t* mark = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1)); /* mark[c] = row that saw colour c */
  if (!mark) { free(up_ptr); free(up); return -1; }
  for (int64_t c = 0; c <= n; ++c) mark[c] = -1;
  for (int64_t i = 0; i < n; ++i) colors[i] = -1;
  int64_t ncolors = 0;
  for (int64_t s = 0; s < n; ++s) {
    int64_t u = order[s];
    /* every t in W(u) is written by row t itself and by every row of A_U column t */
    for (int64_t q = ia[u] - 1; q < ia[u + 1]; ++q) {
      int64_t t = (q < ia[u]) ? u : ja[q];
      if (t != u && colors[t] >= 0) mark[colors[t]] = u;
      for (int64_t p = up_ptr[t]; p < up_ptr[t + 1]; ++p) {
        int64_t v = up[p];
        if (v != u && colors[v] >= 0) mark[colors[v]] = u;
      }
    }
    int64_t c = 0;
    while (mark[c] == u) ++c;
    colors[u] = (int32_t)c;
    if (c + 1 > ncolors) ncolors = c + 1;
  }
  free(mark); free(up_ptr); free(up);
  return ncolors;
}

/* Stride-bounded greedy colouring (the future work named in Section 6: a maximum stride
 * inside each colour class), in this reading: rows are coloured in ascending order, the
 * sequential greedy colouring of Section 3.2 in the matrix's own order, and row u takes
 * the smallest colour c that no earlier row writing into W(u) holds and whose last member
 * lies at most `stride` rows before u; when no colour qualifies a new one is opened. With
 * stride <= 0 there is no bound (plain greedy in ascending order). Returns the number of
 * colours, -1 on allocation failure. */
int64_t oracle_greedy_color_stride(int64_t n, const int64_t* ia, const int32_t* ja, int64_t stride,
                                   int32_t* colors) {
  int64_t *up_ptr, *up;
  if (build_upper(n, ia, ja, &up_ptr, &up)) return -1;
  int64_t* mark = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1)); /* mark[c] = row that saw colour c */
  int64_t* last = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1)); /* last member of colour c */
  if (!mark || !last) { free(mark); free(last); free(up_ptr); free(up); return -1; }
  for (int64_t c = 0; c <= n; ++c) { mark[c] = -1; last[c] = -1; }
  for (int64_t i = 0; i < n; ++i) colors[i] = -1;
  int64_t ncolors = 0;
  for (int64_t u = 0; u < n; ++u) {
    for (int64_t q = ia[u] - 1; q < ia[u + 1]; ++q) {
      int64_t t = (q < ia[u]) ? u : ja[q];
      if (t != u && colors[t] >= 0) mark[colors[t]] = u;
      for (int64_t p = up_ptr[t]; p < up_ptr[t + 1]; ++p) {
        int64_t v = up[p];
        if (v != u && colors[v] >= 0) mark[colors[v]] = u;
      }
    }
    int64_t c = 0;
    while (c < ncolors && (mark[c] == u || (stride > 0 && u - last[c] > stride))) ++c;
    colors[u] = (int32_t)c;
    last[c] = u;
    if (c + 1 > ncolors) ncolors = c + 1;
  }
  free(mark); free(last); free(up_ptr); free(up);
  return ncolors;
}

/* Validity of a colouring: within each colour class the write sets W(i) are
 * pairwise disjoint. Returns 0 if valid, 1 if two rows of one colour write the
 * same y entry, 2 if a colour is out of [0, ncolors), -1 on allocation failure. */
int oracle_check_coloring(int64_t n, const int64_t* ia, const int32_t* ja, const int32_t* colors,
                          int64_t ncolors) {
  int64_t* cnt = (int64_t*)calloc((size_t)ncolors + 1, sizeof(int64_t));
  int64_t* rows = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  int64_t* owner = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  int64_t* owner_col = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  if (!cnt || !rows || !owner || !owner_col) { free(cnt); free(rows); free(owner); free(owner_col); return -1; }
  int rc = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (colors[i] < 0 || colors[i] >= ncolors) { rc = 2; goto done; }
    cnt[colors[i] + 1]++;
  }
  for (int64_t c = 0; c < ncolors; ++c) cnt[c + 1] += cnt[c];
  for (int64_t i = 0; i < n; ++i) rows[cnt[colors[i]]++] = i; /* rows grouped by colour */
  for (int64_t t = 0; t < n; ++t) { owner[t] = -1; owner_col[t] = -1; }
  for (int64_t s = 0; s < n; ++s) {
    int64_t u = rows[s];
    int64_t c = colors[u];
    for (int64_t q = ia[u] - 1; q < ia[u + 1]; ++q) {
      int64_t t = (q < ia[u]) ? u : ja[q];
      if (owner_col[t] == c && owner[t] != u) { rc = 1; goto done; }
      owner_col[t] = c;
      owner[t] = u;
    }
  }
done:
  free(cnt); free(rows); free(owner); free(owner_col);
  return rc;
}
