/*
 * csrc.h - C ABI of the GB300 (sm_103a) CSRC sparse matrix-vector library.
 *
 * CSRC ("compressed sparse row-column") stores a structurally symmetric n-by-n
 * matrix A = A_D + A_L + A_U as five arrays (Batista, Ainsworth Jr., Ribeiro,
 * arXiv:1003.0952, Section 2):
 *   ad[n]       the diagonal,
 *   ia[n+1]     row pointers into the strictly lower part,
 *   ja[h]       column index of each lower entry a_ij (j < i), ascending per row,
 *   al[h]       the lower value a_ij,
 *   au[h]       its mirror a_ji, stored at the same position,
 * with h = (nnz - n)/2 stored pairs. Each stored pair gathers al*x[j] into
 * y[i] and scatters au*x[i] into y[j] (Fig. 2(a)), so A x and A^T x (al and au
 * swapped, Section 5) cost the same.
 *
 * Conventions shared by every entry point:
 *  - Indices are 0-based int32 (CSRC_FLAG_ONE_BASED accepts 1-based input).
 *    n < 2^31 and h < 2^31.
 *  - A handle owns all of its device memory. Every input array passed to a
 *    create call is read during the call and not retained. The caller keeps
 *    ownership of its arrays.
 *  - x and y are caller-owned vectors of n elements. With CSRC_F64 storage
 *    they are double; with CSRC_F32 or CSRC_BF16 storage they are float. They
 *    may be device pointers or host pointers: host buffers are staged through
 *    handle-owned device buffers with copies enqueued on the given stream. y is
 *    overwritten (y = A x, the semantics of Fig. 2(a)). x and y must not
 *    overlap.
 *  - Calls that take a stream are asynchronous on it (0 = legacy default
 *    stream). Errors that the host can detect are returned at once, before
 *    anything is enqueued. Errors that only the device can detect are recorded
 *    in the handle's device status word and read by
 *    csrc_get_last_device_error(). No call throws or aborts the process.
 *  - One handle must not be used by two concurrent calls: its scratch buffers
 *    are shared.
 */
#ifndef CSRC_GB300_CSRC_H
#define CSRC_GB300_CSRC_H

#include <stddef.h>
#include <stdint.h>

#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct csrc_matrix_s* csrc_handle; /* opaque; owns all device arrays */

typedef enum {
  CSRC_OK = 0,
  CSRC_ERR_INVALID_ARG = 1,          /* null pointer, negative size, bad enum, n or h too large */
  CSRC_ERR_NOT_STRUCT_SYMMETRIC = 2, /* a_ij stored without a_ji and CSRC_FLAG_PAD_PATTERN not set */
  CSRC_ERR_INDEX_RANGE = 3,          /* a row or column index outside [0, n) */
  CSRC_ERR_DUPLICATE = 4,            /* CSR row with repeated or unsorted columns */
  CSRC_ERR_ALIAS = 5,                /* x and y overlap */
  CSRC_ERR_NOT_PARTITIONED = 6,      /* a band strategy was requested before a partition could be built */
  CSRC_ERR_NOT_COLORED = 7,          /* CSRC_STRAT_COLOR requested before csrc_color() */
  CSRC_ERR_OUT_OF_MEMORY = 8,        /* device or host allocation failed */
  CSRC_ERR_CUDA = 9,                 /* a CUDA runtime call failed (no device, launch failure, ...) */
  CSRC_ERR_DEVICE_TIMEOUT = 10,      /* a bounded device wait ran out (device status word) */
  CSRC_ERR_DEVICE_BOUNDS = 11,       /* a device-side index check failed (device status word) */
  CSRC_ERR_RANGE = 12,               /* an x value lies outside the double-float range (device status word) */
  CSRC_ERR_MISMATCH = 13,            /* (not returned any more: batch members may differ in storage type) */
  CSRC_ERR_NOT_NUM_SYMMETRIC = 14,   /* CSRC_FLAG_SYMMETRIC_VALUES set but some a_ij != a_ji */
  CSRC_ERR_NOT_CONVERGED = 15,       /* csrc_bicg reached maxit above the tolerance (x = last iterate) */
  CSRC_ERR_BREAKDOWN = 16,           /* csrc_bicg met (r, r*) = 0 or (A p, p*) = 0 (x = last iterate) */
  CSRC_ERR_NOT_FOUND = 17,           /* csrc_tune_cache_lookup: no entry for this key */
  CSRC_ERR_IO = 18                   /* the tuning cache file cannot be written */
} csrc_status;

typedef enum { CSRC_F64 = 0, CSRC_F32 = 1, CSRC_BF16 = 2 } csrc_dtype; /* storage of ad, al, au */

typedef enum {
  CSRC_STRAT_AUTO = 0,   /* the handle's tuned choice (CSRC_STRAT_WINDOW until csrc_autotune() runs) */
  CSRC_STRAT_WINDOW = 1, /* private windows (Section 3.1 local buffers) whose scatter is sorted by target
                            when the plan is built: every window row is summed by one lane, with no
                            atomics; rows below a band are folded in by a deterministic accumulation
                            kernel. Bitwise reproducible from run to run. */
  CSRC_STRAT_COLOR = 2,  /* colour-ordered rows, no atomics (needs csrc_color() or csrc_color_stride()):
                            every class in one cooperative launch with a bounded grid barrier */
  CSRC_STRAT_ATOMIC = 3, /* stream-order windows flushed with global FP64/FP32 atomic adds */
  CSRC_STRAT_WINDOW_ATOMIC = 4 /* stream-order windows: each pair scatters into the shared-memory window
                                  with an atomic add as it streams past, rows below a band go through the
                                  accumulation kernel (the same deterministic fold as CSRC_STRAT_WINDOW) */
} csrc_strategy;

enum {
  CSRC_FLAG_PAD_PATTERN = 1, /* add an explicit zero a_ji for every a_ij without a mirror */
  CSRC_FLAG_ONE_BASED = 2,   /* row_ptr / row / col are 1-based (Fortran, as in Fig. 2) */
  CSRC_FLAG_FP64_ARITH = 4,  /* CSRC_F64 only: every multiply and add on the FP64 pipe. This is the
                                default for CSRC_F64 storage; the flag is accepted for clarity */
  CSRC_FLAG_DF32_ARITH = 64, /* CSRC_F64 only, stream-order strategies (CSRC_STRAT_WINDOW_ATOMIC and
                                CSRC_STRAT_ATOMIC): the scatter products and window sums in double-float
                                arithmetic on the FP32 pipes (about 2^-46 relative per operation instead of
                                2^-53, values and x within [2^-50, 2^63) in magnitude), the gather on the
                                FP64 pipe. CSRC_STRAT_WINDOW, CSRC_STRAT_COLOR and products with several
                                right-hand sides keep FP64 arithmetic */
  CSRC_FLAG_SYMMETRIC_VALUES = 16, /* numerically symmetric matrix (Section 2.2): every a_ji equals a_ij
                                     bit for bit (checked at creation), au is not stored and the
                                     kernels scatter with al, so a product streams 12 instead of 20
                                     bytes per pair in FP64; A^T x = A x */
  CSRC_FLAG_COMPRESS_INDICES = 32, /* the window strategy's single-vector plans keep each pair's band-local
                                     window slot as 16 bits (index compression): a product streams 2
                                     instead of 4 index bytes per pair (18 / 10 / 6 bytes per pair in
                                     FP64 / FP32 / BF16); a plan whose windows exceed 65,536 rows keeps
                                     32-bit slots */
  CSRC_FLAG_NODE_BLOCKS = 8  /* when the matrix has node blocks (B = 2 or 3 consecutive rows sharing
                                their columns, as with B unknowns per FE node), run node-block units */
};

/* Summary of a handle (csrc_get_info). Byte counts are per product y = A x. */
typedef struct {
  int64_t n;                /* rows */
  int64_t pairs;            /* h = stored off-diagonal pairs */
  int64_t nnz;              /* n + 2h */
  int32_t storage;          /* csrc_dtype */
  int32_t arith;            /* 0 = double-float, 1 = FP64 pipe, 2 = FP32 */
  int64_t model_bytes;      /* ia + ja + al + au + ad + x + y (Table 1's ws for CSRC_F64) */
  int32_t nbands;           /* execution bands of the window plan (0 before it is built); the window
                               strategy's lists when built, else the stream-order plan's */
  int32_t page_rows;        /* rows per window page of the stream-order plan (0 for the lists) */
  int64_t spill_entries;    /* window slots written to the spill buffer per product */
  int64_t spill_rows;       /* rows that receive spilled partial sums */
  int64_t accum_bytes;      /* accumulation traffic per product (spill write+read, indices, y update) */
  int32_t max_window_slots; /* largest window in rows */
  int32_t smem_bytes;       /* dynamic shared memory of the band kernel */
  int32_t ncolors;          /* colours (0 before csrc_color) */
  int32_t tuned_strategy;   /* csrc_strategy picked by csrc_autotune (0 = not tuned) */
  int32_t tuned_rk;         /* columns per pass picked by csrc_autotune_spmm (0 = up to 8) */
  int32_t group;            /* lanes per row of the band kernel (0 before the plan is built) */
  int64_t nstages;          /* shared-memory ring stages of one single-vector product */
  int32_t block;            /* rows per node block the single-vector product runs (1 = plain rows) */
  int64_t m;                /* columns: n for square handles, m >= n for rectangular ones */
  int64_t rect_nnz;         /* entries of the auxiliary CSR of a rectangular handle (0 when square) */
  /* the window strategy's lists (0 before they are built): */
  int64_t list_entries;     /* list entries of all bands (n + 2h) */
  int64_t list_slices;      /* slices of 32 window rows */
  int64_t list_lane_steps;  /* lanes issued: 32 x the longest list of every slice (>= list_entries) */
  int64_t list_bytes;       /* bytes the window strategy's product kernel moves per product */
  /* the stream-order plan (window-atomic and atomic strategies; 0 before it is built): */
  int32_t stream_nbands;
  int64_t stream_spill_entries;
  int32_t precision;        /* csrc_dtype of the window strategy's values (csrc_set_precision) */
  double error_bound;       /* its componentwise error bound (csrc_autotune_precision), 0 before
                               the window strategy's lists are built */
} csrc_info;

/*
 * Build a handle from a full CSR matrix (both triangles and the diagonal).
 * Section 2: every a_ij with j < i becomes al at row i, its mirror a_ji
 * becomes au at the same position, and a_ii becomes ad[i] (0 when absent).
 *   n        rows (= columns), 0 <= n < 2^31
 *   row_ptr  host, int64[n+1], row_ptr[0] = 0 (1 with CSRC_FLAG_ONE_BASED)
 *   col      host, int32[row_ptr[n]], strictly ascending within each row
 *   val      host, double[row_ptr[n]]
 *   storage  CSRC_F64 keeps the doubles. CSRC_F32 / CSRC_BF16 round each value
 *            once to nearest-even (BF16 directly from double, not through FP32).
 *   flags    CSRC_FLAG_* bits
 *   stream   stream used for the uploads (the handle is usable once it completes)
 * Errors: INVALID_ARG, INDEX_RANGE, DUPLICATE (repeated/unsorted columns),
 * NOT_STRUCT_SYMMETRIC, OUT_OF_MEMORY, CUDA. On error *out is set to NULL.
 */
csrc_status csrc_create_from_csr(csrc_handle* out, int32_t n, const int64_t* row_ptr, const int32_t* col,
                                 const double* val, csrc_dtype storage, uint32_t flags, cudaStream_t stream);

/*
 * Build a handle for a rectangular n-by-m matrix, m >= n (Section 2.1, Fig. 2(b)): the
 * n-by-n block of columns 0..n-1 (A_S) must have a symmetric pattern and is stored as
 * CSRC exactly as csrc_create_from_csr stores a square matrix; the entries of columns
 * n..m-1 (A_R) go to an auxiliary CSR, plus a column-major copy of it for A^T. This is
 * the matrix of one subdomain in an overlapping decomposition: its own unknowns first,
 * then the overlap.
 *   n, m     rows and columns, 0 <= n <= m < 2^31
 *   row_ptr  host, int64[n+1]; col host, int32[row_ptr[n]] in [0, m), strictly ascending
 *            within each row; val host, double[row_ptr[n]]; base as csrc_create_from_csr
 * On the handle, csrc_spmv reads x of m entries and writes y of n (A_S x[0..n) by the
 * chosen strategy, then each row adds its A_R row), and csrc_spmv_t reads x of n entries
 * and writes y of m (A_S^T x into y[0..n), A_R^T x into y[n..m)). Partition, colouring,
 * autotuning and profiling work as for a square handle (they concern A_S).
 * csrc_spmm_batched, csrc_autotune_spmm and csrc_spmv_noalloc return INVALID_ARG for
 * rectangular handles.
 * Errors: as csrc_create_from_csr, and INVALID_ARG when m < n. On error *out is NULL.
 */
csrc_status csrc_create_rect_from_csr(csrc_handle* out, int32_t n, int32_t m, const int64_t* row_ptr,
                                      const int32_t* col, const double* val, csrc_dtype storage, uint32_t flags,
                                      cudaStream_t stream);

/*
 * Build a handle from coordinate triples (host arrays of nnz entries, any order).
 * Duplicate (row, col) entries are summed first. The rest is as
 * csrc_create_from_csr.
 */
csrc_status csrc_create_from_coo(csrc_handle* out, int32_t n, int64_t nnz, const int32_t* row,
                                 const int32_t* col, const double* val, csrc_dtype storage, uint32_t flags,
                                 cudaStream_t stream);

/*
 * Non-zero-guided row partition (Section 3.1): nbands contiguous row bands. Row i
 * weighs w_i = 1 + 2*(ia[i+1]-ia[i]) (the w_i sum to nnz). Boundary b_t is the
 * smallest r whose prefix weight P(r) satisfies P(r)*nbands >= t*nnz, so b_0 = 0
 * and b_nbands = n. nbands = 0 picks a count from the matrix and the GPU: whole
 * waves of SMs x 4 bands, each of about 100,000 non-zeros for FP64 values and 180,000
 * for FP32 / BF16. The window plan that the kernels run is built from these bands; a
 * band whose window would not fit in shared memory is split in two, and an automatic
 * count that needed splits is replaced by the next whole number of waves, so that
 * the bands stay equal. Both are cached in the handle. Synchronous.
 *   band_ptr_out  host int32[nbands+1] (nullable). Receives b_0..b_nbands.
 *                 With nbands = 0 it must hold csrc_info.nbands+1 entries.
 * Errors: INVALID_ARG, OUT_OF_MEMORY, CUDA.
 */
csrc_status csrc_partition(csrc_handle h, int32_t nbands, int32_t* band_ptr_out);

/*
 * Colour the rows for the colour-ordered product (Section 3.2). Rows u and v
 * conflict when their write sets W(i) = {i} U {ja[k] : k in row i} intersect.
 * Colouring runs on the device (Jones-Plassmann rounds, priority of row i =
 * SplitMix64(seed ^ i), smallest free colour). The result equals sequential
 * greedy colouring in decreasing priority order. The colour classes and their
 * row lists are cached in the handle. Synchronous.
 *   ncolors_out  host (nullable): number of colours
 *   colors_out   host int32[n] (nullable): colour of each row
 * Errors: INVALID_ARG, OUT_OF_MEMORY, CUDA, DEVICE_TIMEOUT (a round limit ran out).
 */
csrc_status csrc_color(csrc_handle h, uint64_t seed, int32_t* ncolors_out, int32_t* colors_out);

/*
 * Stride-bounded colouring (the future work named in Section 6: "fixing the maximum allowed
 * stride size inside each color class"), in this reading: rows are coloured in ascending
 * order (the sequential greedy colouring of Section 3.2 in the matrix's own order, which keeps
 * the locality of its reordering), and row i takes the smallest colour c that no earlier row
 * writing into W(i) holds and whose last member lies at most `stride` rows before i; when no
 * colour qualifies a new one is opened. Every class therefore visits its rows with gaps of at
 * most `stride`. stride <= 0 means no bound. Runs on the host (it is sequential by
 * definition); the classes replace any earlier colouring of the handle. Synchronous.
 *   ncolors_out, colors_out  as for csrc_color
 * Errors: INVALID_ARG (more than 65536 colours), OUT_OF_MEMORY, CUDA.
 */
csrc_status csrc_color_stride(csrc_handle h, int64_t stride, int32_t* ncolors_out, int32_t* colors_out);

/*
 * y = A x (Fig. 2(a)) with the given strategy (CSRC_STRAT_AUTO: the handle's tuned strategy,
 * else the window strategy). x and y are device pointers, or host pointers that the call
 * stages through handle-owned device buffers. Asynchronous on stream, except that a call
 * that finds no plan for its strategy (no csrc_partition yet, or plans dropped by a change of
 * band count or precision) first builds one, synchronously and allocating.
 */
csrc_status csrc_spmv(csrc_handle h, const void* x, void* y, csrc_strategy strategy, cudaStream_t stream);

/* y = A^T x: the same kernels with al and au swapped (Section 5). */
csrc_status csrc_spmv_t(csrc_handle h, const void* x, void* y, csrc_strategy strategy, cudaStream_t stream);

/*
 * Batched products Y_b = A_b X_b (or A_b^T X_b) for b < batch, each X_b, Y_b an
 * n_b-by-nrhs row-major device block: double for a CSRC_F64 handle (whatever its
 * csrc_set_precision), float for CSRC_F32 / CSRC_BF16 storage. Members may differ in
 * storage type and precision; all must live on the current device and be square.
 * One vector of one matrix (batch = 1, nrhs = 1) is csrc_spmv / csrc_spmv_t with the
 * handle's tuned strategy. Otherwise every member's columns are cut into chunks of 1, 2, 4
 * or 8 (csrc_autotune_spmm picks the width) and every chunk's bands become tiles of one
 * window-strategy launch per (value type, chunk width), costliest tiles first, followed by
 * one accumulation launch per value type; the launches are captured in a CUDA graph and
 * replayed while the handles, pointers and sizes stay the same. Each member runs plans of
 * its own for batches (bands of up to about 100,000 non-zeros in FP64 and 180,000 in FP32 /
 * BF16, smaller when the whole batch would not fill the GPU several times over). With
 * nrhs = 1, a member tuned to another strategy, or whose windows cannot hold its targets,
 * runs its own launches on the same stream after the graph.
 * Asynchronous on stream; the first call with a new set of arguments builds plans and the
 * graph (synchronous, allocating).
 * Errors: INVALID_ARG (null or host pointers, rectangular handles, handles of another
 * device), ALIAS, OUT_OF_MEMORY, CUDA.
 */
csrc_status csrc_spmm_batched(const csrc_handle* hs, int32_t batch, const void* const* X, void* const* Y,
                              int32_t nrhs, int32_t transpose, cudaStream_t stream);

/* Capacity of the fixed spill array that csrc_spmv_noalloc uses: 2^21 values (16 MiB). */
#define CSRC_NOALLOC_MAX_SPILL_ENTRIES (1 << 21)

/*
 * y = A x (transpose == 0) or y = A^T x (transpose != 0) with the window strategy,
 * allocating no memory. The paper has no counterpart: this entry point serves callers
 * that may not allocate device memory while they compute, such as code whose GPU
 * memory belongs to another allocator's pool, or host threads that must not block on
 * the device synchronisation that cudaMalloc and cudaFree can cause. Such a caller
 * creates its handle and calls csrc_partition once at set-up, then uses this call.
 *
 * It computes what csrc_spmv / csrc_spmv_t compute with CSRC_STRAT_WINDOW, with the
 * same kernels (bit for bit: the window strategy sums every row in a fixed order). The
 * only difference is that the spilled partial sums go to a fixed
 * array of CSRC_NOALLOC_MAX_SPILL_ENTRIES values that the library holds in static
 * device memory (16 MiB on every GPU that loads the library, kept until the process
 * exits), instead of the buffer the handle allocates.
 *   h          a handle on which csrc_partition has succeeded (the plan is not built here)
 *   x, y       device pointers to n elements (double for CSRC_F64 storage, else float),
 *              caller-owned, not overlapping; y is overwritten
 *   transpose  0 for A x, non-zero for A^T x
 *   stream     asynchronous on this stream
 * Set-up: the first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current. Make that first call before any
 * stream capture. The call makes the handle's device current while it runs and gives
 * the caller's current device back before it returns.
 * Sharing: every call on a device, from any handle, uses the same array, which keeps
 * the last call's contents. The band kernel writes every slot the accumulation reads,
 * so nothing needs clearing between calls, but calls that overlap on the GPU (other
 * streams, other threads) race on it and must be serialised by the caller.
 * Errors: INVALID_ARG (null argument, host pointer, or a plan whose spill needs more
 * than CSRC_NOALLOC_MAX_SPILL_ENTRIES values: csrc_info.spill_entries tells in
 * advance), ALIAS, NOT_PARTITIONED (no plan yet, or a plan that cannot run the window
 * strategy), CUDA.
 */
csrc_status csrc_spmv_noalloc(csrc_handle h, const void* x, void* y, int32_t transpose, cudaStream_t stream);

/*
 * Autotuner (not in the paper, whose comparison of colouring and local buffers in
 * Section 4.2 shows that the best strategy depends on the matrix). Times y = A x with
 * the window strategy at three band counts (the automatic one, one wave of SMs x 4 bands
 * fewer and one more), then with the window-atomic and atomic strategies and, when the
 * rows are coloured, the colour strategy. Keeps the fastest band count for the window
 * plans and the fastest strategy as the handle's CSRC_STRAT_AUTO choice, and records
 * both in the tuning cache (csrc_tune_key). Batched products keep a member's choice for
 * single vectors. Synchronous on stream.
 *   x, y  device vectors of n elements used as scratch (y is overwritten)
 * Errors: INVALID_ARG (null or host pointers), OUT_OF_MEMORY, CUDA.
 */
csrc_status csrc_autotune(csrc_handle h, const void* x, void* y, cudaStream_t stream);

/*
 * Pick the columns per pass (1, 2, 4 or 8, at most nrhs) of several-right-hand-side
 * products on this handle by timing Y = A X on the caller's n-by-nrhs row-major device
 * blocks X and Y (Y is overwritten); the choice is recorded in the tuning cache for this
 * nrhs. Synchronous on stream. nrhs = 1 leaves the handle unchanged.
 * Errors: INVALID_ARG, NOT_PARTITIONED, OUT_OF_MEMORY, CUDA.
 */
csrc_status csrc_autotune_spmm(csrc_handle h, const void* X, void* Y, int32_t nrhs, cudaStream_t stream);

/*
 * Precision of the window strategy's values (the paper computes in FP64; this is the
 * reduced-precision form of the product). For a CSRC_F64 handle:
 *   CSRC_F64   (default) FP64 values and FP64 multiply-adds;
 *   CSRC_F32   every value of the window strategy's lists rounded once to nearest FP32;
 *   CSRC_BF16  every value rounded once, directly from the double, to nearest-even BF16;
 * with FP32 / BF16 values, x is rounded to FP32 in the window, the multiply-adds and the
 * partial sums are FP32, and y is written as double. x and y stay double vectors, so a caller
 * switches precision without touching its data. The lists are rebuilt at the new precision on
 * the next product. Only the window strategy (single and batched products, several
 * right-hand sides) runs at this precision; the other strategies keep the storage's. A
 * CSRC_F32 / CSRC_BF16 handle accepts only its storage type.
 * Errors: INVALID_ARG.
 */
csrc_status csrc_set_precision(csrc_handle h, csrc_dtype precision);

/*
 * Pick the cheapest precision of the window strategy that meets a componentwise error
 * budget: max_i |y_i - (A x)_i| / sum_j |a_ij||x_j| <= max_rel_err for every x. The bound used
 * is the rounding-error bound of the lists' arithmetic,
 *   u_v + u_x + (L + P - 1) u_a,
 * with u_v, u_x, u_a the unit roundoffs of the values, of x in the window and of the
 * multiply-adds (2^-53 for FP64; 2^-24 for FP32; 2^-8 for BF16 values), L the longest row of A
 * and P the most partial sums any row is split into across bands. Every precision within the
 * budget is timed on the caller's device vectors x, y (y is overwritten), and the fastest is
 * kept (csrc_set_precision); a wider precision must be more than 3 % faster than a narrower
 * one to be preferred, so near-ties keep the fewer bytes. The decision is kept in the tuning
 * cache (csrc_autotune).
 *   chosen_out  host (nullable): the csrc_dtype picked
 *   bound_out   host (nullable): its error bound
 * Synchronous on stream. Errors: INVALID_ARG (null or host pointers, max_rel_err <= 0, or no
 * precision meets the budget: FP64's own bound is the least attainable), OUT_OF_MEMORY, CUDA.
 */
csrc_status csrc_autotune_precision(csrc_handle h, const void* x, void* y, double max_rel_err, int32_t* chosen_out,
                                    double* bound_out, cudaStream_t stream);

/*
 * The tuning cache. csrc_autotune, csrc_autotune_spmm and csrc_autotune_precision record
 * their decisions in a text file keyed by the matrix (its pattern hash, n, nnz, storage and
 * creation flags) and the device, so that a later process skips the timing. The environment
 * variable CSRC_TUNE selects the behaviour: "cache" (default) reuses a recorded decision and
 * tunes and records on a miss; "full" always tunes and records; "off" leaves the handle's
 * defaults and touches no file. CSRC_TUNE_CACHE names the file (default
 * $XDG_CACHE_HOME/csrc_gb300/tune.txt, else $HOME/.cache/csrc_gb300/tune.txt). Writes are
 * whole-file replacements under a lock within the process; lines that do not parse are
 * ignored.
 */
typedef struct {
  uint64_t pattern_hash; /* FNV-1a 64 of n, ia and ja */
  int64_t n;
  int64_t nnz;
  int32_t storage;       /* csrc_dtype */
  uint32_t flags;        /* creation flags */
  char device[64];       /* device name and SM count, NUL-terminated */
} csrc_tune_key;

enum {
  CSRC_TUNE_STRATEGY = 0,  /* values: strategy, band count of the window strategy's lists (param 0) */
  CSRC_TUNE_KTILE = 1,     /* values: columns per pass (param = number of right-hand sides) */
  CSRC_TUNE_PRECISION = 2  /* values: csrc_dtype (param = error budget) */
};

/* The cache key of a handle (host only, no device work). Errors: INVALID_ARG. */
csrc_status csrc_get_tune_key(csrc_handle h, csrc_tune_key* key);

/* Look up / record one decision: values[0..3] (unused ones 0). lookup returns
 * CSRC_ERR_NOT_FOUND on a miss or when CSRC_TUNE is "off"; store does nothing when it is "off".
 * Host only. Errors: INVALID_ARG, NOT_FOUND, IO. */
csrc_status csrc_tune_cache_lookup(const csrc_tune_key* key, int32_t kind, double param, int32_t values[4]);
csrc_status csrc_tune_cache_store(const csrc_tune_key* key, int32_t kind, double param, const int32_t values[4]);

/* Kernel kinds of csrc_kernel_times. */
enum {
  CSRC_KERNEL_PRODUCT = 0,    /* the kernels that stream the stored pairs (band, colour-row) */
  CSRC_KERNEL_ACCUMULATE = 1, /* the kernel that folds spilled partial sums into y */
  CSRC_KERNEL_OTHER = 2,      /* everything else the product launches */
  CSRC_KERNEL_KINDS = 3
};

/* Device time of the kernels a handle launched while profiling was on. */
typedef struct {
  int64_t launches[CSRC_KERNEL_KINDS]; /* launches per kind */
  double ms[CSRC_KERNEL_KINDS];        /* summed device time per kind, in milliseconds */
} csrc_kernel_times;

/*
 * Turn per-launch kernel timing on (enable != 0) or off for this handle, and drop
 * what was recorded so far. While it is on, every kernel the handle launches is
 * bracketed by two CUDA events on the launch stream (a measurement aid; the paper
 * has no counterpart, it counts time with CPU timers and PAPI).
 * Errors: INVALID_ARG.
 */
csrc_status csrc_set_profiling(csrc_handle h, int32_t enable);

/*
 * Wait for the recorded launches, sum their device time per kernel kind into
 * *out (host), and drop the records. Errors: INVALID_ARG, CUDA.
 */
csrc_status csrc_get_kernel_times(csrc_handle h, csrc_kernel_times* out);

/*
 * Solve A x = b by biconjugate gradients (BiCG: Fletcher's method as in Saad, Iterative
 * Methods for Sparse Linear Systems, 2nd ed., Algorithm 7.3, shadow residual r*_0 = r_0):
 * the oblique-projection solver that Section 1 names as a user of CSRC's implicit
 * transpose. Every iteration runs one csrc_spmv (A p) and one csrc_spmv_t (A^T p*) with
 * the given strategy, and two fused vector passes on the device; inner products are
 * summed in FP64 in a fixed order (deterministic). Stops when ||r||_2 <= rtol ||b||_2 for
 * the recursively updated residual r.
 *   b, x      device vectors of n elements of the handle's vector type (double for
 *             CSRC_F64, float otherwise); x holds the initial guess and receives the solution
 *   rtol      relative tolerance (>= 0); maxit iterations at most (>= 0)
 *   iters_out, relres_out  optional host outputs: iterations run and ||r||_2 / ||b||_2
 *             (0 when b = 0)
 * Square handles only. Synchronises the stream every iteration (the scalars go to the
 * host). The handle keeps six scratch vectors for later calls.
 * Errors: INVALID_ARG, ALIAS, NOT_PARTITIONED, NOT_COLORED, OUT_OF_MEMORY, CUDA, and
 * NOT_CONVERGED / BREAKDOWN (outputs and x still set); a device error raised by the products
 * during the solve (DEVICE_TIMEOUT, DEVICE_BOUNDS, RANGE) is returned and cleared from the
 * handle's status word.
 */
csrc_status csrc_bicg(csrc_handle h, const void* b, void* x, double rtol, int32_t maxit, csrc_strategy strategy,
                      int32_t* iters_out, double* relres_out, cudaStream_t stream);

/*
 * Self-test of the kernels' bounded waits (failure detection without a GPU fault): one CTA
 * waits, with the same bounded mbarrier wait the band kernels use, on a barrier that
 * nothing arrives at, giving up after `cycles` SM clock cycles (clamped to [1000, 2e9]).
 * The expected result is CSRC_ERR_DEVICE_TIMEOUT, read back from a device status word
 * after the kernel has returned normally; the CUDA context stays usable. Returns CSRC_OK
 * only if the wait completed (it cannot), CSRC_ERR_CUDA on a runtime error.
 * Synchronous (default stream of the current device).
 */
csrc_status csrc_selftest_bounded_wait(int64_t cycles);

/* Fill *info (host). */
csrc_status csrc_get_info(csrc_handle h, csrc_info* info);

/* Read and clear the handle's device status word (synchronises the device).
 * Returns CSRC_OK, CSRC_ERR_DEVICE_TIMEOUT, CSRC_ERR_DEVICE_BOUNDS or CSRC_ERR_RANGE. */
csrc_status csrc_get_last_device_error(csrc_handle h);

/* Release every device and host resource of the handle (synchronises first). NULL is allowed. */
csrc_status csrc_destroy(csrc_handle h);

/* Static description of a status code. */
const char* csrc_status_string(csrc_status st);

#ifdef __cplusplus
}
#endif
#endif /* CSRC_GB300_CSRC_H */
