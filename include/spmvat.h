/*
 * spmvat.h - C ABI of the GB300 (sm_103a) library for run-time sparse-format
 * transformation, SpMV and format auto-tuning after Katagiri & Sato, "An
 * Auto-tuning Method for Run-time Data Transformation for Sparse
 * Matrix-Vector Multiplication" (Sec. 2.1 formats and transformations,
 * Sec. 2.2 the D_mat / R_ell auto-tuning rule, Sec. 3 SpMV per format).
 *
 * Conventions for every entry point
 *  - Indices are 0-based int32, values float64. A matrix has n_rows rows and
 *    n_cols columns; nnz < 2^31.
 *  - Pointers named "device" must point to memory of the current CUDA device;
 *    pointers named "host" to host memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream). Work is enqueued on it in stream order. Only the calls marked
 *    SYNC wait for the stream; all others return after enqueueing.
 *  - Nothing throws, exits or prints. Every call returns an spmv_status; on
 *    any error, output handles are set to NULL and no handle memory leaks.
 *  - Kernels never read or write out of bounds on a malformed CRS: entries
 *    with an index out of range are skipped and reported as
 *    SPMV_ERR_INVALID_MATRIX by the next SYNC call that reads the status.
 */
#ifndef SPMVAT_H
#define SPMVAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SPMVAT_VERSION 1

typedef void *spmv_stream_t; /* cudaStream_t */

typedef enum spmv_status {
    SPMV_OK = 0,
    SPMV_ERR_INVALID_ARG = 1,     /* NULL pointer, negative size, bad enum */
    SPMV_ERR_INVALID_MATRIX = 2,  /* IRP not monotone / not 0..nnz, index out of range */
    SPMV_ERR_OOM = 3,             /* the allocator returned NULL */
    SPMV_ERR_MEMORY_CAP = 4,      /* the result would exceed mem_cap_bytes */
    SPMV_ERR_TIMEOUT = 5,         /* a bounded device-side wait ran out */
    SPMV_ERR_CUDA = 6,            /* a CUDA runtime call failed */
    SPMV_ERR_UNSUPPORTED = 7      /* valid request this build does not serve */
} spmv_status;

/* Storage formats of Sec. 2.1. With SPMV_COLWISE, SPMV_CRS denotes the
 * compressed-column result of Phase I (CCS). */
typedef enum spmv_format { SPMV_CRS = 0, SPMV_COO = 1, SPMV_ELL = 2 } spmv_format;
typedef enum spmv_layout { SPMV_ROWWISE = 0, SPMV_COLWISE = 1 } spmv_layout;

/* A CRS matrix (Sec. 2.1: VAL(1:nnz), ICOL(1:nnz), IRP(1:n+1)), 0-based.
 * All three arrays are device memory owned by the caller. */
typedef struct spmv_crs {
    int32_t n_rows;
    int32_t n_cols;
    int64_t nnz;
    const int32_t *irp;  /* device int32[n_rows+1]; irp[0]=0, non-decreasing, irp[n_rows]=nnz */
    const int32_t *icol; /* device int32[nnz]; column of each entry, 0 <= icol < n_cols */
    const double *val;   /* device float64[nnz] */
} spmv_crs;

/* Row-length statistics (Sec. 2.2, Eq. (4)). */
typedef struct spmv_stats {
    double mu;            /* mean nonzeros per row = nnz / n_rows */
    double sigma;         /* population standard deviation of the row lengths */
    double dmat;          /* D_mat = sigma / mu (0 when nnz = 0) */
    int32_t max_row_len;  /* W: the ELL width ("nz", the bandwidth length of Sec. 2.1) */
    int32_t min_row_len;
    int64_t n_empty_rows;
    uint64_t ell_bytes;   /* device bytes a row-wise ELL of this matrix needs */
    int64_t row_len_hist[32]; /* rows per class: 0 = empty, c >= 1: length in [2^(c-1), 2^c) */
} spmv_stats;

/* Parameters of the run-time AT method (Sec. 2.2). */
#define SPMV_DSTAR_PREFIX 0  /* D* = D_mat of the first point, by ascending D_mat, with R_ell < c */
#define SPMV_DSTAR_MAXPASS 1 /* D* = largest D_mat among points with R_ell >= c */
#define SPMV_AT_TRY_COO 1    /* flag: when ELL is rejected, time COO-Row against CRS and keep the faster */
typedef struct spmv_at_params {
    double c;               /* R_ell threshold of the off-line phase; the paper uses 1.0 */
    double dstar;           /* D*: the on-line phase picks ELL iff dmat < dstar */
    uint64_t mem_cap_bytes; /* device bytes a transformation may own; 0 = no cap */
    int32_t timing_reps;    /* timed repetitions per measurement (median); <= 0 means 20 */
    int32_t warmup_reps;    /* untimed repetitions first; < 0 means 3 */
    int32_t dstar_rule;     /* SPMV_DSTAR_PREFIX or SPMV_DSTAR_MAXPASS */
    int32_t flags;          /* SPMV_AT_TRY_COO */
} spmv_at_params;

/* Times of one matrix (Sec. 2.2, Eqs. (1)-(3)); milliseconds, medians. */
typedef struct spmv_timing {
    double t_crs_ms, t_ell_ms, t_trans_ms, t_coo_ms;
    double sp;    /* SP_crs/ell = t_crs / t_ell                         (Eq. 1) */
    double tt;    /* TT_ell = t_trans / t_crs (Eq. 2, read as the cost of the
                     transformation in CRS-SpMV units)                 */
    double r_ell; /* R_ell = SP / TT                                    (Eq. 3) */
    double dmat;  /* D_mat of the matrix                                (Eq. 4) */
} spmv_timing;

/* Opaque handle to a matrix in one format; owns its device arrays. */
typedef struct spmv_matrix spmv_matrix;

/* Read-only view of a handle's arrays (device pointers). ELL slot arrays are
 * column-major over lines with leading dimension ld >= number of lines: slot
 * k of line i is element k*ld + i (Fig. 3 indexing with N replaced by ld).
 * Lines are rows for SPMV_ROWWISE and columns for SPMV_COLWISE. */
typedef struct spmv_matrix_desc {
    int32_t format, layout;
    int32_t n_rows, n_cols;
    int64_t nnz;
    int32_t width;       /* ELL: slots per line; else 0 */
    int32_t ld;          /* ELL: leading dimension; else 0 */
    const int32_t *ptr;  /* CRS: IRP (caller's); column-wise: IRP_T, int32[n_cols+1]; else NULL */
    const int32_t *idx;  /* CRS, COO-Row: ICOL (caller's); CCS, COO-Col: row of each entry;
                            ELL-Row: column of each slot; ELL-Col: row of each slot */
    const int32_t *idx2; /* COO-Row: IROW; COO-Col: column of each entry; else NULL */
    const double *val;   /* values (CRS, COO-Row: the caller's VAL) */
    uint64_t owned_bytes;/* device bytes this handle keeps alive */
} spmv_matrix_desc;

/* Device memory hooks. alloc returns NULL on failure; free releases in stream
 * order on `stream`. Default: a private stream-ordered CUDA memory pool. */
typedef void *(*spmv_alloc_fn)(size_t bytes, void *ctx, spmv_stream_t stream);
typedef void (*spmv_free_fn)(void *ptr, size_t bytes, void *ctx, spmv_stream_t stream);

/* Per-kernel device time gathered while profiling is on. */
typedef struct spmv_kernel_time {
    char name[48];
    uint64_t launches;
    double total_ms;
} spmv_kernel_time;

/* ------------------------------------------------------------------------ */

/* Library version (SPMVAT_VERSION). */
int32_t spmv_version(void);

/* Human-readable name of a status code; never NULL. */
const char *spmv_status_string(spmv_status s);

/* Install device-memory hooks (both non-NULL), or restore the default pool
 * (both NULL). Affects allocations made after the call. */
spmv_status spmv_set_allocator(spmv_alloc_fn alloc, spmv_free_fn free_fn, void *ctx);

/* SYNC. Grows the library's private device-memory pool (on the current
 * device) by allocating `bytes` and freeing them: the pool keeps freed memory,
 * so later transformations on any stream sub-allocate from it instead of
 * mapping new memory in the middle of a computation. No effect when
 * allocator hooks are installed. SPMV_ERR_OOM if the memory is not there. */
spmv_status spmv_reserve(uint64_t bytes, spmv_stream_t stream);

/* SYNC. Row-length statistics of a CRS matrix: mu, sigma, D_mat (Eq. (4),
 * Sec. 2.2), the ELL width W and a length histogram. Reads IRP only, which
 * is why Sec. 4.4 calls D_mat cheap to obtain. Also checks IRP: irp[0] = 0,
 * non-decreasing, irp[n_rows] = nnz, else SPMV_ERR_INVALID_MATRIX. */
spmv_status spmv_analyze(const spmv_crs *A, spmv_stats *out, spmv_stream_t stream);

/* SYNC. Full structural check of a CRS matrix (IRP as in spmv_analyze and
 * every ICOL in [0, n_cols)). SPMV_ERR_INVALID_MATRIX when it fails. */
spmv_status spmv_validate(const spmv_crs *A, spmv_stream_t stream);

/* Bytes of a padded ELL with `n_lines` lines and `width` slots per line
 * (float64 values plus int32 indices, leading dimension rounded up). */
uint64_t spmv_ell_bytes(int32_t n_lines, int32_t width);

/* Build a handle in `format`/`layout` from a CRS matrix (Sec. 2.1):
 *  - (SPMV_CRS, ROWWISE): the CRS itself plus its SpMV schedule (row bins);
 *    borrows IRP/ICOL/VAL. SYNC (runs spmv_analyze).
 *  - (SPMV_COO, ROWWISE): COO-Row, IROW(k) = row of entry k; borrows
 *    VAL/ICOL, which COO-Row shares with the CRS (Sec. 2.1). SYNC (it reads
 *    the size of its SpMV tiles).
 *  - (SPMV_ELL, ROWWISE): ELL-Row, width W = longest row, each row's entries
 *    in CRS order in slots 0..len-1, padding slots value +0.0 with the
 *    column of the row's last entry (0 for an empty row). SYNC.
 *  - (SPMV_CRS, COLWISE): Phase I of Sec. 2.1, CRS -> CCS (per-column
 *    count, prefix sum, scatter): each column lists its rows ascending, and
 *    repeated (i, j) entries in CRS order. SYNC.
 *  - (SPMV_COO, COLWISE): Phase I then Phase II (CCS -> COO-Column). SYNC.
 *  - (SPMV_ELL, COLWISE): Phase I then the CCS padded to ELL over columns
 *    (width = longest column, padding: +0.0 with the column's last row). SYNC.
 * Borrowed caller arrays must stay valid and unchanged until spmv_destroy.
 * `mem_cap_bytes` (0 = none) bounds the device bytes the handle owns; a
 * larger result returns SPMV_ERR_MEMORY_CAP before anything is allocated
 * (the memory policy the paper defers to its reference [7], Sec. 2.2). */
spmv_status spmv_transform(const spmv_crs *A, spmv_format format, spmv_layout layout,
                           uint64_t mem_cap_bytes, spmv_matrix **out, spmv_stream_t stream);

/* Transformation from an existing handle `src` that holds a CCS, i.e. a
 * (SPMV_CRS, COLWISE) or (SPMV_COO, COLWISE) handle (an ELL-Column handle
 * does not keep its CCS): to SPMV_COO (COO-Column, Phase II of Sec. 2.1) or
 * SPMV_ELL (ELL-Column). The new handle shares the CCS arrays with `src`;
 * the two may be destroyed in any order. Asynchronous; a bounded wait of the
 * ELL build that runs out is reported by spmv_matrix_status. */
spmv_status spmv_transform_from(const spmv_matrix *src, spmv_format format,
                                uint64_t mem_cap_bytes, spmv_matrix **out,
                                spmv_stream_t stream);

/* y = A x (Sec. 3) in the handle's format. x: device float64[n_cols], y:
 * device float64[n_rows], overwritten; x and y must not overlap. ELL-Row,
 * and CRS and COO-Row on rows of even length, sum every row in a fixed order
 * (bitwise repeatable). Column-wise formats add into y with atomics, and so
 * do CRS on uneven rows (D_mat > 0.5 or a row of 2048 entries or more) and
 * COO-Row when 128 rows hold more than 6144 entries: those rows are split
 * over threads, so their rounding order may vary between calls (every result
 * stays within the tolerance of a reordered sum). Asynchronous. */
spmv_status spmv_apply(const spmv_matrix *M, const double *x, double *y, spmv_stream_t stream);

/* Fused CRS -> ELL-Row transformation and first SpMV: builds the same
 * ELL-Row handle as spmv_transform(A, SPMV_ELL, SPMV_ROWWISE, ...) and, in
 * the same pass over the CRS, y = A x. SYNC. */
spmv_status spmv_transform_apply(const spmv_crs *A, const double *x, double *y,
                                 uint64_t mem_cap_bytes, spmv_matrix **out,
                                 spmv_stream_t stream);

/* SYNC. Reports whether any bounded device wait in the asynchronous build of
 * this handle or inside spmv_apply on it has run out (SPMV_ERR_TIMEOUT), else
 * SPMV_OK. Neither of those calls waits for the stream. */
spmv_status spmv_matrix_status(const spmv_matrix *M, spmv_stream_t stream);

/* Fill `out` with the handle's arrays and sizes. */
spmv_status spmv_describe(const spmv_matrix *M, spmv_matrix_desc *out);

/* Release a handle. Its device memory is freed in stream order on the stream
 * that created it; work on other streams that uses it must be ordered
 * before (or complete). NULL is ignored. */
void spmv_destroy(spmv_matrix *M);

/* Eqs. (1)-(3) of Sec. 2.2 with Eq. (2) read as TT = t_trans / t_crs:
 * R_ell = (t_crs / t_ell) / (t_trans / t_crs). Host only. */
double spmv_r_ell(double t_crs, double t_ell, double t_trans);

/* Off-line step (4) of Sec. 2.2: D* from m points (dmat[i], rell[i]) and
 * threshold c under `rule` (SPMV_DSTAR_*). PREFIX: points taken by ascending
 * D_mat (ties in input order); D* = D_mat of the first point with
 * R_ell < c, +inf if none fails, 0 if the first already fails. MAXPASS:
 * largest D_mat with R_ell >= c, 0 if none. Host only. */
spmv_status spmv_dstar_from_points(int32_t m, const double *dmat, const double *rell,
                                   double c, int32_t rule, double *dstar);

/* SYNC. Off-line measurement for one matrix (Sec. 2.2 steps (2)): median
 * device times of CRS SpMV, ELL-Row SpMV, the CRS -> ELL-Row transformation
 * and (with SPMV_AT_TRY_COO) COO-Row SpMV, then SP, TT, R_ell and D_mat.
 * SPMV_ERR_MEMORY_CAP if the ELL would exceed p->mem_cap_bytes. */
spmv_status spmv_measure(const spmv_crs *A, const spmv_at_params *p, spmv_timing *out,
                         spmv_stream_t stream);

/* SYNC. Measurement of the ceiling that binds the column-wise products
 * (Sec. 2.1 column-wise formats add every product into y with an FP64 atomic,
 * Fig. 1): the median device time (ms) of `reps` launches that do n_adds
 * FP64 atomic adds into n_targets doubles, lanes on consecutive elements
 * (their best case on banded matrices), and nothing else. */
spmv_status spmv_measure_atomics(int64_t n_targets, int64_t n_adds, int32_t reps, double *ms,
                                 spmv_stream_t stream);

/* SYNC. Off-line phase (Sec. 2.2 steps (1)-(4)): spmv_measure on each of the
 * m matrices, then D* by p->dstar_rule and p->c. dmat_out / rell_out (host
 * double[m], may be NULL) receive the D_mat-R_ell graph; a matrix whose ELL
 * exceeds the cap gets R_ell = 0 (never advantageous). */
spmv_status spmv_calibrate(const spmv_crs *const *set, int32_t m, const spmv_at_params *p,
                           double *dmat_out, double *rell_out, double *dstar_out,
                           spmv_stream_t stream);

/* SYNC. On-line phase (Sec. 2.2): D_mat of A (Eq. (4)); ELL-Row if
 * D_mat < p->dstar and the ELL fits p->mem_cap_bytes, otherwise CRS (or
 * COO-Row when SPMV_AT_TRY_COO is set and it measures faster). `chosen`
 * receives the handle, `stats` (may be NULL) the statistics. */
spmv_status spmv_autotune(const spmv_crs *A, const spmv_at_params *p, spmv_matrix **chosen,
                          spmv_stats *stats, spmv_stream_t stream);

/* SYNC. On-line phase of Sec. 2.2 without building anything: computes
 * D_mat (Eq. (4)) and returns in *format / *layout the format that
 * spmv_autotune would build (ELL-Row if D_mat < p->dstar and the ELL fits
 * p->mem_cap_bytes, else CRS; the SPMV_AT_TRY_COO timing is not run here).
 * `stats` may be NULL. */
spmv_status spmv_autotune_choose(const spmv_crs *A, const spmv_at_params *p, int32_t *format,
                                 int32_t *layout, spmv_stats *stats, spmv_stream_t stream);

/* COO-Row SpMV that allocates no device memory. The paper has no
 * counterpart: this is for callers that cannot allocate device memory while
 * they multiply, such as solvers that reserve all of their memory up front
 * from a fixed arena, or latency-critical loops where an allocation could
 * block or fail between iterations.
 * Computes y = A x like spmv_apply on a COO-Row handle, from caller-owned
 * device arrays: irow, icol (int32[nnz], irow non-decreasing, every index in
 * range), val (float64[nnz]), x (float64[n_cols]), y (float64[n_rows],
 * overwritten). Asynchronous; deterministic like spmv_apply.
 * Its temporary data (partial sums of rows that cross tile boundaries) lives
 * in one fixed device array of SPMV_NOALLOC_SCRATCH_BYTES that every GPU
 * loading the library holds until the process exits; the call allocates and
 * frees nothing. nnz above SPMV_NOALLOC_COO_MAX_NNZ returns
 * SPMV_ERR_UNSUPPORTED before touching the device. All calls share the
 * array: calls whose work overlaps on one device (several streams or host
 * threads) race on it and must be ordered by the caller. The first call on a
 * device looks up the array's device address (a CUDA runtime query, no
 * allocation) and keeps it for the life of the process; make that first call
 * before any stream capture. A cudaDeviceReset makes the kept address stale:
 * do not call this entry point on a device after resetting it. */
#define SPMV_NOALLOC_SCRATCH_BYTES ((1u << 20) + 256u)
#define SPMV_NOALLOC_COO_MAX_NNZ 134217728ll /* 65536 tiles of 2048 entries, 16 bytes of scratch each */
spmv_status spmv_apply_coo_row_noalloc(int32_t n_rows, int32_t n_cols, int64_t nnz, const int32_t *irow,
                                       const int32_t *icol, const double *val, const double *x, double *y,
                                       spmv_stream_t stream);

/* ---- Batches of independent matrices ------------------------------------
 * The paper's method handles one matrix per library call. A batch applies it
 * to m matrices at once: one analysis launch computes Eq. (4) for every
 * matrix and checks its CRS, the on-line rule of Sec. 2.2 is taken per
 * matrix (ELL-Row iff D_mat < p->dstar and the batch's ELL arrays, counted
 * matrix by matrix in order, stay within p->mem_cap_bytes; else CRS), one
 * launch builds all ELL-Row arrays (Sec. 2.1), and each product is one
 * launch over all matrices instead of one per matrix.
 *
 * Vectors are concatenated: matrix i reads x[x_offset_i, x_offset_i +
 * n_cols_i) and writes y[y_offset_i, y_offset_i + n_rows_i), where x_offset_i
 * is the sum of n_cols and y_offset_i the sum of n_rows of matrices 0..i-1.
 * The batch borrows every CRS array: keep them alive and unchanged until
 * spmv_batch_destroy. */
typedef struct spmv_batch spmv_batch;

typedef struct spmv_batch_info {
    int32_t n_matrices;
    int32_t n_ell;         /* matrices stored as ELL-Row */
    int64_t total_rows;    /* length of the concatenated y */
    int64_t total_cols;    /* length of the concatenated x */
    int64_t total_nnz;
    int64_t n_tiles;       /* row tiles of one product launch */
    int32_t grid;          /* CTAs of the persistent product launch */
    int32_t pad;
    uint64_t ell_bytes;    /* device bytes of all ELL-Row arrays */
    uint64_t owned_bytes;  /* all device bytes the batch keeps alive */
} spmv_batch_info;

/* Plan of one matrix of a batch. */
typedef struct spmv_batch_plan {
    double mu, sigma, dmat;   /* Eq. (4) */
    int32_t max_row_len;
    int32_t format;           /* SPMV_ELL or SPMV_CRS (row-wise) */
    int32_t threads_per_row;  /* CRS: lanes sharing a row (1, 8 or 32); ELL: 1 */
    int32_t rows_per_tile;    /* rows per warp tile; CRS with one lane per entry: at most this
                                 many rows and 256 entries (a longer row: a tile of its own) */
    int32_t width, ld;        /* ELL: slots per row and leading dimension; CRS: 0 */
    int64_t x_offset, y_offset;
    const double *ell_val;    /* ELL: device float64[width * ld], slot k of row r at k*ld + r;
                                 rows n_rows..ld-1 are not written. CRS: NULL */
    const int32_t *ell_idx;   /* ELL: column of each slot (padding: +0.0 value, the row's
                                 last column or 0 for an empty row). CRS: NULL */
} spmv_batch_plan;

/* SYNC (once, after the analysis launch; the ELL build is then enqueued
 * asynchronously). mats: host array of m CRS descriptors whose arrays are
 * device memory. p may be NULL (dstar 0: all CRS, no cap). If x and y
 * (device, concatenated as above) are both given, the build launch also
 * computes y = A x for every matrix; give both or neither. Errors:
 * SPMV_ERR_INVALID_ARG (bad sizes or pointers), SPMV_ERR_INVALID_MATRIX (any
 * matrix with a malformed IRP or a column index out of range), SPMV_ERR_OOM,
 * SPMV_ERR_UNSUPPORTED (m above 2^26). */
spmv_status spmv_batch_create(const spmv_crs *mats, int32_t m, const spmv_at_params *p, const double *x,
                              double *y, spmv_batch **out, spmv_stream_t stream);

/* y = A x for every matrix of the batch: one kernel launch, no allocation,
 * no synchronisation, no host work beyond the launch, so that the call can
 * be captured in a CUDA graph. Deterministic. x, y: device, concatenated. */
spmv_status spmv_batch_apply(const spmv_batch *B, const double *x, double *y, spmv_stream_t stream);

/* nvec products per matrix in one launch: y_j = A x_j for j < nvec, vector j
 * of the concatenated x at x + j * ldx (ldx >= total_cols), of y at
 * y + j * ldy (ldy >= total_rows). Each matrix's entries are read once for all
 * vectors. Every product has the bits spmv_batch_apply would give it. Like
 * spmv_batch_apply: no allocation, no synchronisation. */
spmv_status spmv_batch_apply_multi(const spmv_batch *B, const double *x, int64_t ldx, double *y, int64_t ldy,
                                   int32_t nvec, spmv_stream_t stream);

/* Sizes of a batch (host). */
spmv_status spmv_batch_info_get(const spmv_batch *B, spmv_batch_info *out);

/* Plans of matrices first .. first+count-1 into out[0..count-1] (host). */
spmv_status spmv_batch_plan_get(const spmv_batch *B, int32_t first, int32_t count, spmv_batch_plan *out);

/* Frees the batch's device memory (stream-ordered on the creating stream). */
void spmv_batch_destroy(spmv_batch *B);

/* A batch whose whole build runs on the device, so that it can be captured
 * in one CUDA graph together with its products. spmv_batch_prepare does the
 * host part only: it checks the descriptors, picks each CRS member's lanes
 * per row from the schedule table (from the member's mean row length, which
 * the descriptor gives), and allocates the descriptors, an upper bound of the
 * tile records and, when p->dstar > 0, an ELL pool of p->mem_cap_bytes bytes
 * (required then: SPMV_ERR_INVALID_ARG if 0). It launches nothing. SYNC.
 * spmv_batch_build then enqueues, with no allocation, no host work between
 * launches and no synchronisation: the analysis (Eq. (4)), the on-line rule
 * of Sec. 2.2 per matrix (ELL-Row iff D_mat < D* and the ELL arrays of the
 * members chosen before it, in matrix order, and its own fit the cap; the
 * same rule as spmv_batch_create), the tile records, the ELL build and, if x
 * and y are given (both or neither), the first product y = A x. It may be
 * called again (the same plan is rebuilt). Afterwards spmv_batch_apply and
 * spmv_batch_apply_multi run as for any batch, also inside a graph. A
 * malformed member makes the build do no product work; spmv_batch_status
 * (SYNC) then reports SPMV_ERR_INVALID_MATRIX. spmv_batch_info_get and
 * spmv_batch_plan_get on such a batch first wait for its stream (SYNC). */
spmv_status spmv_batch_prepare(const spmv_crs *mats, int32_t m, const spmv_at_params *p, spmv_batch **out,
                               spmv_stream_t stream);
spmv_status spmv_batch_build(spmv_batch *B, const double *x, double *y, spmv_stream_t stream);
/* SYNC (device-planned batches). Status of the last build. */
spmv_status spmv_batch_status(spmv_batch *B);

/* Schedule table of batches, an extension of the paper's on-line rule to the
 * product schedule: lanes per row (1, 8 or 32) of a CRS member by the class of
 * its mean row length mu = nnz / n_rows (class 0: mu < 1, class c >= 1: mu in
 * [2^(c-1), 2^c), the last class open-ended). The off-line phase measures the
 * batch product of each class under each choice and installs the fastest
 * (paper_2407_00019_gb300.calibrate --schedule). Process-wide; read when a
 * batch is created or prepared. The default: 1 below a mean of 32, 8 below
 * 256, 32 above. */
#define SPMV_BATCH_SCHED_CLASSES 10
spmv_status spmv_batch_schedule_set(const int32_t *tpr_by_class, int32_t n);
spmv_status spmv_batch_schedule_get(int32_t *tpr_by_class, int32_t n);

/* SYNC. Median device time (ms, CUDA events on `stream`) of `reps` batch
 * products y = A x after `warm` untimed ones: the measurement of the
 * off-line schedule calibration. */
spmv_status spmv_batch_time(const spmv_batch *B, const double *x, double *y, int32_t warm, int32_t reps,
                            double *ms, spmv_stream_t stream);

/* ---- Serving: continuous batching over a pool of matrices ----------------
 * A server owns N CUDA streams ("slots") and a worker thread. Clients
 * register matrices (the pool) and submit requests; a request asks for k
 * products y_j = A x_j with one matrix of the pool. The worker admits queued
 * requests in arrival order whenever a slot is free, so requests start and
 * finish independently (no batch barrier). Per matrix it keeps a resident
 * format cache: the on-line rule of Sec. 2.2 picks the target format at
 * registration (ELL-Row iff D_mat < dstar and its ELL fits the budget), and
 * the transformation is built, once, when the matrix has been asked for as
 * many products in total as it takes to pay for it: k >= TT / (1 - 1/SP)
 * (Sec. 2.2, Eqs. (1)-(3), with the bytes each step moves standing in for its
 * time), and at least amortize_products. A transformation that can never pay
 * (SP <= 1) or would fill more than a quarter of the budget is not built.
 * Until then, and whenever the cache is full, requests run on CRS. Cached formats are evicted
 * least-recently-used, never while a request uses them; the cache never holds
 * more than mem_budget_bytes. The paper has no serving layer: this is the
 * library's use of its method under a stream of requests. */
typedef struct spmv_server spmv_server;

#define SPMV_SERVER_FIXED_THRESHOLD 1 /* flag: build after amortize_products products, without the
                                          break-even model (only the budget limits the cache) */
#define SPMV_SERVER_PLAIN 2           /* flag: the per-matrix form, for comparison: one slot, requests
                                          one after the other in arrival order, each product one
                                          spmv_apply on the matrix's CRS handle, no format cache */
typedef struct spmv_server_params {
    uint64_t mem_budget_bytes;   /* device bytes the format cache may hold; 0 = no limit */
    double dstar;                /* D*: target format ELL-Row iff D_mat < dstar */
    int32_t n_streams;           /* slots (requests in flight); <= 0 means 4 */
    int32_t amortize_products;   /* least products seen before a transformation is built; <= 0 means 2 */
    int32_t flags;               /* SPMV_SERVER_FIXED_THRESHOLD or 0 */
    int32_t pad;
} spmv_server_params;

typedef struct spmv_server_stats {
    uint64_t submitted, completed, failed, products;
    double bytes;                /* algorithmic bytes of the completed products (byte model of the format used) */
    double p50_ms, p99_ms, mean_ms, max_ms; /* submit -> completion, completed requests */
    double busy_s;               /* first submission to last completion */
    uint64_t cache_hits;         /* requests served from a cached transformation */
    uint64_t cache_misses;       /* requests served in CRS while their target was ELL-Row */
    uint64_t transforms, evictions;
    uint64_t cache_bytes, peak_cache_bytes;
} spmv_server_stats;

/* Creates the server and its worker thread on the current CUDA device. */
spmv_status spmv_server_create(const spmv_server_params *p, spmv_server **out);

/* SYNC. Adds a matrix (device arrays owned by the caller, kept alive and
 * unchanged until spmv_server_destroy) to the pool: analysis, target format,
 * CRS schedule. *id receives its index. */
spmv_status spmv_server_add_matrix(spmv_server *S, const spmv_crs *A, int32_t *id);

/* Queues a request of k >= 0 products with matrix `id`: x (device,
 * k * n_cols float64, product j reads x + j * n_cols) and y (device,
 * k * n_rows float64, overwritten). If `after` is not NULL, the request
 * starts only after the work enqueued on that stream so far (the producer of
 * x); pass cudaStreamLegacy for the legacy default stream, since NULL here
 * means no such dependency. The caller keeps x and y alive until the request completes. *req
 * receives the request's id. Thread-safe. */
spmv_status spmv_server_submit(spmv_server *S, int32_t id, int32_t k, const double *x, double *y,
                               spmv_stream_t after, uint64_t *req);

/* Waits up to timeout_ms (< 0: no limit) for request `req`; then returns its
 * status (SPMV_ERR_TIMEOUT if it has not completed) and, if the pointers are
 * not NULL, its latency (ms) and the format it ran in. A request can be
 * waited for once. Thread-safe. */
spmv_status spmv_server_wait(spmv_server *S, uint64_t req, int32_t timeout_ms, double *latency_ms,
                             int32_t *format);

/* Waits up to timeout_ms for every submitted request. */
spmv_status spmv_server_drain(spmv_server *S, int32_t timeout_ms);

/* Counters and latency percentiles; reset != 0 clears them afterwards. */
spmv_status spmv_server_stats_get(spmv_server *S, spmv_server_stats *out, int32_t reset);

/* Drains, stops the worker and frees the cache and the streams. */
void spmv_server_destroy(spmv_server *S);

/* ---- Schedule hints --------------------------------------------------------
 * The library chooses every schedule itself from the matrix (row lengths,
 * column locality, tile sizes). A hint overrides one of those choices for the
 * whole process, so that a test can run every path on the same matrix and a
 * measurement can compare paths; every path gives the same transformation
 * bits and products within the tolerance of a reordered sum. Value 0 restores
 * the library's own choice; a value a matrix cannot take (for example a slot
 * path of Phase I on a matrix with no entries) is ignored for that matrix.
 * Hints are read when a handle or batch is built, not when it is applied.
 * Not synchronised with calls in flight on other host threads. */
#define SPMV_HINT_PHASE1 0     /* Phase I path (Sec. 2.1): SPMV_PHASE1_* below */
#define SPMV_HINT_CRS_SPLIT 1  /* CRS on regular rows: 1, 2, 4 or 8 threads per row of a staged
                                  128-row tile; -1: V lanes per row without staging */
#define SPMV_HINT_COO_FLAT 2   /* 1: COO-Row as the entry-split product, COO-Column as one
                                  atomic add per entry (the paths taken when a tile does not fit) */
#define SPMV_HINT_BATCH_TPR 3  /* batches: lanes per row of every CRS member, 1, 8 or 32 */
#define SPMV_HINT_COUNT 4
#define SPMV_PHASE1_COUNT 1    /* count, prefix sum, scatter of (k, row), per-column sort */
#define SPMV_PHASE1_KSLOT 2    /* (k, row) slots with ranks */
#define SPMV_PHASE1_ROWPOS 3   /* {k, row} slots sorted by row in registers */
#define SPMV_PHASE1_GROUPED 4  /* {row, value} records per 64-column group */
#define SPMV_PHASE1_SYMMETRIC 5 /* structurally symmetric matrices: IRP_T = IRP, ICOL_T = ICOL, values
                                  gathered from the mirror entries (other matrices: the library's choice) */

/* Set hint `hint` (SPMV_HINT_*) to `value`; SPMV_ERR_INVALID_ARG for an
 * unknown hint. */
spmv_status spmv_set_hint(int32_t hint, int32_t value);

/* Current value of a hint (0 for an unknown one). */
int32_t spmv_get_hint(int32_t hint);

/* Instrumentation: number of kernels this library has launched so far. */
uint64_t spmv_launch_count(void);

/* Turn per-kernel timing on (1) or off (0). While on, each launch is
 * bracketed by CUDA events on its stream. */
spmv_status spmv_profile_enable(int32_t on);

/* SYNC on the recorded events. Copies up to `cap` per-kernel totals into
 * `out` (host), returns how many kernels have totals; `reset` != 0 clears. */
int32_t spmv_profile_read(spmv_kernel_time *out, int32_t cap, int32_t reset);

/* SYNC. Test hook for the bounded waits: runs the decoupled look-back scan
 * on `n` device counters with a first tile that never publishes its sum and
 * a spin limit of `spin_limit` polls, so every later tile must give up.
 * Returns the status the scan reports (SPMV_ERR_TIMEOUT expected) in
 * *observed. Leaves the device usable. */
spmv_status spmv_debug_scan_timeout(int32_t n, int32_t spin_limit, int32_t *observed,
                                    spmv_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* SPMVAT_H */
