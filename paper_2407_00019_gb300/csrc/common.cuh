// Shared device helpers and the internal launcher interface of libspmvat.
// Target: sm_103a (GB300). All kernels are written for 32-wide warps,
// 152 SMs, up to 227 KB of shared memory per CTA and TMA bulk copies.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace spmvat {

// Bits OR-ed into a device status word by kernels.
enum : int {
    ST_BAD_INDEX = 1,  // an index (column / row / position) out of range
    ST_TIMEOUT = 2,    // a bounded wait ran out
    ST_BAD_PTR = 4,    // IRP not 0 .. nnz or not non-decreasing
    ST_REDO = 8,       // a fast path met a case it does not cover (internal:
                       // the host reruns the step on the general path)
};

// Per-call accumulator of spmv_analyze (one device struct).
struct AnalyzeAcc {
    unsigned long long sum_len;
    unsigned long long sum_len2;
    unsigned long long n_empty;
    unsigned long long hist[32];
    int max_len;
    int min_len;
    int status;
    int pad;
};

// Bounded-wait budget: polls of a flag or mbarrier before a kernel gives up
// and reports ST_TIMEOUT. With the backoff used below this is ~1-2 s.
constexpr long long kSpinLimit = 1ll << 22;

// ---------------------------------------------------------------- host side
// Launch accounting and optional per-kernel event timing (api.cu).
struct KernelScope {
    KernelScope(const char *name, cudaStream_t s);
    ~KernelScope();
    int slot;
    cudaStream_t stream;
};
int sm_count();  // SMs of the current device (cached)
int hint_value(int hint);  // spmv_set_hint value (0: the library's choice)

inline unsigned ceil_div_u(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

// Raise a kernel's dynamic shared-memory limit (cheap host call; made before
// every launch so that each device and each instantiation gets it).
template <class K>
cudaError_t set_smem_attr(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// ------------------------------------------------------------- device side
__device__ __forceinline__ unsigned lane_id() {
    unsigned l;
    asm volatile("mov.u32 %0, %%laneid;" : "=r"(l));
    return l;
}
__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// 32-byte global stores (sm_100 and later), streaming cache policy: a thread
// that owns 32 consecutive bytes writes them in one instruction, so a warp's
// store covers whole 32-byte sectors. Two 16-byte stores per thread instead
// leave every sector half-written by each instruction; on GB300 that pattern
// wrote a 223 MB buffer at 0.6 of the rate of whole-sector stores. (Loads in
// the same pattern lose nothing: the second half of a sector hits L1.) The
// address must be 32-byte aligned.
__device__ __forceinline__ void st_cs_v8(int32_t *p, const int (&v)[8]) {
    asm volatile("st.global.cs.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
                 :: "l"(p), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}
__device__ __forceinline__ void st_cs_v4d(double *p, double a, double b, double c, double d) {
    asm volatile("st.global.cs.v4.f64 [%0], {%1, %2, %3, %4};" :: "l"(p), "d"(a), "d"(b), "d"(c), "d"(d) : "memory");
}

// Largest i in [lo, hi) with a[i] <= key, given a[lo] <= key (a sorted).
__device__ __forceinline__ int last_le(const int32_t *a, int lo, int hi, long long key) {
    while (hi - lo > 1) {
        int mid = lo + ((hi - lo) >> 1);
        if ((long long)a[mid] <= key) lo = mid; else hi = mid;
    }
    return lo;
}

// ---- mbarrier + TMA bulk copy (global -> shared), inline PTX -------------
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Poll with backoff; false after `limit` polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity, long long limit) {
    for (long long i = 0; i < limit; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (i > 16) __nanosleep(256);
    }
    return false;
}
// 1-D bulk copy of `bytes` (multiple of 16; both addresses 16-byte aligned)
// from global memory into this CTA's shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void *sdst, const void *gsrc, unsigned bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(sdst)),
        "l"(gsrc), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// ---- cp.async (global -> shared, 4 / 8-byte granules), commit groups ------
__device__ __forceinline__ void cp_async_8(void *s, const void *g) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_4(void *s, const void *g) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// ---- acquire/release accesses for the look-back scan ----------------------
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// ---- warp / block reductions ----------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// --------------------------------------------------------------- launchers
// All return cudaGetLastError() after enqueueing on `s`.

// analyze / validate (kernels_rowwise.cu)
// The longest row and the row-pointer checks of launch_analyze only (what
// an ELL build needs): max_len and status of `acc` (zeroed by the caller).
cudaError_t launch_row_width(const int32_t *irp, int32_t n_rows, int64_t nnz, AnalyzeAcc *acc, cudaStream_t s);
cudaError_t launch_analyze(const int32_t *irp, int32_t n_rows, int64_t nnz, AnalyzeAcc *acc, cudaStream_t s);
cudaError_t launch_validate_idx(const int32_t *idx, int64_t n, int32_t bound, int *status, cudaStream_t s);

// tile_lines: out[t] = line holding entry t*tile, t < ceil(nnz/tile)
size_t tile_lines_bytes(int64_t nnz, int tile);
cudaError_t launch_tile_lines(const int32_t *ptr, int32_t n_lines, int64_t nnz, int tile, int32_t *out,
                              cudaStream_t s);

// pointer expansion: out[k] = line of entry k (COO-Row IROW, Phase II column)
cudaError_t launch_expand(const int32_t *ptr, int32_t n_lines, int64_t nnz, int32_t *out, cudaStream_t s,
                          const char *name = "expand");

// compressed lines -> padded column-major ELL; optional fused y = A x
cudaError_t launch_lines_to_ell(const int32_t *ptr, const int32_t *idx, const double *val, int32_t n_lines,
                                int32_t idx_bound, int32_t width, int32_t ld, double *eval, int32_t *eidx,
                                const double *x, double *y, int *status, cudaStream_t s,
                                const char *name = "lines_to_ell");

// Phase I (kernels_colwise.cu)
cudaError_t launch_col_count(const int32_t *icol, int64_t nnz, int32_t n_cols, int32_t *nc, int32_t *rank,
                             int *status, cudaStream_t s);
// Exclusive scan in place over a[0..n) with a[n] = total; also max element
// (atomicMax into *maxv) and, when long_list != NULL, the indices of
// elements > long_thresh appended to long_list (count in *long_count).
size_t scan_scratch_bytes(int64_t n);
cudaError_t launch_scan(int32_t *a, int64_t n, void *scratch, int32_t *maxv, int32_t long_thresh,
                        int32_t *long_list, int32_t *long_count, int *status, long long spin_limit,
                        int debug_stall_first, cudaStream_t s);
size_t col_scatter_scratch_bytes(int64_t nnz);
// Places entries with rank >= min_rank at IRP_T[col] + rank as (k, row).
// With only_if != NULL the grid returns at once when *only_if == 0.
// have_tile_lines: `scratch` already holds the tile lines of this nnz.
cudaError_t launch_col_scatter(const int32_t *irp, int32_t n_rows, const int32_t *icol, int64_t nnz,
                               int32_t n_cols, const int32_t *cp, const int32_t *rank, int2 *pairs,
                               int32_t *scratch, int *status, cudaStream_t s, int min_rank = 0,
                               const int32_t *only_if = nullptr, bool have_tile_lines = false);
// Slot path of Phase I: count + place ranks < col_slot_cap() in T (slot-major).
size_t col_slot_bytes(int32_t n_cols);
int col_slot_cap();
cudaError_t launch_col_claim(const int32_t *irp, int32_t n_rows, const int32_t *icol, int64_t nnz, int32_t n_cols,
                             int32_t *nc, int32_t *rank, int2 *T, int32_t *n_over, int32_t *scratch, int *status,
                             cudaStream_t s);
cudaError_t launch_col_fixup_slots(const int32_t *cp, int32_t n_cols, const int32_t *irp, int32_t n_rows,
                                   const double *val, const int2 *T, int2 *pairs, const int32_t *long_list,
                                   int32_t *keys_tmp, int32_t *trow, double *tval, cudaStream_t s);
// Row-position slot path of Phase I (no repeated (i, j) entries, columns of
// at most col_rv_long_cap() entries, at most `ov_cap` entries beyond the
// slots; otherwise ST_REDO; rows below 2^27 - 1). `slots`:
// col_rk_slot_bytes(n_cols) bytes of {k, row} records. The claim's `scratch`
// is unused (its rows are owned by lanes).
size_t col_rk_slot_bytes(int32_t n_cols);
int col_rv_long_cap();
cudaError_t launch_col_claim_rk(const int32_t *irp, int32_t n_rows, const int32_t *icol, int64_t nnz, int32_t n_cols,
                                int32_t *nc, void *slots, int4 *ov, int64_t ov_cap, int32_t *n_ov, int32_t *scratch,
                                int *status, cudaStream_t s);
cudaError_t launch_col_fixup_rk(const int32_t *cp, int32_t n_cols, int32_t n_rows, const double *val,
                                const void *slots, const int4 *ov, int64_t ov_cap, const int32_t *n_ov,
                                const int32_t *long_list, int32_t *trow, double *tval, int *status, cudaStream_t s);
// Grouped row-value path of Phase I: records in regions of 64-column groups
// (col_grp_region_bytes), group counts gcnt (col_grp_count + 1 entries, zeroed)
// turned into the groups' first positions by launch_scan before the fix-up.
long long col_grp_count(int32_t n_cols);
size_t col_grp_region_bytes(int32_t n_cols);
size_t col_grp_scratch_bytes(int64_t nnz);  // tile lines of the claim's tiles
// number of `samples` evenly spread entries k with 1 <= ICOL[k+1] - ICOL[k] <= 8,
// added into *out
cudaError_t launch_col_locality(const int32_t *icol, int64_t nnz, int samples, int32_t *out, cudaStream_t s);
cudaError_t launch_col_claim_grp(const int32_t *irp, int32_t n_rows, const int32_t *icol, const double *val,
                                 int64_t nnz, int32_t n_cols, int32_t *gcnt, void *regions, int32_t *scratch,
                                 int *status, cudaStream_t s);
// writes IRP_T (cp), ICOL_T, VAL_T, the longest column and the long-column list
// (preceded by its count)
cudaError_t launch_col_fixup_grp(const int32_t *gpos, int32_t n_cols, const void *regions, int32_t *cp,
                                 int32_t *trow, double *tval, int32_t *colmax, int32_t *long_list, int *status,
                                 cudaStream_t s);
// Structurally symmetric path of Phase I (square matrices): ICOL_T = ICOL and
// VAL_T[p] = VAL[mirror of p]; ST_REDO when an entry has no mirror or a row is
// not strictly ascending. cnt (zeroed u64[3]): [2] receives the longest row.
// `scratch`: ccs_sym_scratch_bytes(nnz).
size_t ccs_sym_scratch_bytes(int64_t nnz);
cudaError_t launch_ccs_sym(const int32_t *irp, int32_t n, const int32_t *icol, const double *val, int64_t nnz,
                           int32_t *scratch, int32_t *trow, double *tval, unsigned long long *cnt, int *status,
                           cudaStream_t s);
// failures of the symmetric path's conditions among one entry of each of
// `samples` evenly spread rows, added into *fails
cudaError_t launch_sym_sample(const int32_t *irp, int32_t n, const int32_t *icol, int64_t nnz, int samples,
                              int32_t *fails, cudaStream_t s);
// `pairs` must have 16 bytes of slack after its nnz elements.
// `long_list` is preceded by its device-side count.
cudaError_t launch_col_fixup(const int32_t *cp, int32_t n_cols, const int32_t *irp, int32_t n_rows,
                             const double *val, int2 *pairs, const int32_t *long_list, int32_t *keys_tmp,
                             int32_t *trow, double *tval, int *status, cudaStream_t s);

// SpMV (kernels_spmv.cu)
cudaError_t launch_spmv_crs_vector(int v, const int32_t *irp, const int32_t *icol, const double *val,
                                   const int32_t *rows, int64_t count, const double *x, double *y,
                                   cudaStream_t s);
int crs_rows_cap(int max_row_len);
cudaError_t launch_spmv_crs_rows(int split, int cap, const int32_t *irp, const int32_t *icol, const double *val,
                                 int32_t n_rows, const double *x, double *y, cudaStream_t s);
cudaError_t launch_spmv_ell_row(const double *eval, const int32_t *eidx, int32_t n_rows, int32_t width,
                                int32_t ld, const double *x, double *y, cudaStream_t s);
// nnz: the entries of the matrix (not the slots); with padding at least a
// quarter of the slots, the adds of zero slots are left out where x_j is finite.
cudaError_t launch_spmv_ell_col(const double *eval, const int32_t *eidx, int32_t n_rows, int32_t n_cols,
                                int32_t width, int32_t ld, int64_t nnz, const double *x, double *y, cudaStream_t s);
// COO-Row over 2048-entry tiles with a carry pass (the allocation-free entry
// point). `scratch`: coo_row_scratch_bytes(nnz); `status` may be NULL (then a
// word inside the scratch is used).
size_t coo_row_scratch_bytes(int64_t nnz);
cudaError_t launch_spmv_coo_row(const int32_t *irow, const int32_t *icol, const double *val, int64_t nnz,
                                int32_t n_rows, int32_t n_cols, const double *x, double *y, void *scratch,
                                int *status, cudaStream_t s);
// line-aligned COO: tile bounds (int32[ceil(n_lines/128) + 1]) from the line pointers, largest tile
cudaError_t launch_line_tile_bounds(const int32_t *ptr, int32_t n_lines, int64_t nnz, int32_t *tb, int32_t *maxn,
                                    const char *name, cudaStream_t s);
int coo_rows_cap(int max_n);
cudaError_t launch_spmv_coo_row_rows(int split, int cap, const int32_t *irow, const int32_t *icol,
                                     const double *val, const int32_t *tb, int32_t n_rows, int32_t n_cols,
                                     const double *x, double *y, cudaStream_t s);
// COO-Column over 128-column tiles (tb from launch_line_tile_bounds; cap from
// coo_rows_cap of the largest tile); zeroes y first.
cudaError_t launch_spmv_coo_col_cols(int split, int cap, const int32_t *trow, const int32_t *tcol, const double *tval,
                                     const int32_t *tb, int32_t n_rows, int32_t n_cols, const double *x, double *y,
                                     cudaStream_t s);
// Entry-split products for uneven rows (CRS: tl from launch_spmv_seg_lines,
// spmv_seg_scratch_bytes; COO: lines = IROW, tl unused); zero y first.
size_t spmv_seg_scratch_bytes(int64_t nnz);
cudaError_t launch_spmv_seg_lines(const int32_t *irp, int32_t n_rows, int64_t nnz, int32_t *tl, cudaStream_t s);
cudaError_t launch_spmv_seg(bool coo, const int32_t *lines, const int32_t *icol, const double *val, int64_t nnz,
                            int32_t n_rows, int32_t n_cols, const int32_t *tl, const double *x, double *y,
                            cudaStream_t s);
// n_adds coalesced FP64 atomic adds into y[0..n) (measurement of the
// column-wise products' ceiling)
cudaError_t launch_atomic_ceiling(double *y, long long n, long long n_adds, cudaStream_t s);
cudaError_t launch_spmv_coo_col(const int32_t *row, const int32_t *col, const double *val, int64_t nnz,
                                int32_t n_rows, const double *x, double *y, cudaStream_t s);
cudaError_t launch_spmv_ccs(const int32_t *cp, const int32_t *trow, const double *tval, int32_t n_rows,
                            int32_t n_cols, const double *x, double *y, cudaStream_t s);

// Batches of independent matrices (kernels_batch.cu). One descriptor per
// matrix; work items ("tiles") are records {matrix and row count, first
// row, first entry, entry count} of at most 32 rows that never cross a
// matrix, ordered by matrix.
enum : int { BATCH_CRS = 0, BATCH_ELL = 2 };
struct BatchMat {
    const int32_t *irp, *icol;  // the caller's CRS
    const double *val;
    double *eval;               // ELL-Row slots (column-major, leading dim ld) or NULL
    int32_t *ecol;
    long long xoff, yoff;       // segment offsets in the concatenated x and y
    long long nnz;
    int n_rows, n_cols;
    int width, ld;              // ELL width and leading dimension
    int fmt;                    // BATCH_CRS or BATCH_ELL
    int tpr;                    // CRS tiles: lanes per row (1, 8, 32)
    int rpt;                    // rows per tile (1..32; CRS with one lane per entry: at most)
    int pad;
};
struct BatchAcc {               // per-matrix statistics of the analysis pass
    unsigned long long sum_len, sum_len2;
    int max_len;
    int min_len;                // stored as INT_MAX - min so that atomicMax applies
    int n_empty;
    int status;
};
constexpr int kBatchThreads = 256;
constexpr int kBatchMatBits = 26;  // tile records pack the matrix index (< 2^26) and the row count
constexpr int kBatchChunk = 2048; // rows per work item of the analysis pass
int batch_grid(int kernel);       // persistent grid: 0 analyze, 1 build, 2 build+multiply, 3 apply, 4 multi
cudaError_t launch_batch_analyze(const BatchMat *mats, const int2 *chunks, long long n_chunks, BatchAcc *acc,
                                 cudaStream_t s);
// ELL transform of the ELL matrices' tiles; with x (and y) also y = A x for
// every tile given.
// Tile records of every matrix: with tiles == NULL the count per matrix
// into cnt[m]; otherwise the records, matrix i's from tiles[cnt[i]] on.
cudaError_t launch_batch_tiles(const BatchMat *mats, int m, long long *cnt, int4 *tiles, cudaStream_t s,
                               const long long *d_nt = nullptr);
// d_nt (optional): the tile count in device memory (a batch planned on the
// device); `n_tiles` then bounds it and only sizes the grid.
cudaError_t launch_batch_build(const BatchMat *mats, const int4 *tiles, long long n_tiles, const double *x,
                               double *y, cudaStream_t s, const long long *d_nt = nullptr);
cudaError_t launch_batch_apply(const BatchMat *mats, const int4 *tiles, long long n_tiles, const double *x,
                               double *y, cudaStream_t s, const long long *d_nt = nullptr);
// nvec products y_j = A x_j (vector j at x + j * ldx, y + j * ldy), one launch.
cudaError_t launch_batch_apply_multi(const BatchMat *mats, const int4 *tiles, long long n_tiles, const double *x,
                                     long long ldx, double *y, long long ldy, int nvec, cudaStream_t s,
                                     const long long *d_nt = nullptr);
// The plan of a batch on the device (graph-capturable build): per matrix the
// statistics of Eq. (4) into plans, the on-line rule with the cap in matrix
// order, ELL pointers into `pool`; bytes: scratch u64[2m]; tot (zeroed u64[2]):
// number of ELL members and their bytes. Errors of the analysis go to *status.
struct BatchPlanOut {
    double mu, sigma, dmat;
    int max_row_len;
    int pad;
};
cudaError_t launch_batch_plan(BatchMat *mats, const BatchAcc *acc, int m, double dstar, unsigned long long cap,
                              unsigned char *pool, unsigned long long *bytes, BatchPlanOut *plans,
                              unsigned long long *tot, int *status, cudaStream_t s);
// Exclusive scan of the tile counts in place, total into *n_tiles (0 and
// ST_REDO when it exceeds cap).
cudaError_t launch_batch_tile_offsets(long long *cnt, int m, long long cap, long long *n_tiles, int *status,
                                      cudaStream_t s);

}  // namespace spmvat
