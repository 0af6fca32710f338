// C ABI of libspmvat (declared in include/spmvat.h): handles, device memory,
// dispatch to the kernels, and the run-time AT method of Sec. 2.2.
#include <algorithm>
#include <atomic>
#include <cfloat>
#include <climits>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "host_mem.h"
#include "spmvat.h"

using namespace spmvat;

namespace {

// ------------------------------------------------------------------ memory
std::mutex g_mu;
Hooks g_hooks;
cudaMemPool_t g_pools[64] = {};

cudaMemPool_t pool_for(int dev) {
    std::lock_guard<std::mutex> lk(g_mu);
    dev &= 63;
    if (!g_pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        if (cudaMemPoolCreate(&p, &props) != cudaSuccess) { cudaGetLastError(); return nullptr; }
        unsigned long long keep = ULLONG_MAX;  // keep freed blocks for reuse
        cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        // never make one stream wait for another to reuse a block: callers
        // run independent transformations on several streams at once
        int no = 0;
        cudaMemPoolSetAttribute(p, cudaMemPoolReuseAllowInternalDependencies, &no);
        g_pools[dev] = p;
    }
    return g_pools[dev];
}

}  // namespace

namespace spmvat {

spmv_status alloc_buf(size_t bytes, cudaStream_t s, BufPtr *out) {
    Hooks h;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        h = g_hooks;
    }
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    void *p = nullptr;
    if (h.alloc) {
        p = h.alloc(bytes, h.ctx, s);
    } else {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return SPMV_ERR_CUDA; }
        cudaMemPool_t pool = pool_for(dev);
        if (!pool) return SPMV_ERR_CUDA;
        cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, pool, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return e == cudaErrorMemoryAllocation ? SPMV_ERR_OOM : SPMV_ERR_CUDA;
        }
    }
    if (!p) return SPMV_ERR_OOM;
    auto b = std::make_shared<DevBuf>();
    b->p = p;
    b->bytes = bytes;
    b->stream = s;
    b->hooks = h;
    *out = b;
    return SPMV_OK;
}

spmv_status status_from_dev(int st) {
    if (st & ST_TIMEOUT) return SPMV_ERR_TIMEOUT;
    if (st & (ST_BAD_INDEX | ST_BAD_PTR)) return SPMV_ERR_INVALID_MATRIX;
    return SPMV_OK;
}

// Schedule hints (spmv_set_hint): process-wide, 0 = the library's choice.
static std::atomic<int> g_hints[SPMV_HINT_COUNT];
int hint_value(int hint) { return (hint >= 0 && hint < SPMV_HINT_COUNT) ? g_hints[hint].load() : 0; }

}  // namespace spmvat

namespace {

// ------------------------------------------------------- launch accounting
std::atomic<unsigned long long> g_launches{0};
std::atomic<int> g_profile_on{0};
struct ProfRec {
    std::string name;
    cudaEvent_t e0, e1;
};
std::mutex g_pmu;
std::vector<ProfRec> g_pending;
std::vector<cudaEvent_t> g_event_pool;
std::map<std::string, std::pair<unsigned long long, double>> g_totals;

cudaEvent_t get_event() {
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    return e;
}

int g_sm_count[64] = {};

inline cudaStream_t S(spmv_stream_t s) { return reinterpret_cast<cudaStream_t>(s); }
inline int32_t round_up32(int64_t n) { return (int32_t)((n + 31) / 32 * 32); }
inline uint64_t ell_bytes(int64_t lines, int64_t width) {
    return (uint64_t)round_up32(lines) * (uint64_t)width * 12ull;
}

spmv_status check_crs(const spmv_crs *A) {
    if (!A) return SPMV_ERR_INVALID_ARG;
    if (A->n_rows <= 0 || A->n_cols <= 0 || A->nnz < 0 || A->nnz >= (int64_t)INT_MAX) return SPMV_ERR_INVALID_ARG;
    if (!A->irp) return SPMV_ERR_INVALID_ARG;
    if (A->nnz > 0 && (!A->icol || !A->val)) return SPMV_ERR_INVALID_ARG;
    return SPMV_OK;
}

}  // namespace

// --------------------------------------------------------------- handles
struct spmv_matrix {
    int32_t format = 0, layout = 0;
    int32_t n_rows = 0, n_cols = 0;
    int64_t nnz = 0;
    int32_t width = 0, ld = 0;
    const int32_t *ptr = nullptr;
    const int32_t *idx = nullptr;
    const int32_t *idx2 = nullptr;
    const double *val = nullptr;
    std::vector<BufPtr> bufs;      // everything this handle keeps alive
    std::vector<BufPtr> ccs_bufs;  // the CCS arrays (column-wise handles), shareable
    int32_t colmax = 0;            // longest column (handles holding a CCS)
    cudaStream_t home = nullptr;
    // CRS schedule
    int crs_seg = 0;               // entry-split product (uneven rows)
    const int32_t *seg_tl = nullptr; //    and the tile lines it needs
    int coo_seg = 0;               // COO-Row entry-split product
    int crs_v = 1;
    int coo_rows_split = 0;        // > 0: COO over row- (column-) aligned tiles, threads per line
    int coo_rows_cap = 0;          //      shared-memory entries per tile
    const int32_t *coo_tb = nullptr; //    tile bounds
    int crs_rows_split = 0;        // > 0: ELL-order row-tile kernel, threads per row
    int crs_rows_cap = 0;          //      and its shared-memory capacity (entries)
    int *status = nullptr;         // device status word of bounded waits in apply
    uint64_t owned() const {
        uint64_t t = 0;
        for (auto &b : bufs) t += b->bytes;
        return t;
    }
};

namespace spmvat {

KernelScope::KernelScope(const char *name, cudaStream_t s) : slot(-1), stream(s) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (!g_profile_on.load(std::memory_order_relaxed)) return;
    std::lock_guard<std::mutex> lk(g_pmu);
    cudaEvent_t e0 = get_event(), e1 = get_event();
    if (!e0 || !e1) return;
    cudaEventRecord(e0, s);
    g_pending.push_back({name, e0, e1});
    slot = (int)g_pending.size() - 1;
}
KernelScope::~KernelScope() {
    if (slot < 0) return;
    std::lock_guard<std::mutex> lk(g_pmu);
    if (slot < (int)g_pending.size()) cudaEventRecord(g_pending[slot].e1, stream);
}

int sm_count() {
    int dev = 0;
    cudaGetDevice(&dev);
    dev &= 63;
    if (!g_sm_count[dev]) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        g_sm_count[dev] = n > 0 ? n : 1;
    }
    return g_sm_count[dev];
}

}  // namespace spmvat

namespace {

// ------------------------------------------------------------- analyze core
// Runs k_analyze (+ optional ICOL validation) and returns the statistics.
spmv_status analyze_core(const spmv_crs *A, bool validate_icol, spmv_stats *out, cudaStream_t s) {
    BufPtr acc_buf;
    CKS(alloc_buf(sizeof(AnalyzeAcc), s, &acc_buf));
    AnalyzeAcc *acc = reinterpret_cast<AnalyzeAcc *>(acc_buf->p);
    CK(cudaMemsetAsync(acc, 0, sizeof(AnalyzeAcc), s));
    CK(launch_analyze(A->irp, A->n_rows, A->nnz, acc, s));
    if (validate_icol && A->nnz > 0) CK(launch_validate_idx(A->icol, A->nnz, A->n_cols, &acc->status, s));
    AnalyzeAcc h;
    CK(cudaMemcpyAsync(&h, acc, sizeof(AnalyzeAcc), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    spmv_status st = status_from_dev(h.status);
    if (st != SPMV_OK) return st;
    if ((long long)h.sum_len != A->nnz) return SPMV_ERR_INVALID_MATRIX;
    const double n = (double)A->n_rows;
    // sigma^2 = (n * S2 - S1^2) / n^2, numerator exact in 128-bit integers
    const unsigned __int128 num =
        (unsigned __int128)(unsigned long long)A->n_rows * h.sum_len2 -
        (unsigned __int128)h.sum_len * h.sum_len;
    const double mu = (double)h.sum_len / n;
    const double sigma = std::sqrt((double)num) / n;
    memset(out, 0, sizeof(*out));
    out->mu = mu;
    out->sigma = sigma;
    out->dmat = (h.sum_len == 0) ? 0.0 : sigma / mu;
    out->max_row_len = h.max_len;
    out->min_row_len = INT_MAX - h.min_len;
    out->n_empty_rows = (int64_t)h.n_empty;
    out->ell_bytes = ell_bytes(A->n_rows, h.max_len);
    for (int c = 0; c < 32; ++c) out->row_len_hist[c] = (int64_t)h.hist[c];
    return SPMV_OK;
}

// The longest row and the row-pointer checks only (an ELL-Row build needs no
// other statistic): st->max_row_len and st->ell_bytes, the rest zero.
spmv_status analyze_width(const spmv_crs *A, spmv_stats *out, cudaStream_t s) {
    BufPtr acc_buf;
    CKS(alloc_buf(sizeof(AnalyzeAcc), s, &acc_buf));
    AnalyzeAcc *acc = reinterpret_cast<AnalyzeAcc *>(acc_buf->p);
    CK(cudaMemsetAsync(acc, 0, sizeof(AnalyzeAcc), s));
    CK(launch_row_width(A->irp, A->n_rows, A->nnz, acc, s));
    AnalyzeAcc h;
    CK(cudaMemcpyAsync(&h, acc, sizeof(AnalyzeAcc), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    CKS(status_from_dev(h.status));
    memset(out, 0, sizeof(*out));
    out->max_row_len = h.max_len;
    out->ell_bytes = ell_bytes(A->n_rows, h.max_len);
    return SPMV_OK;
}

spmv_matrix *new_handle(const spmv_crs *A, int format, int layout, cudaStream_t s) {
    spmv_matrix *M = new (std::nothrow) spmv_matrix();
    if (!M) return nullptr;
    M->format = format;
    M->layout = layout;
    M->n_rows = A->n_rows;
    M->n_cols = A->n_cols;
    M->nnz = A->nnz;
    M->home = s;
    return M;
}

// Lanes per row of the vector CRS kernel (rows too long for a staged tile):
// half the largest power of two at or below the longest row, 1..32.
int vector_lanes(int max_len) {
    int v = 1;
    while (v < 32 && 2 * (v * 2) <= max_len) v *= 2;
    return v;
}

// The column-index check of a CRS whose IRP analyze_core has already checked.
spmv_status validate_icol(const spmv_crs *A, cudaStream_t s) {
    if (A->nnz <= 0) return SPMV_OK;
    BufPtr w;
    CKS(alloc_buf(16, s, &w));
    CK(cudaMemsetAsync(w->p, 0, 16, s));
    CK(launch_validate_idx(A->icol, A->nnz, A->n_cols, reinterpret_cast<int *>(w->p), s));
    int h = 0;
    CK(cudaMemcpyAsync(&h, w->p, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return status_from_dev(h);
}

spmv_status crs_plan_from(const spmv_crs *A, const spmv_stats &st, uint64_t cap, spmv_matrix **out, cudaStream_t s);

spmv_status build_crs_plan(const spmv_crs *A, uint64_t cap, spmv_matrix **out, cudaStream_t s) {
    spmv_stats st;
    CKS(analyze_core(A, true, &st, s));
    return crs_plan_from(A, st, cap, out, s);
}

// CRS schedule from statistics of an analysed, index-checked CRS.
spmv_status crs_plan_from(const spmv_crs *A, const spmv_stats &st, uint64_t cap, spmv_matrix **out, cudaStream_t s) {
    std::unique_ptr<spmv_matrix> M(new_handle(A, SPMV_CRS, SPMV_ROWWISE, s));
    if (!M) return SPMV_ERR_OOM;
    M->ptr = A->irp;
    M->idx = A->icol;
    M->val = A->val;
    const bool regular = st.dmat <= 0.5 && st.max_row_len < 2048;
    if (regular) {
        // Regular rows: 128-row tiles staged in shared memory with SPLIT
        // threads per row, or, when a tile of the longest rows would not fit,
        // V lanes per row. SPMV_HINT_CRS_SPLIT forces SPLIT (or, -1, the
        // vector kernel) for tests and measurements.
        const int hint = hint_value(SPMV_HINT_CRS_SPLIT);
        const int cap = crs_rows_cap(st.max_row_len);
        int split = st.mu <= 8.0 ? 2 : 4;
        if (hint == 1 || hint == 2 || hint == 4 || hint == 8) split = hint;
        M->crs_v = vector_lanes(st.max_row_len);
        if (cap > 0 && hint >= 0) {
            M->crs_rows_split = split;
            M->crs_rows_cap = cap;
        }
    } else {
        // uneven rows: the entry-split product (same work per thread whatever
        // the row lengths); its tile lines are computed once, here
        BufPtr tl;
        CKS(alloc_buf(spmv_seg_scratch_bytes(A->nnz), s, &tl));
        if (A->nnz > 0) CK(launch_spmv_seg_lines(A->irp, A->n_rows, A->nnz, reinterpret_cast<int32_t *>(tl->p), s));
        M->crs_seg = 1;
        M->seg_tl = reinterpret_cast<const int32_t *>(tl->p);
        M->bufs.push_back(tl);
    }
    *out = M.release();
    return SPMV_OK;
}

spmv_status build_coo_row(const spmv_crs *A, uint64_t cap, spmv_matrix **out, cudaStream_t s) {
    const uint64_t need = (uint64_t)A->nnz * 4;
    if (cap && need > cap) return SPMV_ERR_MEMORY_CAP;
    std::unique_ptr<spmv_matrix> M(new_handle(A, SPMV_COO, SPMV_ROWWISE, s));
    if (!M) return SPMV_ERR_OOM;
    BufPtr irow, acc_buf;
    CKS(alloc_buf(need, s, &irow));
    // IRP checks (the transformation reads no column index), read at the sync below
    CKS(alloc_buf(sizeof(AnalyzeAcc), s, &acc_buf));
    CK(cudaMemsetAsync(acc_buf->p, 0, sizeof(AnalyzeAcc), s));
    CK(launch_row_width(A->irp, A->n_rows, A->nnz, reinterpret_cast<AnalyzeAcc *>(acc_buf->p), s));
    CK(launch_expand(A->irp, A->n_rows, A->nnz, reinterpret_cast<int32_t *>(irow->p), s, "crs_to_coo_row"));
    BufPtr sw;
    CKS(alloc_buf(16, s, &sw));
    CK(cudaMemsetAsync(sw->p, 0, 16, s));
    M->status = reinterpret_cast<int *>(sw->p);
    M->bufs.push_back(sw);
    int hirp = 0;
    CK(cudaMemcpyAsync(&hirp, &reinterpret_cast<AnalyzeAcc *>(acc_buf->p)->status, sizeof(int),
                       cudaMemcpyDeviceToHost, s));
    if (A->nnz <= 0) {
        CK(cudaStreamSynchronize(s));
        CKS(status_from_dev(hirp));
    }
    // SpMV schedule: row-aligned tiles when the largest tile fits shared memory
    if (A->nnz > 0) {
        const int64_t tiles = ((int64_t)A->n_rows + 127) / 128;
        BufPtr tb;
        CKS(alloc_buf((size_t)(tiles + 1) * 4, s, &tb));
        int32_t *maxn = reinterpret_cast<int32_t *>(sw->p) + 1;  // second word of the status block
        CK(launch_line_tile_bounds(A->irp, A->n_rows, A->nnz, reinterpret_cast<int32_t *>(tb->p), maxn,
                                   "coo_row_tile_bounds", s));
        int h[2] = {0, 0};
        CK(cudaMemcpyAsync(h, sw->p, sizeof(h), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        CKS(status_from_dev(hirp));
        const int cap = coo_rows_cap(h[1]);
        if (cap > 0 && hint_value(SPMV_HINT_COO_FLAT) != 1) {
            M->coo_rows_cap = cap;
            M->coo_rows_split = ((double)A->nnz / A->n_rows <= 8.0) ? 2 : 4;
            M->coo_tb = reinterpret_cast<const int32_t *>(tb->p);
            M->bufs.push_back(tb);
        } else {
            M->coo_seg = 1;  // tiles too large for shared memory: entry-split product
        }
    }
    M->ptr = A->irp;
    M->idx = A->icol;
    M->idx2 = reinterpret_cast<const int32_t *>(irow->p);
    M->val = A->val;
    M->bufs.push_back(irow);
    *out = M.release();
    return SPMV_OK;
}

// CRS -> ELL-Row (optionally fused with y = A x). `st` from analyze_core.
spmv_status build_ell_row(const spmv_crs *A, const spmv_stats &st, uint64_t cap, const double *x, double *y,
                          spmv_matrix **out, cudaStream_t s) {
    const int32_t W = st.max_row_len;
    const int32_t ld = round_up32(A->n_rows);
    const uint64_t need = ell_bytes(A->n_rows, W);
    if (cap && need > cap) return SPMV_ERR_MEMORY_CAP;
    std::unique_ptr<spmv_matrix> M(new_handle(A, SPMV_ELL, SPMV_ROWWISE, s));
    if (!M) return SPMV_ERR_OOM;
    BufPtr ev, ei, stw;
    CKS(alloc_buf((size_t)ld * W * 8, s, &ev));
    CKS(alloc_buf((size_t)ld * W * 4, s, &ei));
    CKS(alloc_buf(16, s, &stw));
    CK(cudaMemsetAsync(stw->p, 0, 16, s));
    if (W == 0 && y) CK(cudaMemsetAsync(y, 0, sizeof(double) * (size_t)A->n_rows, s));
    CK(launch_lines_to_ell(A->irp, A->icol, A->val, A->n_rows, A->n_cols, W, ld,
                           reinterpret_cast<double *>(ev->p), reinterpret_cast<int32_t *>(ei->p), x, y,
                           reinterpret_cast<int *>(stw->p), s, "crs_to_ell_row"));
    int hst = 0;
    CK(cudaMemcpyAsync(&hst, stw->p, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    CKS(status_from_dev(hst));
    M->width = W;
    M->ld = ld;
    M->idx = reinterpret_cast<const int32_t *>(ei->p);
    M->val = reinterpret_cast<const double *>(ev->p);
    M->bufs.push_back(ev);
    M->bufs.push_back(ei);
    *out = M.release();
    return SPMV_OK;
}

// Phase I (CRS -> CCS). On success M holds the CCS in ccs_bufs/bufs.
// Three ways to the same CCS, bit for bit:
//   GRP   : slots carry (row, value) in regions of 64-column groups written
//           as coalesced runs per CTA, one atomic per (CTA, group); groups of
//           at most 2048 entries. For scattered columns.
//   RK    : slots carry (k, row), no per-entry ranks, a register sort per
//           column, VAL gathered by k. For neighbouring columns. Needs
//           >= 8 entries per column on average, no repeated (i, j), columns of
//           at most col_rv_long_cap() entries and few entries beyond the slots;
//           the kernels report ST_REDO when one of these fails.
//   KSLOT : slots carry (k, row); any matrix with >= 8 entries per column.
//   COUNT : count, scan, scatter of (k, row); any matrix.
enum class P1 { GRP, RK, KSLOT, COUNT };
constexpr int kLocalitySamples = 4096;
constexpr int kSymSamples = 4096;
constexpr spmv_status kRedo = (spmv_status)-1;  // internal: rerun on KSLOT

// The grouped row-value path: claim, scan of the group counts, fix-up (which
// also writes IRP_T and finds the longest column), long columns.
spmv_status phase1_grp(const spmv_crs *A, uint64_t cap_ell_col, bool want_ell, std::unique_ptr<spmv_matrix> &M,
                       cudaStream_t s, const int *irp_status) {
    const int64_t nnz = A->nnz;
    const int32_t nc = A->n_cols;
    const long long ng = col_grp_count(nc);
    BufPtr cp, trow, tval, gcnt, regions, scan_scr, words, longl, sct;
    CKS(alloc_buf((size_t)(ng + 1) * 4, s, &gcnt));
    CKS(alloc_buf(col_grp_region_bytes(nc), s, &regions));
    CKS(alloc_buf(scan_scratch_bytes(ng), s, &scan_scr));
    CKS(alloc_buf(col_grp_scratch_bytes(nnz), s, &sct));
    CKS(alloc_buf(64, s, &words));  // [0] status [1] colmax
    const int64_t max_long = std::min<int64_t>(nc, nnz / 33 + 1);
    CKS(alloc_buf((size_t)(max_long + 1) * 4, s, &longl));  // [0] count, then the list
    int32_t *d_g = reinterpret_cast<int32_t *>(gcnt->p);
    int *d_status = reinterpret_cast<int *>(words->p);
    int32_t *d_colmax = reinterpret_cast<int32_t *>(words->p) + 1;
    int32_t *d_long = reinterpret_cast<int32_t *>(longl->p);
    CK(cudaMemsetAsync(d_g, 0, (size_t)(ng + 1) * 4, s));
    CK(cudaMemsetAsync(words->p, 0, 64, s));
    CK(cudaMemsetAsync(d_long, 0, 4, s));
    CK(launch_col_claim_grp(A->irp, A->n_rows, A->icol, A->val, nnz, nc, d_g, regions->p,
                            reinterpret_cast<int32_t *>(sct->p), d_status, s));
    CK(launch_scan(d_g, ng, scan_scr->p, nullptr, INT_MAX, nullptr, nullptr, d_status, kSpinLimit, 0, s));
    CKS(alloc_buf((size_t)(nc + 1) * 4, s, &cp));
    CKS(alloc_buf((size_t)nnz * 4, s, &trow));
    CKS(alloc_buf((size_t)nnz * 8, s, &tval));
    int32_t *d_cp = reinterpret_cast<int32_t *>(cp->p);
    CK(launch_col_fixup_grp(d_g, nc, regions->p, d_cp, reinterpret_cast<int32_t *>(trow->p),
                            reinterpret_cast<double *>(tval->p), d_colmax, d_long + 1, d_status, s));
    int hw[2] = {0, 0};
    int hirp = 0;
    CK(cudaMemcpyAsync(hw, words->p, sizeof(hw), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&hirp, irp_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    CKS(status_from_dev(hirp));
    CKS(status_from_dev(hw[0]));
    if (hw[0] & ST_REDO) return kRedo;
    if (want_ell && cap_ell_col && ell_bytes(nc, hw[1]) > cap_ell_col) return SPMV_ERR_MEMORY_CAP;
    M->ptr = d_cp;
    M->idx = reinterpret_cast<const int32_t *>(trow->p);
    M->val = reinterpret_cast<const double *>(tval->p);
    M->ccs_bufs = {cp, trow, tval};
    M->colmax = hw[1];
    return SPMV_OK;
}

// The structurally symmetric path (square matrices whose pattern equals its
// transpose's, rows strictly ascending): IRP_T = IRP, ICOL_T = ICOL, VAL_T by
// mirror gathers, one kernel. kRedo when the kernel finds the conditions
// broken (the general paths then run).
spmv_status phase1_sym(const spmv_crs *A, uint64_t cap_ell_col, bool want_ell, std::unique_ptr<spmv_matrix> &M,
                       cudaStream_t s, const int *irp_status) {
    const int64_t nnz = A->nnz;
    const int32_t n = A->n_rows;
    BufPtr cp, trow, tval, words, sct;
    CKS(alloc_buf((size_t)(n + 1) * 4, s, &cp));
    CKS(alloc_buf((size_t)nnz * 4, s, &trow));
    CKS(alloc_buf((size_t)nnz * 8, s, &tval));
    CKS(alloc_buf(64, s, &words));  // [0] status, [1..3] u64: (unused, unused, longest row)
    CKS(alloc_buf(ccs_sym_scratch_bytes(nnz), s, &sct));
    CK(cudaMemsetAsync(words->p, 0, 64, s));
    CK(cudaMemcpyAsync(cp->p, A->irp, (size_t)(n + 1) * 4, cudaMemcpyDeviceToDevice, s));
    int *d_status = reinterpret_cast<int *>(words->p);
    unsigned long long *d_cnt = reinterpret_cast<unsigned long long *>(words->p) + 1;
    CK(launch_ccs_sym(A->irp, n, A->icol, A->val, nnz, reinterpret_cast<int32_t *>(sct->p),
                      reinterpret_cast<int32_t *>(trow->p), reinterpret_cast<double *>(tval->p), d_cnt, d_status, s));
    unsigned long long hw[4] = {0, 0, 0, 0};
    int hirp = 0;
    CK(cudaMemcpyAsync(hw, words->p, sizeof(hw), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&hirp, irp_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    CKS(status_from_dev(hirp));
    const int dst = (int)(hw[0] & 0xffffffffu);
    CKS(status_from_dev(dst));
    if (dst & ST_REDO) return kRedo;  // not symmetric, or a row out of order
    const int32_t colmax = (int32_t)hw[3];
    if (want_ell && cap_ell_col && ell_bytes(A->n_cols, colmax) > cap_ell_col) return SPMV_ERR_MEMORY_CAP;
    M->ptr = reinterpret_cast<const int32_t *>(cp->p);
    M->idx = reinterpret_cast<const int32_t *>(trow->p);
    M->val = reinterpret_cast<const double *>(tval->p);
    M->ccs_bufs = {cp, trow, tval};
    M->colmax = colmax;
    return SPMV_OK;
}

spmv_status phase1_try(const spmv_crs *A, uint64_t cap_ell_col, bool want_ell, P1 mode,
                       std::unique_ptr<spmv_matrix> &M, cudaStream_t s, const int *irp_status) {
    const int64_t nnz = A->nnz;
    const int32_t nc = A->n_cols;
    if (mode == P1::GRP) return phase1_grp(A, cap_ell_col, want_ell, M, s, irp_status);
    const bool rk = mode == P1::RK, slots = mode != P1::COUNT;
    BufPtr cp, trow, tval, rank, pairs, scan_scr, words, longl, tslots, sct0, ovl;
    CKS(alloc_buf((size_t)(nc + 1) * 4, s, &cp));
    if (!rk) CKS(alloc_buf((size_t)nnz * 4, s, &rank));
    CKS(alloc_buf(scan_scratch_bytes(nc), s, &scan_scr));
    CKS(alloc_buf(64, s, &words));  // [0] status [1] colmax [2] entries beyond the slots
    const int64_t max_long = std::min<int64_t>(nc, nnz / 33 + 1);
    CKS(alloc_buf((size_t)(max_long + 1) * 4, s, &longl));  // [0] count, then the list
    int32_t *d_cp = reinterpret_cast<int32_t *>(cp->p);
    int *d_status = reinterpret_cast<int *>(words->p);
    int32_t *d_colmax = reinterpret_cast<int32_t *>(words->p) + 1;
    int32_t *d_over = reinterpret_cast<int32_t *>(words->p) + 2;
    int32_t *d_long = reinterpret_cast<int32_t *>(longl->p);
    CK(cudaMemsetAsync(d_cp, 0, (size_t)(nc + 1) * 4, s));
    CK(cudaMemsetAsync(words->p, 0, 64, s));
    CK(cudaMemsetAsync(d_long, 0, 4, s));
    const int64_t ov_cap = nnz / 8 + 1024;
    if (rk) {
        CKS(alloc_buf(col_rk_slot_bytes(nc), s, &tslots));
        CKS(alloc_buf((size_t)ov_cap * sizeof(int4), s, &ovl));
        CK(launch_col_claim_rk(A->irp, A->n_rows, A->icol, nnz, nc, d_cp, tslots->p,
                               reinterpret_cast<int4 *>(ovl->p), ov_cap, d_over, nullptr, d_status, s));
    } else if (slots) {
        CKS(alloc_buf(col_slot_bytes(nc), s, &tslots));
        CKS(alloc_buf(col_scatter_scratch_bytes(nnz), s, &sct0));
        CK(launch_col_claim(A->irp, A->n_rows, A->icol, nnz, nc, d_cp, reinterpret_cast<int32_t *>(rank->p),
                            reinterpret_cast<int2 *>(tslots->p), d_over, reinterpret_cast<int32_t *>(sct0->p),
                            d_status, s));
    } else {
        CK(launch_col_count(A->icol, nnz, nc, d_cp, reinterpret_cast<int32_t *>(rank->p), d_status, s));
    }
    CK(launch_scan(d_cp, nc, scan_scr->p, d_colmax, 32, d_long + 1, d_long, d_status, kSpinLimit, 0, s));
    int hw[2] = {0, 0};
    int hirp = 0;
    if (want_ell) {
        // the ELL-Column width decides the cap check before anything else is built
        CK(cudaMemcpyAsync(hw, words->p, sizeof(hw), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(&hirp, irp_status, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        CKS(status_from_dev(hirp));
        CKS(status_from_dev(hw[0]));
        if (cap_ell_col && ell_bytes(nc, hw[1]) > cap_ell_col) return SPMV_ERR_MEMORY_CAP;
        if (hw[0] & ST_REDO) return kRedo;
    }
    CKS(alloc_buf((size_t)nnz * 4, s, &trow));
    CKS(alloc_buf((size_t)nnz * 8, s, &tval));
    if (rk) {
        CK(launch_col_fixup_rk(d_cp, nc, A->n_rows, A->val, tslots->p, reinterpret_cast<const int4 *>(ovl->p),
                               ov_cap,
                               d_over, d_long + 1, reinterpret_cast<int32_t *>(trow->p),
                               reinterpret_cast<double *>(tval->p), d_status, s));
    } else {
        CKS(alloc_buf((size_t)nnz * 8 + 16, s, &pairs));  // slack: staged copies round the end up
        if (slots) {
            // entries beyond the slot capacity (long columns) go to the pairs
            // array at IRP_T[col] + rank; the grid exits at once when there are none
            CK(launch_col_scatter(A->irp, A->n_rows, A->icol, nnz, nc, d_cp, reinterpret_cast<int32_t *>(rank->p),
                                  reinterpret_cast<int2 *>(pairs->p), reinterpret_cast<int32_t *>(sct0->p), d_status,
                                  s, col_slot_cap(), d_over, true));
            CK(launch_col_fixup_slots(d_cp, nc, A->irp, A->n_rows, A->val,
                                      reinterpret_cast<const int2 *>(tslots->p), reinterpret_cast<int2 *>(pairs->p),
                                      d_long + 1, reinterpret_cast<int32_t *>(rank->p),
                                      reinterpret_cast<int32_t *>(trow->p), reinterpret_cast<double *>(tval->p), s));
        } else {
            BufPtr sct;
            CKS(alloc_buf(col_scatter_scratch_bytes(nnz), s, &sct));
            CK(launch_col_scatter(A->irp, A->n_rows, A->icol, nnz, nc, d_cp, reinterpret_cast<int32_t *>(rank->p),
                                  reinterpret_cast<int2 *>(pairs->p), reinterpret_cast<int32_t *>(sct->p), d_status,
                                  s));
            CK(launch_col_fixup(d_cp, nc, A->irp, A->n_rows, A->val, reinterpret_cast<int2 *>(pairs->p), d_long + 1,
                                reinterpret_cast<int32_t *>(rank->p), reinterpret_cast<int32_t *>(trow->p),
                                reinterpret_cast<double *>(tval->p), d_status, s));
        }
    }
    CK(cudaMemcpyAsync(hw, words->p, sizeof(hw), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&hirp, irp_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    CKS(status_from_dev(hirp));
    CKS(status_from_dev(hw[0]));
    if (hw[0] & ST_REDO) return kRedo;
    const int32_t colmax = hw[1];
    M->ptr = d_cp;
    M->idx = reinterpret_cast<const int32_t *>(trow->p);
    M->val = reinterpret_cast<const double *>(tval->p);
    M->ccs_bufs = {cp, trow, tval};
    M->colmax = colmax;
    return SPMV_OK;
}

// `cap_ell_col`: when want_ell, fail with MEMORY_CAP before building the CCS
// if an ELL-Column of the longest column would exceed it (checked after the count).
spmv_status phase1(const spmv_crs *A, uint64_t cap_ccs, uint64_t cap_ell_col, bool want_ell,
                   std::unique_ptr<spmv_matrix> &M, cudaStream_t s, const int *irp_status) {
    const int64_t nnz = A->nnz;
    const int32_t nc = A->n_cols;
    const uint64_t own = (uint64_t)(nc + 1) * 4 + (uint64_t)nnz * 12;
    if (!want_ell && cap_ccs && own > cap_ccs) return SPMV_ERR_MEMORY_CAP;
    // The slot paths need >= 8 entries per column on average (slot array at
    // most 4x the pairs array); SPMV_HINT_PHASE1 forces a path (tests and
    // measurements).
    const int force = hint_value(SPMV_HINT_PHASE1);
    // A square matrix whose sampled entries all have their mirror (and rows
    // in ascending order) first tries the structurally symmetric path.
    if (A->n_rows == A->n_cols && nnz > 0 && (force == 0 || force == SPMV_PHASE1_SYMMETRIC)) {
        bool try_sym = force == SPMV_PHASE1_SYMMETRIC;
        if (!try_sym) {
            BufPtr fw;
            CKS(alloc_buf(16, s, &fw));
            CK(cudaMemsetAsync(fw->p, 0, 16, s));
            CK(launch_sym_sample(A->irp, A->n_rows, A->icol, nnz, kSymSamples, reinterpret_cast<int32_t *>(fw->p),
                                 s));
            int32_t hf = 0;
            CK(cudaMemcpyAsync(&hf, fw->p, sizeof(hf), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            try_sym = hf == 0;
        }
        if (try_sym) {
            spmv_status st = phase1_sym(A, cap_ell_col, want_ell, M, s, irp_status);
            if (st != kRedo) return st;
        }
    }
    const bool dense_cols = (int64_t)col_slot_cap() * nc <= 4 * nnz && nnz > 0;
    // the register-sort fix-ups (row-position and grouped paths) pack
    // (row << 5 | slot) into 32 bits
    const bool key_ok = A->n_rows < (1 << 27) - 1;
    P1 mode = dense_cols ? (key_ok ? P1::RK : P1::KSLOT) : P1::COUNT;
    if (mode == P1::RK && !force) {
        // Where a row's neighbouring entries have neighbouring columns (banded
        // and stencil matrices), the per-column slots of the row-position path
        // receive their stores in shared sectors and its VAL gathers stay
        // local; where columns are scattered, the grouped path's compact group
        // regions and coalesced runs win (measured: 27-point stencil 0.74 vs
        // 1.16 ms, power law with random columns 3.29 (row-value slots) vs
        // 2.73 ms). A sample of 4096 neighbouring pairs decides.
        BufPtr lw;
        CKS(alloc_buf(16, s, &lw));
        CK(cudaMemsetAsync(lw->p, 0, 16, s));
        CK(launch_col_locality(A->icol, nnz, kLocalitySamples, reinterpret_cast<int32_t *>(lw->p), s));
        int32_t hl = 0;
        CK(cudaMemcpyAsync(&hl, lw->p, sizeof(hl), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (hl < kLocalitySamples / 4) mode = P1::GRP;
    }
    if (force == SPMV_PHASE1_COUNT) mode = P1::COUNT;
    if (force == SPMV_PHASE1_KSLOT && nnz > 0) mode = P1::KSLOT;
    if (force == SPMV_PHASE1_ROWPOS && nnz > 0 && key_ok) mode = P1::RK;
    if (force == SPMV_PHASE1_GROUPED && nnz > 0 && key_ok) mode = P1::GRP;
    spmv_status st = phase1_try(A, cap_ell_col, want_ell, mode, M, s, irp_status);
    if (st == kRedo) st = phase1_try(A, cap_ell_col, want_ell, P1::KSLOT, M, s, irp_status);
    return st;
}

spmv_status ell_col_from_ccs(const spmv_matrix *src, uint64_t cap, spmv_matrix **out, cudaStream_t s) {
    const int32_t W = src->colmax;
    const int32_t ld = round_up32(src->n_cols);
    if (cap && ell_bytes(src->n_cols, W) > cap) return SPMV_ERR_MEMORY_CAP;
    std::unique_ptr<spmv_matrix> M(new (std::nothrow) spmv_matrix());
    if (!M) return SPMV_ERR_OOM;
    M->format = SPMV_ELL;
    M->layout = SPMV_COLWISE;
    M->n_rows = src->n_rows;
    M->n_cols = src->n_cols;
    M->nnz = src->nnz;
    M->home = s;
    BufPtr ev, ei, stw;
    CKS(alloc_buf((size_t)ld * W * 8, s, &ev));
    CKS(alloc_buf((size_t)ld * W * 4, s, &ei));
    CKS(alloc_buf(16, s, &stw));
    CK(cudaMemsetAsync(stw->p, 0, 16, s));
    CK(launch_lines_to_ell(src->ptr, src->idx, src->val, src->n_cols, src->n_rows, W, ld,
                           reinterpret_cast<double *>(ev->p), reinterpret_cast<int32_t *>(ei->p), nullptr, nullptr,
                           reinterpret_cast<int *>(stw->p), s, "ccs_to_ell_col"));
    // The CCS indices were produced and checked by Phase I, so only a bounded
    // wait of the build can fail: it is reported by spmv_matrix_status.
    M->width = W;
    M->ld = ld;
    M->idx = reinterpret_cast<const int32_t *>(ei->p);
    M->val = reinterpret_cast<const double *>(ev->p);
    M->status = reinterpret_cast<int *>(stw->p);
    M->bufs = {ev, ei, stw};
    *out = M.release();
    return SPMV_OK;
}

spmv_status coo_col_from_ccs(const spmv_matrix *src, uint64_t cap, spmv_matrix **out, cudaStream_t s) {
    const uint64_t need = (uint64_t)src->nnz * 4;
    if (cap && need > cap) return SPMV_ERR_MEMORY_CAP;
    std::unique_ptr<spmv_matrix> M(new (std::nothrow) spmv_matrix());
    if (!M) return SPMV_ERR_OOM;
    M->format = SPMV_COO;
    M->layout = SPMV_COLWISE;
    M->n_rows = src->n_rows;
    M->n_cols = src->n_cols;
    M->nnz = src->nnz;
    M->home = s;
    BufPtr tcol;
    CKS(alloc_buf(need, s, &tcol));
    CK(launch_expand(src->ptr, src->n_cols, src->nnz, reinterpret_cast<int32_t *>(tcol->p), s, "ccs_to_coo_col"));
    M->ptr = src->ptr;
    M->idx = src->idx;
    M->idx2 = reinterpret_cast<const int32_t *>(tcol->p);
    M->val = src->val;
    M->ccs_bufs = src->ccs_bufs;
    M->colmax = src->colmax;
    M->bufs = src->ccs_bufs;
    M->bufs.push_back(tcol);
    // SpMV schedule: 128-column tiles when a tile of the longest columns fits
    // shared memory (bounded by the longest column, known here: no sync)
    const int tcap = coo_rows_cap((int)std::min<int64_t>((int64_t)128 * src->colmax, (int64_t)(INT_MAX / 32)));
    if (src->nnz > 0 && tcap > 0 && hint_value(SPMV_HINT_COO_FLAT) != 1) {
        const int64_t tiles = ((int64_t)src->n_cols + 127) / 128;
        BufPtr tb;
        CKS(alloc_buf((size_t)(tiles + 1) * 4, s, &tb));
        CK(launch_line_tile_bounds(src->ptr, src->n_cols, src->nnz, reinterpret_cast<int32_t *>(tb->p), nullptr,
                                   "coo_col_tile_bounds", s));
        M->coo_rows_cap = tcap;
        M->coo_rows_split = ((double)src->nnz / src->n_cols <= 8.0) ? 2 : 4;
        M->coo_tb = reinterpret_cast<const int32_t *>(tb->p);
        M->bufs.push_back(tb);
    }
    *out = M.release();
    return SPMV_OK;
}

spmv_status apply_core(const spmv_matrix *M, const double *x, double *y, cudaStream_t s) {
    if (M->layout == SPMV_ROWWISE) {
        switch (M->format) {
            case SPMV_CRS:
                if (M->crs_seg) {
                    CK(launch_spmv_seg(false, M->ptr, M->idx, M->val, M->nnz, M->n_rows, M->n_cols, M->seg_tl, x, y,
                                       s));
                } else if (M->crs_rows_split > 0) {
                    CK(launch_spmv_crs_rows(M->crs_rows_split, M->crs_rows_cap, M->ptr, M->idx, M->val, M->n_rows,
                                            x, y, s));
                } else if (M->n_rows > 0) {
                    CK(launch_spmv_crs_vector(M->crs_v, M->ptr, M->idx, M->val, nullptr, M->n_rows, x, y, s));
                }
                return SPMV_OK;
            case SPMV_COO: {
                if (M->coo_rows_split > 0) {
                    CK(launch_spmv_coo_row_rows(M->coo_rows_split, M->coo_rows_cap, M->idx2, M->idx, M->val, M->coo_tb,
                                                M->n_rows, M->n_cols, x, y, s));
                    return SPMV_OK;
                }
                if (M->coo_seg) {
                    CK(launch_spmv_seg(true, M->idx2, M->idx, M->val, M->nnz, M->n_rows, M->n_cols, nullptr, x, y, s));
                    return SPMV_OK;
                }
                // no entries: y = 0
                CK(cudaMemsetAsync(y, 0, sizeof(double) * (size_t)M->n_rows, s));
                return SPMV_OK;
            }
            case SPMV_ELL:
                if (M->width == 0) { CK(cudaMemsetAsync(y, 0, sizeof(double) * (size_t)M->n_rows, s)); return SPMV_OK; }
                CK(launch_spmv_ell_row(M->val, M->idx, M->n_rows, M->width, M->ld, x, y, s));
                return SPMV_OK;
        }
    } else {
        switch (M->format) {
            case SPMV_CRS:
                CK(launch_spmv_ccs(M->ptr, M->idx, M->val, M->n_rows, M->n_cols, x, y, s));
                return SPMV_OK;
            case SPMV_COO:
                if (M->coo_rows_split > 0) {
                    CK(launch_spmv_coo_col_cols(M->coo_rows_split, M->coo_rows_cap, M->idx, M->idx2, M->val,
                                                M->coo_tb, M->n_rows, M->n_cols, x, y, s));
                    return SPMV_OK;
                }
                CK(launch_spmv_coo_col(M->idx, M->idx2, M->val, M->nnz, M->n_rows, x, y, s));
                return SPMV_OK;
            case SPMV_ELL:
                CK(launch_spmv_ell_col(M->val, M->idx, M->n_rows, M->n_cols, M->width, M->ld, M->nnz, x, y, s));
                return SPMV_OK;
        }
    }
    return SPMV_ERR_INVALID_ARG;
}

double median(std::vector<float> v) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const size_t m = v.size() / 2;
    return (v.size() % 2) ? v[m] : 0.5 * ((double)v[m - 1] + v[m]);
}

// Median device time (ms) of fn() over reps after warm-up runs.
template <typename F>
spmv_status time_median(F fn, int warm, int reps, cudaStream_t s, double *ms) {
    for (int i = 0; i < warm; ++i) CKS(fn());
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return SPMV_ERR_CUDA; }
    std::vector<float> t;
    spmv_status st = SPMV_OK;
    for (int i = 0; i < reps && st == SPMV_OK; ++i) {
        cudaEventRecord(e0, s);
        st = fn();
        cudaEventRecord(e1, s);
        if (st == SPMV_OK) {
            if (cudaEventSynchronize(e1) != cudaSuccess) { cudaGetLastError(); st = SPMV_ERR_CUDA; break; }
            float f = 0.f;
            cudaEventElapsedTime(&f, e0, e1);
            t.push_back(f);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != SPMV_OK) return st;
    *ms = median(t);
    return SPMV_OK;
}

}  // namespace

// =================================================================== C ABI
extern "C" {

int32_t spmv_version(void) { return SPMVAT_VERSION; }

const char *spmv_status_string(spmv_status s) {
    switch (s) {
        case SPMV_OK: return "SPMV_OK";
        case SPMV_ERR_INVALID_ARG: return "SPMV_ERR_INVALID_ARG";
        case SPMV_ERR_INVALID_MATRIX: return "SPMV_ERR_INVALID_MATRIX";
        case SPMV_ERR_OOM: return "SPMV_ERR_OOM";
        case SPMV_ERR_MEMORY_CAP: return "SPMV_ERR_MEMORY_CAP";
        case SPMV_ERR_TIMEOUT: return "SPMV_ERR_TIMEOUT";
        case SPMV_ERR_CUDA: return "SPMV_ERR_CUDA";
        case SPMV_ERR_UNSUPPORTED: return "SPMV_ERR_UNSUPPORTED";
    }
    return "SPMV_ERR_UNKNOWN";
}

spmv_status spmv_set_allocator(spmv_alloc_fn alloc, spmv_free_fn free_fn, void *ctx) {
    if ((alloc == nullptr) != (free_fn == nullptr)) return SPMV_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    g_hooks.alloc = alloc;
    g_hooks.free = free_fn;
    g_hooks.ctx = alloc ? ctx : nullptr;
    return SPMV_OK;
}

spmv_status spmv_reserve(uint64_t bytes, spmv_stream_t stream) {
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (g_hooks.alloc) return SPMV_OK;  // the caller's allocator owns the memory
    }
    if (bytes == 0) return SPMV_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return SPMV_ERR_CUDA; }
    cudaMemPool_t pool = pool_for(dev);
    if (!pool) return SPMV_ERR_CUDA;
    cudaStream_t s = S(stream);
    void *p = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(&p, (size_t)bytes, pool, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? SPMV_ERR_OOM : SPMV_ERR_CUDA;
    }
    CK(cudaFreeAsync(p, s));
    CK(cudaStreamSynchronize(s));  // freed and complete: any stream may reuse it at once
    return SPMV_OK;
}

uint64_t spmv_ell_bytes(int32_t n_lines, int32_t width) {
    if (n_lines < 0 || width < 0) return 0;
    return ell_bytes(n_lines, width);
}

spmv_status spmv_analyze(const spmv_crs *A, spmv_stats *out, spmv_stream_t stream) {
    CKS(check_crs(A));
    if (!out) return SPMV_ERR_INVALID_ARG;
    return analyze_core(A, false, out, S(stream));
}

spmv_status spmv_validate(const spmv_crs *A, spmv_stream_t stream) {
    CKS(check_crs(A));
    spmv_stats st;
    return analyze_core(A, true, &st, S(stream));
}

spmv_status spmv_transform(const spmv_crs *A, spmv_format format, spmv_layout layout, uint64_t mem_cap_bytes,
                           spmv_matrix **out, spmv_stream_t stream) {
    if (!out) return SPMV_ERR_INVALID_ARG;
    *out = nullptr;
    CKS(check_crs(A));
    if ((int)format < SPMV_CRS || (int)format > SPMV_ELL) return SPMV_ERR_INVALID_ARG;
    if ((int)layout != SPMV_ROWWISE && (int)layout != SPMV_COLWISE) return SPMV_ERR_INVALID_ARG;
    cudaStream_t s = S(stream);
    if (layout == SPMV_ROWWISE) {
        if (format == SPMV_CRS) return build_crs_plan(A, mem_cap_bytes, out, s);
        if (format == SPMV_COO) return build_coo_row(A, mem_cap_bytes, out, s);
        spmv_stats st;
        CKS(analyze_width(A, &st, s));
        return build_ell_row(A, st, mem_cap_bytes, nullptr, nullptr, out, s);
    }
    // column-wise: Phase I first
    std::unique_ptr<spmv_matrix> M(new_handle(A, SPMV_CRS, SPMV_COLWISE, s));
    if (!M) return SPMV_ERR_OOM;
    // IRP checks run ahead of Phase I; their result is read with Phase I's own
    // status at its final synchronisation (Phase I kernels stay in bounds on
    // any IRP).
    BufPtr acc_buf;
    CKS(alloc_buf(sizeof(AnalyzeAcc), s, &acc_buf));
    CK(cudaMemsetAsync(acc_buf->p, 0, sizeof(AnalyzeAcc), s));
    CK(launch_row_width(A->irp, A->n_rows, A->nnz, reinterpret_cast<AnalyzeAcc *>(acc_buf->p), s));
    const int *irp_status = &reinterpret_cast<AnalyzeAcc *>(acc_buf->p)->status;
    CKS(phase1(A, format == SPMV_CRS ? mem_cap_bytes : 0, mem_cap_bytes, format == SPMV_ELL, M, s, irp_status));
    M->bufs = M->ccs_bufs;
    if (format == SPMV_CRS) {
        *out = M.release();
        return SPMV_OK;
    }
    if (format == SPMV_COO) return coo_col_from_ccs(M.get(), mem_cap_bytes, out, s);
    return ell_col_from_ccs(M.get(), mem_cap_bytes, out, s);
}

spmv_status spmv_transform_from(const spmv_matrix *src, spmv_format format, uint64_t mem_cap_bytes,
                                spmv_matrix **out, spmv_stream_t stream) {
    if (!out) return SPMV_ERR_INVALID_ARG;
    *out = nullptr;
    if (!src || src->layout != SPMV_COLWISE || src->ccs_bufs.empty()) return SPMV_ERR_INVALID_ARG;
    if (format == SPMV_COO) return coo_col_from_ccs(src, mem_cap_bytes, out, S(stream));
    if (format == SPMV_ELL) return ell_col_from_ccs(src, mem_cap_bytes, out, S(stream));
    return SPMV_ERR_INVALID_ARG;
}

spmv_status spmv_apply(const spmv_matrix *M, const double *x, double *y, spmv_stream_t stream) {
    if (!M || !x || !y) return SPMV_ERR_INVALID_ARG;
    return apply_core(M, x, y, S(stream));
}

spmv_status spmv_transform_apply(const spmv_crs *A, const double *x, double *y, uint64_t mem_cap_bytes,
                                 spmv_matrix **out, spmv_stream_t stream) {
    if (!out) return SPMV_ERR_INVALID_ARG;
    *out = nullptr;
    CKS(check_crs(A));
    if (!x || !y) return SPMV_ERR_INVALID_ARG;
    spmv_stats st;
    CKS(analyze_width(A, &st, S(stream)));
    return build_ell_row(A, st, mem_cap_bytes, x, y, out, S(stream));
}

spmv_status spmv_describe(const spmv_matrix *M, spmv_matrix_desc *out) {
    if (!M || !out) return SPMV_ERR_INVALID_ARG;
    memset(out, 0, sizeof(*out));
    out->format = M->format;
    out->layout = M->layout;
    out->n_rows = M->n_rows;
    out->n_cols = M->n_cols;
    out->nnz = M->nnz;
    out->width = M->width;
    out->ld = M->ld;
    out->ptr = M->ptr;
    out->idx = M->idx;
    out->idx2 = M->idx2;
    out->val = M->val;
    out->owned_bytes = M->owned();
    return SPMV_OK;
}

void spmv_destroy(spmv_matrix *M) { delete M; }

double spmv_r_ell(double t_crs, double t_ell, double t_trans) {
    const double sp = t_crs / t_ell;   // Eq. (1)
    const double tt = t_trans / t_crs; // Eq. (2), transformation in CRS-SpMV units
    return sp / tt;                    // Eq. (3)
}

spmv_status spmv_dstar_from_points(int32_t m, const double *dmat, const double *rell, double c, int32_t rule,
                                   double *dstar) {
    if (m < 0 || !dstar || (m > 0 && (!dmat || !rell))) return SPMV_ERR_INVALID_ARG;
    if (rule == SPMV_DSTAR_MAXPASS) {
        double best = 0.0;
        for (int32_t i = 0; i < m; ++i)
            if (rell[i] >= c && dmat[i] > best) best = dmat[i];
        *dstar = best;
        return SPMV_OK;
    }
    if (rule != SPMV_DSTAR_PREFIX) return SPMV_ERR_INVALID_ARG;
    std::vector<int32_t> ord(m);
    for (int32_t i = 0; i < m; ++i) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) { return dmat[a] < dmat[b]; });
    double d = INFINITY;
    for (int32_t t = 0; t < m; ++t) {
        if (rell[ord[t]] < c) {
            d = (t == 0) ? 0.0 : dmat[ord[t]];
            break;
        }
    }
    *dstar = d;
    return SPMV_OK;
}

spmv_status spmv_measure(const spmv_crs *A, const spmv_at_params *p, spmv_timing *out, spmv_stream_t stream) {
    CKS(check_crs(A));
    if (!p || !out) return SPMV_ERR_INVALID_ARG;
    cudaStream_t s = S(stream);
    const int reps = p->timing_reps > 0 ? p->timing_reps : 20;
    const int warm = p->warmup_reps >= 0 ? p->warmup_reps : 3;
    memset(out, 0, sizeof(*out));
    spmv_stats st;
    CKS(analyze_core(A, false, &st, s));
    out->dmat = st.dmat;
    if (p->mem_cap_bytes && st.ell_bytes > p->mem_cap_bytes) return SPMV_ERR_MEMORY_CAP;
    BufPtr xb, yb;
    CKS(alloc_buf(sizeof(double) * (size_t)A->n_cols, s, &xb));
    CKS(alloc_buf(sizeof(double) * (size_t)A->n_rows, s, &yb));
    CK(cudaMemsetAsync(xb->p, 0, sizeof(double) * (size_t)A->n_cols, s));
    const double *x = reinterpret_cast<const double *>(xb->p);
    double *y = reinterpret_cast<double *>(yb->p);
    spmv_matrix *crs = nullptr;
    CKS(build_crs_plan(A, 0, &crs, s));
    std::unique_ptr<spmv_matrix> crs_h(crs);
    CKS(time_median([&] { return apply_core(crs, x, y, s); }, warm, reps, s, &out->t_crs_ms));
    // t_trans: device work of CRS -> ELL-Row (the row-pointer pass + the ELL
    // build, as spmv_transform runs them) into preallocated arrays;
    // allocation is not timed.
    const int32_t W = st.max_row_len, ld = round_up32(A->n_rows);
    BufPtr ev, ei, acc, stw;
    CKS(alloc_buf((size_t)ld * W * 8, s, &ev));
    CKS(alloc_buf((size_t)ld * W * 4, s, &ei));
    CKS(alloc_buf(sizeof(AnalyzeAcc), s, &acc));
    CKS(alloc_buf(16, s, &stw));
    CK(cudaMemsetAsync(stw->p, 0, 16, s));
    auto trans = [&]() -> spmv_status {
        CK(cudaMemsetAsync(acc->p, 0, sizeof(AnalyzeAcc), s));
        CK(launch_row_width(A->irp, A->n_rows, A->nnz, reinterpret_cast<AnalyzeAcc *>(acc->p), s));
        CK(launch_lines_to_ell(A->irp, A->icol, A->val, A->n_rows, A->n_cols, W, ld,
                               reinterpret_cast<double *>(ev->p), reinterpret_cast<int32_t *>(ei->p), nullptr,
                               nullptr, reinterpret_cast<int *>(stw->p), s, "crs_to_ell_row"));
        return SPMV_OK;
    };
    CKS(time_median(trans, warm, reps, s, &out->t_trans_ms));
    spmv_matrix ell;
    ell.format = SPMV_ELL;
    ell.layout = SPMV_ROWWISE;
    ell.n_rows = A->n_rows;
    ell.n_cols = A->n_cols;
    ell.nnz = A->nnz;
    ell.width = W;
    ell.ld = ld;
    ell.idx = reinterpret_cast<const int32_t *>(ei->p);
    ell.val = reinterpret_cast<const double *>(ev->p);
    CKS(time_median([&] { return apply_core(&ell, x, y, s); }, warm, reps, s, &out->t_ell_ms));
    if (p->flags & SPMV_AT_TRY_COO) {
        spmv_matrix *coo = nullptr;
        CKS(build_coo_row(A, 0, &coo, s));
        std::unique_ptr<spmv_matrix> coo_h(coo);
        CKS(time_median([&] { return apply_core(coo, x, y, s); }, warm, reps, s, &out->t_coo_ms));
    }
    int hst = 0;
    CK(cudaMemcpyAsync(&hst, stw->p, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    CKS(status_from_dev(hst));
    out->sp = out->t_crs_ms / out->t_ell_ms;
    out->tt = out->t_trans_ms / out->t_crs_ms;
    out->r_ell = spmv_r_ell(out->t_crs_ms, out->t_ell_ms, out->t_trans_ms);
    return SPMV_OK;
}

spmv_status spmv_measure_atomics(int64_t n_targets, int64_t n_adds, int32_t reps, double *ms, spmv_stream_t stream) {
    if (n_targets <= 0 || n_adds <= 0 || reps <= 0 || !ms) return SPMV_ERR_INVALID_ARG;
    cudaStream_t s = S(stream);
    BufPtr yb;
    CKS(alloc_buf(sizeof(double) * (size_t)n_targets, s, &yb));
    double *y = reinterpret_cast<double *>(yb->p);
    CK(cudaMemsetAsync(y, 0, sizeof(double) * (size_t)n_targets, s));
    return time_median([&]() -> spmv_status {
        CK(launch_atomic_ceiling(y, n_targets, n_adds, s));
        return SPMV_OK;
    }, 3, reps, s, ms);
}

spmv_status spmv_calibrate(const spmv_crs *const *set, int32_t m, const spmv_at_params *p, double *dmat_out,
                           double *rell_out, double *dstar_out, spmv_stream_t stream) {
    if (!set || m < 0 || !p || !dstar_out) return SPMV_ERR_INVALID_ARG;
    std::vector<double> d(m), r(m);
    for (int32_t i = 0; i < m; ++i) {
        spmv_timing t;
        spmv_status st = spmv_measure(set[i], p, &t, stream);
        if (st == SPMV_ERR_MEMORY_CAP) {
            spmv_stats ss;
            CKS(spmv_analyze(set[i], &ss, stream));
            d[i] = ss.dmat;
            r[i] = 0.0;
        } else if (st != SPMV_OK) {
            return st;
        } else {
            d[i] = t.dmat;
            r[i] = t.r_ell;
        }
        if (dmat_out) dmat_out[i] = d[i];
        if (rell_out) rell_out[i] = r[i];
    }
    return spmv_dstar_from_points(m, d.data(), r.data(), p->c, p->dstar_rule, dstar_out);
}

spmv_status spmv_autotune(const spmv_crs *A, const spmv_at_params *p, spmv_matrix **chosen, spmv_stats *stats,
                          spmv_stream_t stream) {
    if (!chosen || !p) return SPMV_ERR_INVALID_ARG;
    *chosen = nullptr;
    CKS(check_crs(A));
    cudaStream_t s = S(stream);
    spmv_stats st;
    CKS(analyze_core(A, false, &st, s));  // on-line step (1): D_mat
    if (stats) *stats = st;
    const bool fits = !p->mem_cap_bytes || st.ell_bytes <= p->mem_cap_bytes;
    if (st.dmat < p->dstar && fits) return build_ell_row(A, st, p->mem_cap_bytes, nullptr, nullptr, chosen, s);
    // CRS (or COO-Row): the statistics are known, only the indices need checking
    CKS(validate_icol(A, s));
    if (p->flags & SPMV_AT_TRY_COO) {
        spmv_matrix *crs = nullptr, *coo = nullptr;
        CKS(crs_plan_from(A, st, p->mem_cap_bytes, &crs, s));
        std::unique_ptr<spmv_matrix> crs_h(crs);
        spmv_status e = build_coo_row(A, p->mem_cap_bytes, &coo, s);
        if (e == SPMV_ERR_MEMORY_CAP) { *chosen = crs_h.release(); return SPMV_OK; }
        CKS(e);
        std::unique_ptr<spmv_matrix> coo_h(coo);
        BufPtr xb, yb;
        CKS(alloc_buf(sizeof(double) * (size_t)A->n_cols, s, &xb));
        CKS(alloc_buf(sizeof(double) * (size_t)A->n_rows, s, &yb));
        CK(cudaMemsetAsync(xb->p, 0, sizeof(double) * (size_t)A->n_cols, s));
        const double *x = reinterpret_cast<const double *>(xb->p);
        double *y = reinterpret_cast<double *>(yb->p);
        const int reps = p->timing_reps > 0 ? p->timing_reps : 20;
        const int warm = p->warmup_reps >= 0 ? p->warmup_reps : 3;
        double tc = 0, to = 0;
        CKS(time_median([&] { return apply_core(crs, x, y, s); }, warm, reps, s, &tc));
        CKS(time_median([&] { return apply_core(coo, x, y, s); }, warm, reps, s, &to));
        *chosen = (to < tc) ? coo_h.release() : crs_h.release();
        return SPMV_OK;
    }
    return crs_plan_from(A, st, p->mem_cap_bytes, chosen, s);
}

spmv_status spmv_autotune_choose(const spmv_crs *A, const spmv_at_params *p, int32_t *format, int32_t *layout,
                                 spmv_stats *stats, spmv_stream_t stream) {
    if (!p || !format || !layout) return SPMV_ERR_INVALID_ARG;
    CKS(check_crs(A));
    spmv_stats st;
    CKS(analyze_core(A, false, &st, S(stream)));
    if (stats) *stats = st;
    const bool fits = !p->mem_cap_bytes || st.ell_bytes <= p->mem_cap_bytes;
    *format = (st.dmat < p->dstar && fits) ? SPMV_ELL : SPMV_CRS;
    *layout = SPMV_ROWWISE;
    return SPMV_OK;
}

spmv_status spmv_matrix_status(const spmv_matrix *M, spmv_stream_t stream) {
    if (!M) return SPMV_ERR_INVALID_ARG;
    if (!M->status) return SPMV_OK;
    int h = 0;
    CK(cudaMemcpyAsync(&h, M->status, sizeof(int), cudaMemcpyDeviceToHost, S(stream)));
    CK(cudaStreamSynchronize(S(stream)));
    return status_from_dev(h);
}

uint64_t spmv_launch_count(void) { return g_launches.load(); }

spmv_status spmv_set_hint(int32_t hint, int32_t value) {
    if (hint < 0 || hint >= SPMV_HINT_COUNT) return SPMV_ERR_INVALID_ARG;
    g_hints[hint].store(value);
    return SPMV_OK;
}

int32_t spmv_get_hint(int32_t hint) { return hint_value(hint); }

spmv_status spmv_profile_enable(int32_t on) {
    g_profile_on.store(on ? 1 : 0);
    return SPMV_OK;
}

int32_t spmv_profile_read(spmv_kernel_time *out, int32_t cap, int32_t reset) {
    std::lock_guard<std::mutex> lk(g_pmu);
    for (auto &r : g_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.e1) == cudaSuccess && cudaEventElapsedTime(&ms, r.e0, r.e1) == cudaSuccess) {
            auto &t = g_totals[r.name];
            t.first += 1;
            t.second += ms;
        } else {
            cudaGetLastError();
        }
        g_event_pool.push_back(r.e0);
        g_event_pool.push_back(r.e1);
    }
    g_pending.clear();
    int32_t n = 0;
    for (auto &kv : g_totals) {
        if (out && n < cap) {
            memset(&out[n], 0, sizeof(out[n]));
            strncpy(out[n].name, kv.first.c_str(), sizeof(out[n].name) - 1);
            out[n].launches = kv.second.first;
            out[n].total_ms = kv.second.second;
        }
        ++n;
    }
    if (reset) g_totals.clear();
    return n;
}

spmv_status spmv_debug_scan_timeout(int32_t n, int32_t spin_limit, int32_t *observed, spmv_stream_t stream) {
    if (n <= 0 || spin_limit <= 0 || !observed) return SPMV_ERR_INVALID_ARG;
    cudaStream_t s = S(stream);
    BufPtr a, scr, words;
    CKS(alloc_buf((size_t)(n + 1) * 4, s, &a));
    CKS(alloc_buf(scan_scratch_bytes(n), s, &scr));
    CKS(alloc_buf(16, s, &words));
    CK(cudaMemsetAsync(a->p, 0, (size_t)(n + 1) * 4, s));
    CK(cudaMemsetAsync(words->p, 0, 16, s));
    CK(launch_scan(reinterpret_cast<int32_t *>(a->p), n, scr->p, nullptr, INT_MAX, nullptr, nullptr,
                   reinterpret_cast<int *>(words->p), spin_limit, 1, s));
    int hst = 0;
    CK(cudaMemcpyAsync(&hst, words->p, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *observed = (int32_t)status_from_dev(hst);
    return SPMV_OK;
}

}  // extern "C"
