// C ABI for batches of independent matrices (declared in include/spmvat.h):
// one analysis launch, the on-line rule of Sec. 2.2 per matrix, one ELL
// build launch and one SpMV launch for the whole batch.
#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"
#include "host_mem.h"
#include "spmvat.h"

using namespace spmvat;

struct spmv_batch {
    int32_t m = 0;
    int64_t total_rows = 0, total_cols = 0, total_nnz = 0;
    int64_t n_tiles = 0;
    int32_t n_ell = 0;
    uint64_t ell_bytes = 0;
    std::vector<BatchMat> host_mats;
    std::vector<spmv_batch_plan> plans;
    BufPtr mats, tiles, ell_pool;
    const BatchMat *d_mats = nullptr;
    const int4 *d_tiles = nullptr;
    // planned on the device (spmv_batch_prepare + spmv_batch_build)
    bool device_plan = false, built = false, fetched = false;
    double dstar = 0.0;
    uint64_t cap = 0;
    int64_t tile_cap = 0;            // tile records allocated (an upper bound of the count)
    long long n_chunks = 0;
    BufPtr chunks, acc, bytes, plan_out, counts, words;  // words: status, totals, tile count
    const long long *d_ntiles = nullptr;
    cudaStream_t home = nullptr;
    uint64_t owned() const {
        uint64_t t = 0;
        for (const BufPtr *b : {&mats, &tiles, &ell_pool, &chunks, &acc, &bytes, &plan_out, &counts, &words})
            if (*b) t += (*b)->bytes;
        return t;
    }
};

namespace {

inline cudaStream_t S(spmv_stream_t s) { return reinterpret_cast<cudaStream_t>(s); }
inline int32_t round_up32(int64_t n) { return (int32_t)((n + 31) / 32 * 32); }

// The batch schedule table (spmv_batch_schedule_set): lanes per row of a
// CRS member by the class of its mean row length mu = nnz / n (class 0: mu <
// 1; class c >= 1: mu in [2^(c-1), 2^c), the last class open-ended). The
// default: one lane per entry ("merge" tiles of whole rows) below a mean of
// 32 entries, 8 lanes per row below 256, a whole warp above.
constexpr int kSchedClasses = SPMV_BATCH_SCHED_CLASSES;
std::atomic<int> g_tpr[kSchedClasses] = {{1}, {1}, {1}, {1}, {1}, {1}, {8}, {8}, {8}, {32}};

int sched_class(double mu) {
    if (!(mu >= 1.0)) return 0;
    const int c = (int)std::floor(std::log2(mu)) + 1;
    return std::min(c, kSchedClasses - 1);
}

// Lanes per row of a CRS tile (the hint overrides the table).
int threads_per_row(double mu) {
    const int v = hint_value(SPMV_HINT_BATCH_TPR);
    if (v == 1 || v == 8 || v == 32) return v;
    return g_tpr[sched_class(mu)].load();
}

spmv_status check_one(const spmv_crs &A) {
    if (A.n_rows <= 0 || A.n_cols <= 0 || A.nnz < 0 || A.nnz >= (int64_t)INT_MAX) return SPMV_ERR_INVALID_ARG;
    if (!A.irp) return SPMV_ERR_INVALID_ARG;
    if (A.nnz > 0 && (!A.icol || !A.val)) return SPMV_ERR_INVALID_ARG;
    return SPMV_OK;
}

template <class V>
spmv_status upload(const std::vector<V> &h, cudaStream_t s, BufPtr *out) {
    CKS(alloc_buf(sizeof(V) * std::max<size_t>(h.size(), 1), s, out));
    if (!h.empty()) CK(cudaMemcpyAsync((*out)->p, h.data(), sizeof(V) * h.size(), cudaMemcpyHostToDevice, s));
    return SPMV_OK;
}

spmv_status create_core(const spmv_crs *mats, int32_t m, const spmv_at_params *p, const double *x, double *y,
                        spmv_batch *B, cudaStream_t s) {
    const double dstar = p ? p->dstar : 0.0;
    const uint64_t cap = (p && p->mem_cap_bytes) ? p->mem_cap_bytes : UINT64_MAX;
    B->m = m;
    B->host_mats.resize(m);
    B->plans.resize(m);
    std::vector<int2> chunks;
    for (int32_t i = 0; i < m; ++i) {
        const spmv_crs &A = mats[i];
        BatchMat &D = B->host_mats[i];
        memset(&D, 0, sizeof(D));
        D.irp = A.irp;
        D.icol = A.icol;
        D.val = A.val;
        D.xoff = B->total_cols;
        D.yoff = B->total_rows;
        D.nnz = A.nnz;
        D.n_rows = A.n_rows;
        D.n_cols = A.n_cols;
        B->total_cols += A.n_cols;
        B->total_rows += A.n_rows;
        B->total_nnz += A.nnz;
        for (int32_t r = 0; r < A.n_rows; r += kBatchChunk) chunks.push_back(make_int2(i, r));
    }
    // Analysis of every matrix (Eq. (4)) plus index checks, one launch.
    CKS(upload(B->host_mats, s, &B->mats));
    BufPtr chunk_buf, acc_buf;
    CKS(upload(chunks, s, &chunk_buf));
    CKS(alloc_buf(sizeof(BatchAcc) * (size_t)m, s, &acc_buf));
    CK(cudaMemsetAsync(acc_buf->p, 0, sizeof(BatchAcc) * (size_t)m, s));
    CK(launch_batch_analyze(reinterpret_cast<const BatchMat *>(B->mats->p),
                            reinterpret_cast<const int2 *>(chunk_buf->p), (long long)chunks.size(),
                            reinterpret_cast<BatchAcc *>(acc_buf->p), s));
    std::vector<BatchAcc> acc(m);
    CK(cudaMemcpyAsync(acc.data(), acc_buf->p, sizeof(BatchAcc) * (size_t)m, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));

    // On-line rule per matrix (Sec. 2.2): ELL-Row iff D_mat < D* and the
    // batch's ELL arrays stay within the cap (matrices taken in order).
    std::vector<uint64_t> ell_off(m, 0);
    for (int32_t i = 0; i < m; ++i) {
        const BatchAcc &a = acc[i];
        BatchMat &D = B->host_mats[i];
        spmv_batch_plan &P = B->plans[i];
        spmv_status st = status_from_dev(a.status);
        if (st != SPMV_OK) return st;
        if ((long long)a.sum_len != D.nnz) return SPMV_ERR_INVALID_MATRIX;
        const double n = (double)D.n_rows;
        const unsigned __int128 num = (unsigned __int128)(unsigned long long)D.n_rows * a.sum_len2 -
                                      (unsigned __int128)a.sum_len * a.sum_len;
        memset(&P, 0, sizeof(P));
        P.mu = (double)a.sum_len / n;
        P.sigma = std::sqrt((double)num) / n;
        P.dmat = a.sum_len == 0 ? 0.0 : P.sigma / P.mu;
        P.max_row_len = a.max_len;
        P.x_offset = D.xoff;
        P.y_offset = D.yoff;
        const uint64_t eb = (uint64_t)round_up32(D.n_rows) * (uint64_t)a.max_len * 12ull;
        if (P.dmat < dstar && B->ell_bytes + eb <= cap) {
            D.fmt = BATCH_ELL;
            D.width = a.max_len;
            D.ld = round_up32(D.n_rows);
            D.tpr = 1;
            D.rpt = 32;
            ell_off[i] = B->ell_bytes;
            B->ell_bytes += eb;
            B->n_ell += 1;
        } else {
            D.fmt = BATCH_CRS;
            D.tpr = threads_per_row((double)D.nnz / (double)D.n_rows);
            D.rpt = 32 / D.tpr;  // one lane per entry: at most 32 rows (and 256 entries) per tile
        }
        P.format = D.fmt == BATCH_ELL ? SPMV_ELL : SPMV_CRS;
        P.threads_per_row = D.tpr;
        P.rows_per_tile = D.rpt;
        P.width = D.width;
        P.ld = D.ld;
    }
    // ELL arrays of all ELL matrices in one allocation: per matrix the values
    // (8 * ld * W bytes, a multiple of 256) then the indices (4 * ld * W).
    if (B->n_ell > 0) {
        CKS(alloc_buf(B->ell_bytes, s, &B->ell_pool));
        unsigned char *base = reinterpret_cast<unsigned char *>(B->ell_pool->p);
        for (int32_t i = 0; i < m; ++i) {
            BatchMat &D = B->host_mats[i];
            if (D.fmt != BATCH_ELL) continue;
            D.eval = reinterpret_cast<double *>(base + ell_off[i]);
            D.ecol = reinterpret_cast<int32_t *>(base + ell_off[i] + (uint64_t)D.ld * D.width * 8ull);
            B->plans[i].ell_val = D.eval;
            B->plans[i].ell_idx = D.ecol;
        }
    }
    // the descriptors again, now with the plan; the analysis launch is done
    // with the first copy (the stream was synchronised above)
    CK(cudaMemcpyAsync(B->mats->p, B->host_mats.data(), sizeof(BatchMat) * (size_t)m, cudaMemcpyHostToDevice, s));
    B->d_mats = reinterpret_cast<const BatchMat *>(B->mats->p);
    // tiles: count per matrix, offsets on the host, then the records
    BufPtr cnt_buf;
    CKS(alloc_buf(sizeof(long long) * (size_t)m, s, &cnt_buf));
    long long *d_cnt = reinterpret_cast<long long *>(cnt_buf->p);
    CK(launch_batch_tiles(B->d_mats, m, d_cnt, nullptr, s));
    std::vector<long long> cnt(m);
    CK(cudaMemcpyAsync(cnt.data(), d_cnt, sizeof(long long) * (size_t)m, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    long long total = 0;
    for (int32_t i = 0; i < m; ++i) {
        const long long c = cnt[i];
        cnt[i] = total;
        total += c;
    }
    B->n_tiles = total;
    CK(cudaMemcpyAsync(d_cnt, cnt.data(), sizeof(long long) * (size_t)m, cudaMemcpyHostToDevice, s));
    CKS(alloc_buf(sizeof(int4) * (size_t)std::max<long long>(total, 1), s, &B->tiles));
    CK(launch_batch_tiles(B->d_mats, m, d_cnt, reinterpret_cast<int4 *>(B->tiles->p), s));
    B->d_tiles = reinterpret_cast<const int4 *>(B->tiles->p);
    // One launch builds every ELL matrix (and, given x, computes y for all).
    if (x || B->n_ell > 0) CK(launch_batch_build(B->d_mats, B->d_tiles, B->n_tiles, x, y, s));
    return SPMV_OK;
}

// Tile records a matrix can need with `tpr` lanes per row, whatever its
// format turns out to be (ELL members: 32-row tiles). Greedy CRS tiles of at
// most 32 rows and kTileCap entries: a tile closed by the entry cap and the
// next one hold more than kTileCap entries together, so there are at most
// nnz / (kTileCap / 2) + 1 of those, and n / 32 closed by the row cap.
long long tile_bound(const spmv_crs &A, int tpr) {
    const long long n = A.n_rows, nnz = A.nnz;
    const long long ell = (n + 31) / 32;
    long long crs = n;
    if (tpr == 1) crs = (n + 31) / 32 + nnz / 112 + 2;
    else if (tpr == 8) crs = (n + 3) / 4;
    return std::max(ell, crs);
}

struct PlanWords {                   // device words of a batch planned on the device
    int status;
    int pad;
    unsigned long long n_ell, ell_bytes;
    long long n_tiles;
};

// Copies the device plan to the host (after the stream has run the build).
spmv_status fetch_plan(spmv_batch *B) {
    if (!B->device_plan || B->fetched) return SPMV_OK;
    if (!B->built) return SPMV_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(B->home));
    PlanWords w;
    CK(cudaMemcpy(&w, B->words->p, sizeof(w), cudaMemcpyDeviceToHost));
    CKS(status_from_dev(w.status & ~ST_REDO));
    if (w.status & ST_REDO) return SPMV_ERR_UNSUPPORTED;  // more tile records than bounded (not expected)
    std::vector<BatchPlanOut> po(B->m);
    CK(cudaMemcpy(po.data(), B->plan_out->p, sizeof(BatchPlanOut) * (size_t)B->m, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(B->host_mats.data(), B->mats->p, sizeof(BatchMat) * (size_t)B->m, cudaMemcpyDeviceToHost));
    B->plans.assign(B->m, spmv_batch_plan{});
    for (int32_t i = 0; i < B->m; ++i) {
        const BatchMat &D = B->host_mats[i];
        spmv_batch_plan &P = B->plans[i];
        P.mu = po[i].mu;
        P.sigma = po[i].sigma;
        P.dmat = po[i].dmat;
        P.max_row_len = po[i].max_row_len;
        P.format = D.fmt == BATCH_ELL ? SPMV_ELL : SPMV_CRS;
        P.threads_per_row = D.tpr;
        P.rows_per_tile = D.rpt;
        P.width = D.width;
        P.ld = D.ld;
        P.x_offset = D.xoff;
        P.y_offset = D.yoff;
        P.ell_val = D.eval;
        P.ell_idx = D.ecol;
    }
    B->n_ell = (int32_t)w.n_ell;
    B->ell_bytes = w.ell_bytes;
    B->n_tiles = w.n_tiles;
    B->fetched = true;
    return SPMV_OK;
}

spmv_status prepare_core(const spmv_crs *mats, int32_t m, const spmv_at_params *p, spmv_batch *B, cudaStream_t s) {
    B->device_plan = true;
    B->home = s;
    B->dstar = p ? p->dstar : 0.0;
    B->cap = p ? p->mem_cap_bytes : 0;
    if (B->dstar > 0.0 && B->cap == 0) return SPMV_ERR_INVALID_ARG;  // the ELL pool is sized by the cap
    B->m = m;
    B->host_mats.resize(m);
    std::vector<int2> chunks;
    for (int32_t i = 0; i < m; ++i) {
        const spmv_crs &A = mats[i];
        BatchMat &D = B->host_mats[i];
        memset(&D, 0, sizeof(D));
        D.irp = A.irp;
        D.icol = A.icol;
        D.val = A.val;
        D.xoff = B->total_cols;
        D.yoff = B->total_rows;
        D.nnz = A.nnz;
        D.n_rows = A.n_rows;
        D.n_cols = A.n_cols;
        D.fmt = BATCH_CRS;
        D.tpr = threads_per_row((double)A.nnz / (double)A.n_rows);
        D.rpt = 32 / D.tpr;
        B->total_cols += A.n_cols;
        B->total_rows += A.n_rows;
        B->total_nnz += A.nnz;
        B->tile_cap += tile_bound(A, D.tpr);
        for (int32_t r = 0; r < A.n_rows; r += kBatchChunk) chunks.push_back(make_int2(i, r));
    }
    B->n_chunks = (long long)chunks.size();
    CKS(upload(B->host_mats, s, &B->mats));
    CKS(upload(chunks, s, &B->chunks));
    CKS(alloc_buf(sizeof(BatchAcc) * (size_t)m, s, &B->acc));
    CKS(alloc_buf(sizeof(unsigned long long) * 2 * (size_t)m, s, &B->bytes));
    CKS(alloc_buf(sizeof(BatchPlanOut) * (size_t)m, s, &B->plan_out));
    CKS(alloc_buf(sizeof(long long) * (size_t)m, s, &B->counts));
    CKS(alloc_buf(sizeof(PlanWords), s, &B->words));
    CKS(alloc_buf(sizeof(int4) * (size_t)std::max<int64_t>(B->tile_cap, 1), s, &B->tiles));
    if (B->dstar > 0.0) CKS(alloc_buf(B->cap, s, &B->ell_pool));
    B->d_mats = reinterpret_cast<const BatchMat *>(B->mats->p);
    B->d_tiles = reinterpret_cast<const int4 *>(B->tiles->p);
    B->d_ntiles = &reinterpret_cast<PlanWords *>(B->words->p)->n_tiles;
    CK(cudaStreamSynchronize(s));  // the uploads read host vectors that are kept, but finish them here
    return SPMV_OK;
}

spmv_status build_core(spmv_batch *B, const double *x, double *y, cudaStream_t s) {
    PlanWords *w = reinterpret_cast<PlanWords *>(B->words->p);
    BatchMat *mats = reinterpret_cast<BatchMat *>(B->mats->p);
    long long *cnt = reinterpret_cast<long long *>(B->counts->p);
    CK(cudaMemsetAsync(B->acc->p, 0, sizeof(BatchAcc) * (size_t)B->m, s));
    CK(cudaMemsetAsync(w, 0, sizeof(PlanWords), s));
    CK(launch_batch_analyze(B->d_mats, reinterpret_cast<const int2 *>(B->chunks->p), B->n_chunks,
                            reinterpret_cast<BatchAcc *>(B->acc->p), s));
    CK(launch_batch_plan(mats, reinterpret_cast<const BatchAcc *>(B->acc->p), B->m, B->dstar,
                         B->cap ? B->cap : ~0ull,
                         B->ell_pool ? reinterpret_cast<unsigned char *>(B->ell_pool->p) : nullptr,
                         reinterpret_cast<unsigned long long *>(B->bytes->p),
                         reinterpret_cast<BatchPlanOut *>(B->plan_out->p), &w->n_ell, &w->status, s));
    CK(launch_batch_tiles(B->d_mats, B->m, cnt, nullptr, s));
    CK(launch_batch_tile_offsets(cnt, B->m, B->tile_cap, &w->n_tiles, &w->status, s));
    CK(launch_batch_tiles(B->d_mats, B->m, cnt, reinterpret_cast<int4 *>(B->tiles->p), s, B->d_ntiles));
    if (x || B->dstar > 0.0) CK(launch_batch_build(B->d_mats, B->d_tiles, B->tile_cap, x, y, s, B->d_ntiles));
    B->built = true;
    B->fetched = false;
    return SPMV_OK;
}

}  // namespace

extern "C" {

spmv_status spmv_batch_prepare(const spmv_crs *mats, int32_t m, const spmv_at_params *p, spmv_batch **out,
                               spmv_stream_t stream) {
    if (!out) return SPMV_ERR_INVALID_ARG;
    *out = nullptr;
    if (!mats || m <= 0) return SPMV_ERR_INVALID_ARG;
    if (m > (1 << kBatchMatBits)) return SPMV_ERR_UNSUPPORTED;
    for (int32_t i = 0; i < m; ++i) CKS(check_one(mats[i]));
    spmv_batch *B = new (std::nothrow) spmv_batch();
    if (!B) return SPMV_ERR_OOM;
    spmv_status st = prepare_core(mats, m, p, B, S(stream));
    if (st != SPMV_OK) {
        delete B;
        return st;
    }
    *out = B;
    return SPMV_OK;
}

spmv_status spmv_batch_build(spmv_batch *B, const double *x, double *y, spmv_stream_t stream) {
    if (!B || !B->device_plan) return SPMV_ERR_INVALID_ARG;
    if ((x == nullptr) != (y == nullptr)) return SPMV_ERR_INVALID_ARG;
    return build_core(B, x, y, S(stream));
}

spmv_status spmv_batch_status(spmv_batch *B) {
    if (!B) return SPMV_ERR_INVALID_ARG;
    return fetch_plan(B);
}

spmv_status spmv_batch_schedule_set(const int32_t *tpr_by_class, int32_t n) {
    if (n < 0 || n > kSchedClasses || (n > 0 && !tpr_by_class)) return SPMV_ERR_INVALID_ARG;
    for (int32_t c = 0; c < n; ++c)
        if (tpr_by_class[c] != 1 && tpr_by_class[c] != 8 && tpr_by_class[c] != 32) return SPMV_ERR_INVALID_ARG;
    for (int32_t c = 0; c < n; ++c) g_tpr[c].store(tpr_by_class[c]);
    return SPMV_OK;
}

spmv_status spmv_batch_time(const spmv_batch *B, const double *x, double *y, int32_t warm, int32_t reps,
                            double *ms, spmv_stream_t stream) {
    if (!B || !x || !y || !ms || warm < 0 || reps <= 0) return SPMV_ERR_INVALID_ARG;
    cudaStream_t s = S(stream);
    for (int32_t i = 0; i < warm; ++i) CKS(spmv_batch_apply(B, x, y, stream));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        cudaEventDestroy(e0);
        return SPMV_ERR_CUDA;
    }
    std::vector<float> t;
    spmv_status st = SPMV_OK;
    for (int32_t i = 0; i < reps && st == SPMV_OK; ++i) {
        cudaEventRecord(e0, s);
        st = spmv_batch_apply(B, x, y, stream);
        cudaEventRecord(e1, s);
        float f = 0.f;
        if (st == SPMV_OK && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&f, e0, e1) == cudaSuccess)
            t.push_back(f);
        else if (st == SPMV_OK)
            st = SPMV_ERR_CUDA;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != SPMV_OK) {
        cudaGetLastError();
        return st;
    }
    std::sort(t.begin(), t.end());
    const size_t h = t.size() / 2;
    *ms = (t.size() % 2) ? t[h] : 0.5 * ((double)t[h - 1] + t[h]);
    return SPMV_OK;
}

spmv_status spmv_batch_schedule_get(int32_t *tpr_by_class, int32_t n) {
    if (!tpr_by_class || n < 0 || n > kSchedClasses) return SPMV_ERR_INVALID_ARG;
    for (int32_t c = 0; c < n; ++c) tpr_by_class[c] = g_tpr[c].load();
    return SPMV_OK;
}

spmv_status spmv_batch_create(const spmv_crs *mats, int32_t m, const spmv_at_params *p, const double *x, double *y,
                              spmv_batch **out, spmv_stream_t stream) {
    if (!out) return SPMV_ERR_INVALID_ARG;
    *out = nullptr;
    if (!mats || m <= 0) return SPMV_ERR_INVALID_ARG;
    if (m > (1 << kBatchMatBits)) return SPMV_ERR_UNSUPPORTED;
    if ((x == nullptr) != (y == nullptr)) return SPMV_ERR_INVALID_ARG;
    for (int32_t i = 0; i < m; ++i) CKS(check_one(mats[i]));
    spmv_batch *B = new (std::nothrow) spmv_batch();
    if (!B) return SPMV_ERR_OOM;
    spmv_status st = create_core(mats, m, p, x, y, B, S(stream));
    if (st != SPMV_OK) {
        delete B;
        return st;
    }
    *out = B;
    return SPMV_OK;
}

spmv_status spmv_batch_apply(const spmv_batch *B, const double *x, double *y, spmv_stream_t stream) {
    if (!B || !x || !y) return SPMV_ERR_INVALID_ARG;
    if (B->device_plan) {
        if (!B->built) return SPMV_ERR_INVALID_ARG;
        CK(launch_batch_apply(B->d_mats, B->d_tiles, B->tile_cap, x, y, S(stream), B->d_ntiles));
        return SPMV_OK;
    }
    CK(launch_batch_apply(B->d_mats, B->d_tiles, B->n_tiles, x, y, S(stream)));
    return SPMV_OK;
}

spmv_status spmv_batch_apply_multi(const spmv_batch *B, const double *x, int64_t ldx, double *y, int64_t ldy,
                                   int32_t nvec, spmv_stream_t stream) {
    if (!B || nvec < 0) return SPMV_ERR_INVALID_ARG;
    if (nvec == 0) return SPMV_OK;
    if (!x || !y || ldx < B->total_cols || ldy < B->total_rows) return SPMV_ERR_INVALID_ARG;
    if (B->device_plan) {
        if (!B->built) return SPMV_ERR_INVALID_ARG;
        CK(launch_batch_apply_multi(B->d_mats, B->d_tiles, B->tile_cap, x, (long long)ldx, y, (long long)ldy, nvec,
                                    S(stream), B->d_ntiles));
        return SPMV_OK;
    }
    CK(launch_batch_apply_multi(B->d_mats, B->d_tiles, B->n_tiles, x, (long long)ldx, y, (long long)ldy, nvec,
                                S(stream)));
    return SPMV_OK;
}

spmv_status spmv_batch_info_get(const spmv_batch *B, spmv_batch_info *out) {
    if (!B || !out) return SPMV_ERR_INVALID_ARG;
    CKS(fetch_plan(const_cast<spmv_batch *>(B)));
    memset(out, 0, sizeof(*out));
    out->n_matrices = B->m;
    out->n_ell = B->n_ell;
    out->total_rows = B->total_rows;
    out->total_cols = B->total_cols;
    out->total_nnz = B->total_nnz;
    out->n_tiles = B->n_tiles;
    out->grid = (int32_t)std::min<long long>(B->n_tiles, batch_grid(3));
    out->ell_bytes = B->ell_bytes;
    out->owned_bytes = B->owned();
    return SPMV_OK;
}

spmv_status spmv_batch_plan_get(const spmv_batch *B, int32_t first, int32_t count, spmv_batch_plan *out) {
    if (!B || !out || first < 0 || count < 0 || (int64_t)first + count > B->m) return SPMV_ERR_INVALID_ARG;
    CKS(fetch_plan(const_cast<spmv_batch *>(B)));
    for (int32_t i = 0; i < count; ++i) out[i] = B->plans[first + i];
    return SPMV_OK;
}

void spmv_batch_destroy(spmv_batch *B) { delete B; }

}  // extern "C"
