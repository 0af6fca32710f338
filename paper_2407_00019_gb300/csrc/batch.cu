// C ABI for batches of independent matrices (declared in include/spmvat.h):
// one analysis launch, the on-line rule of Sec. 2.2 per matrix, one ELL
// build launch and one SpMV launch for the whole batch.
#include <algorithm>
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
    uint64_t owned() const {
        uint64_t t = 0;
        for (const BufPtr *b : {&mats, &tiles, &ell_pool})
            if (*b) t += (*b)->bytes;
        return t;
    }
};

namespace {

inline cudaStream_t S(spmv_stream_t s) { return reinterpret_cast<cudaStream_t>(s); }
inline int32_t round_up32(int64_t n) { return (int32_t)((n + 31) / 32 * 32); }

// Lanes per row of a CRS tile. Short rows (the usual case) get one lane each
// and 32-row tiles staged through shared memory; rows long enough that one
// lane would run through hundreds of entries get 8 lanes, or a whole warp.
int threads_per_row(double mu, int max_len) {
    const int v = hint_value(SPMV_HINT_BATCH_TPR);
    if (v == 1 || v == 8 || v == 32) return v;
    if (max_len <= 256 || mu <= 16.0) return 1;
    return mu <= 128.0 ? 8 : 32;
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
            D.tpr = threads_per_row(P.mu, a.max_len);
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

}  // namespace

extern "C" {

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
    CK(launch_batch_apply(B->d_mats, B->d_tiles, B->n_tiles, x, y, S(stream)));
    return SPMV_OK;
}

spmv_status spmv_batch_apply_multi(const spmv_batch *B, const double *x, int64_t ldx, double *y, int64_t ldy,
                                   int32_t nvec, spmv_stream_t stream) {
    if (!B || nvec < 0) return SPMV_ERR_INVALID_ARG;
    if (nvec == 0) return SPMV_OK;
    if (!x || !y || ldx < B->total_cols || ldy < B->total_rows) return SPMV_ERR_INVALID_ARG;
    CK(launch_batch_apply_multi(B->d_mats, B->d_tiles, B->n_tiles, x, (long long)ldx, y, (long long)ldy, nvec,
                                S(stream)));
    return SPMV_OK;
}

spmv_status spmv_batch_info_get(const spmv_batch *B, spmv_batch_info *out) {
    if (!B || !out) return SPMV_ERR_INVALID_ARG;
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
    for (int32_t i = 0; i < count; ++i) out[i] = B->plans[first + i];
    return SPMV_OK;
}

void spmv_batch_destroy(spmv_batch *B) { delete B; }

}  // extern "C"
