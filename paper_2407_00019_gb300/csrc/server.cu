// Serving runtime (declared in include/spmvat.h): continuous batching of
// SpMV requests over a pool of matrices, with a resident per-matrix format
// cache under a device-memory budget. Each matrix is held as a batch of one
// (its CRS schedule, and its ELL-Row when cached), so a request's k products
// are one multi-vector launch that reads the matrix once.
//
// Threads: clients call add/submit/wait; one worker thread owns the slots,
// the pending queue and the cache, and is the only caller of the transform
// and product entry points for requests. Completion is signalled by a host
// function enqueued after a request's products on its slot's stream; it only
// stamps the time and wakes the worker (no CUDA call, no lock held by anyone
// across a CUDA call).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <climits>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "spmvat.h"

namespace {

using Clock = std::chrono::steady_clock;
double now_s() { return std::chrono::duration<double>(Clock::now().time_since_epoch()).count(); }

enum : int { R_PENDING = 0, R_RUNNING = 1, R_DONE = 2, R_REAPED = 3 };

// Admission counts a transformation as its arrays and tile records plus this
// much for its small buffers (each allocation is rounded up to 256 bytes).
constexpr uint64_t kHandleSlack = 4096;

struct Request {
    uint64_t id = 0;
    int32_t mat = 0, k = 0;
    const double *x = nullptr;
    double *y = nullptr;
    cudaEvent_t ready = nullptr;  // recorded on the caller's `after` stream, or NULL
    double t_submit = 0.0;
    std::atomic<double> t_done{0.0};
    int32_t format = SPMV_CRS;
    bool cached = false;
    spmv_status status = SPMV_OK;
    std::atomic<int> state{R_PENDING};
    spmv_server *srv = nullptr;
};

struct MatEntry {
    spmv_crs A{};
    int32_t target = SPMV_CRS;
    uint64_t target_bytes = 0;       // device bytes of the target transformation
    spmv_batch *crs = nullptr;       // the matrix alone as a batch, in CRS (always present)
    spmv_matrix *plain = nullptr;    // CRS handle of spmv_transform: SPMV_SERVER_PLAIN, and uneven rows
    bool uneven = false;             // D_mat > 0.5 or a row of 2048 entries or more: products in CRS
                                     // run as spmv_apply on `plain` (the entry-split product), which on
                                     // such rows beats the batch product even with k vectors at once
    spmv_batch *fast = nullptr;      // the same in its target format (cached), or NULL
    cudaEvent_t built = nullptr;     // recorded after the transformation's kernels
    uint64_t fast_bytes = 0;
    int64_t products = 0;            // products asked for so far
    int64_t breakeven = 0;           // products before the transformation pays off; < 0: never
    int inflight_fast = 0;           // running requests that use `fast`
    uint64_t last_use = 0;
    double bytes_crs = 0.0, bytes_fast = 0.0;  // algorithmic bytes per product
};

}  // namespace

struct spmv_server {
    spmv_server_params p{};
    int device = 0;
    std::vector<cudaStream_t> streams;
    std::vector<Request *> slot_req;  // worker only
    cudaStream_t ctrl = nullptr;      // registration work

    std::mutex pool_mu;               // guards the vector, not the entries
    std::vector<std::unique_ptr<MatEntry>> mats;

    std::mutex in_mu;                 // incoming queue and the request table
    std::deque<Request *> incoming;
    std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
    uint64_t next_id = 1;

    std::thread worker;
    std::atomic<bool> stop{false};
    std::mutex wake_mu;
    std::condition_variable wake_cv;
    bool wake = false;

    std::mutex done_mu;
    std::condition_variable done_cv;
    std::atomic<uint64_t> outstanding{0};

    std::mutex stats_mu;
    spmv_server_stats stats{};
    std::vector<double> lat_ms;
    double t_first = 0.0, t_last = 0.0;
    uint64_t lru = 0;                 // worker only
};

namespace {

void poke(spmv_server *S) {
    {
        std::lock_guard<std::mutex> lk(S->wake_mu);
        S->wake = true;
    }
    S->wake_cv.notify_one();
}

void CUDART_CB on_done(void *arg) {
    Request *r = static_cast<Request *>(arg);
    r->t_done.store(now_s());
    r->state.store(R_DONE, std::memory_order_release);
    poke(r->srv);
}

MatEntry *entry(spmv_server *S, int32_t id) {
    std::lock_guard<std::mutex> lk(S->pool_mu);
    return (id >= 0 && id < (int32_t)S->mats.size()) ? S->mats[id].get() : nullptr;
}

// Frees least-recently-used idle transformations until `bytes` more fit.
bool make_room(spmv_server *S, uint64_t bytes) {
    const uint64_t budget = S->p.mem_budget_bytes;
    if (budget == 0) return true;
    if (bytes > budget) return false;
    while (S->stats.cache_bytes + bytes > budget) {
        MatEntry *victim = nullptr;
        std::vector<MatEntry *> all;
        {
            std::lock_guard<std::mutex> lk(S->pool_mu);
            for (auto &e : S->mats) all.push_back(e.get());
        }
        for (MatEntry *e : all)
            if (e->fast && e->inflight_fast == 0 && (!victim || e->last_use < victim->last_use)) victim = e;
        if (!victim) return false;
        spmv_batch_destroy(victim->fast);
        victim->fast = nullptr;
        std::lock_guard<std::mutex> lk(S->stats_mu);
        S->stats.cache_bytes -= victim->fast_bytes;
        S->stats.evictions += 1;
        victim->fast_bytes = 0;
    }
    return true;
}

void admit(spmv_server *S, Request *r, int slot) {
    cudaStream_t s = S->streams[slot];
    MatEntry *E = entry(S, r->mat);
    if (r->ready) cudaStreamWaitEvent(s, r->ready, 0);
    E->products += r->k;
    if ((S->p.flags & SPMV_SERVER_PLAIN) || (E->uneven && !E->fast && E->target == SPMV_CRS)) {
        // the per-matrix form (one spmv_apply per product, CRS, in arrival
        // order), and CRS products of uneven rows
        r->status = SPMV_OK;
        for (int32_t j = 0; j < r->k && r->status == SPMV_OK; ++j)
            r->status = spmv_apply(E->plain, r->x + (size_t)j * E->A.n_cols, r->y + (size_t)j * E->A.n_rows, s);
        r->format = SPMV_CRS;
        r->cached = false;
        r->state.store(R_RUNNING);
        S->slot_req[slot] = r;
        if (cudaLaunchHostFunc(s, on_done, r) != cudaSuccess) {
            cudaGetLastError();
            cudaStreamSynchronize(s);
            r->status = r->status == SPMV_OK ? SPMV_ERR_CUDA : r->status;
            on_done(r);
        }
        return;
    }
    spmv_batch *H = E->crs;
    bool miss = false;
    if (E->target != SPMV_CRS) {
        if (E->fast) {
            H = E->fast;
        } else if (E->breakeven >= 0 && E->products >= E->breakeven && make_room(S, E->target_bytes)) {
            spmv_batch *M = nullptr;
            if (!E->built && cudaEventCreateWithFlags(&E->built, cudaEventDisableTiming) != cudaSuccess) {
                cudaGetLastError();
                E->built = nullptr;
            }
            spmv_at_params ell;
            memset(&ell, 0, sizeof(ell));
            ell.dstar = INFINITY;  // the target is ELL-Row
            if (E->built && spmv_batch_create(&E->A, 1, &ell, nullptr, nullptr, &M, s) == SPMV_OK) {
                cudaEventRecord(E->built, s);  // requests on other slots wait for the build
                spmv_batch_info d;
                spmv_batch_info_get(M, &d);
                E->fast = M;
                E->fast_bytes = d.owned_bytes;
                H = M;
                std::lock_guard<std::mutex> lk(S->stats_mu);
                S->stats.transforms += 1;
                S->stats.cache_bytes += d.owned_bytes;
                S->stats.peak_cache_bytes = std::max(S->stats.peak_cache_bytes, S->stats.cache_bytes);
            }
            miss = true;  // this request paid for the transformation
        } else {
            miss = true;
        }
    }
    r->cached = (H == E->fast && H != nullptr);
    if (r->cached) {
        E->inflight_fast += 1;
        cudaStreamWaitEvent(s, E->built, 0);
    }
    r->format = r->cached ? E->target : SPMV_CRS;
    E->last_use = ++S->lru;
    {
        std::lock_guard<std::mutex> lk(S->stats_mu);
        if (E->target != SPMV_CRS) {
            if (r->cached && !miss) S->stats.cache_hits += 1;
            else S->stats.cache_misses += 1;
        }
    }
    // the request's k products in one launch: the matrix is read once for all k
    r->status = spmv_batch_apply_multi(H, r->x, E->A.n_cols, r->y, E->A.n_rows, r->k, s);
    r->state.store(R_RUNNING);
    S->slot_req[slot] = r;
    if (cudaLaunchHostFunc(s, on_done, r) != cudaSuccess) {
        cudaGetLastError();
        cudaStreamSynchronize(s);
        r->status = r->status == SPMV_OK ? SPMV_ERR_CUDA : r->status;
        on_done(r);
    }
}

void reap(spmv_server *S, Request *r) {
    MatEntry *E = entry(S, r->mat);
    if (r->cached) E->inflight_fast -= 1;
    const double t_done = r->t_done.load();
    {
        std::lock_guard<std::mutex> lk(S->stats_mu);
        if (r->status == SPMV_OK) {
            S->stats.completed += 1;
            S->stats.products += (uint64_t)r->k;
            S->stats.bytes += (double)r->k * (r->cached ? E->bytes_fast : E->bytes_crs);
            S->lat_ms.push_back((t_done - r->t_submit) * 1e3);
        } else {
            S->stats.failed += 1;
        }
        S->t_last = std::max(S->t_last, t_done);
    }
    if (r->ready) {
        cudaEventDestroy(r->ready);
        r->ready = nullptr;
    }
    {
        std::lock_guard<std::mutex> lk(S->done_mu);
        r->state.store(R_REAPED, std::memory_order_release);
        S->outstanding.fetch_sub(1);
    }
    S->done_cv.notify_all();
}

void worker_main(spmv_server *S) {
    cudaSetDevice(S->device);
    std::deque<Request *> pending;
    const int n = (int)S->streams.size();
    for (;;) {
        {
            std::lock_guard<std::mutex> lk(S->in_mu);
            while (!S->incoming.empty()) {
                pending.push_back(S->incoming.front());
                S->incoming.pop_front();
            }
        }
        int busy = 0;
        for (int i = 0; i < n; ++i) {
            Request *r = S->slot_req[i];
            if (r && r->state.load(std::memory_order_acquire) == R_DONE) {
                S->slot_req[i] = nullptr;
                reap(S, r);
            }
            busy += S->slot_req[i] != nullptr;
        }
        for (int i = 0; i < n && !pending.empty(); ++i) {
            if (S->slot_req[i]) continue;
            Request *r = pending.front();
            pending.pop_front();
            admit(S, r, i);
            ++busy;
        }
        if (S->stop.load() && pending.empty() && busy == 0) {
            std::lock_guard<std::mutex> lk(S->in_mu);
            if (S->incoming.empty()) break;
        }
        std::unique_lock<std::mutex> lk(S->wake_mu);
        S->wake_cv.wait_for(lk, std::chrono::microseconds(500), [S] { return S->wake; });
        S->wake = false;
    }
}

double percentile(std::vector<double> v, double q) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const size_t i = (size_t)std::min<double>((double)v.size() - 1, std::ceil(q * (double)v.size()) - 1);
    return v[i];
}

}  // namespace

extern "C" {

spmv_status spmv_server_create(const spmv_server_params *p, spmv_server **out) {
    if (!out) return SPMV_ERR_INVALID_ARG;
    *out = nullptr;
    std::unique_ptr<spmv_server> S(new (std::nothrow) spmv_server());
    if (!S) return SPMV_ERR_OOM;
    if (p) S->p = *p;
    if (S->p.n_streams <= 0) S->p.n_streams = 4;
    if (S->p.flags & SPMV_SERVER_PLAIN) S->p.n_streams = 1;  // serial, one request at a time
    if (S->p.n_streams > 64) return SPMV_ERR_INVALID_ARG;
    if (S->p.amortize_products <= 0) S->p.amortize_products = 2;
    if (cudaGetDevice(&S->device) != cudaSuccess) { cudaGetLastError(); return SPMV_ERR_CUDA; }
    S->streams.assign(S->p.n_streams, nullptr);
    S->slot_req.assign(S->p.n_streams, nullptr);
    for (auto &s : S->streams)
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            for (auto &t : S->streams) if (t) cudaStreamDestroy(t);
            return SPMV_ERR_CUDA;
        }
    if (cudaStreamCreateWithFlags(&S->ctrl, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        for (auto &t : S->streams) cudaStreamDestroy(t);
        return SPMV_ERR_CUDA;
    }
    spmv_server *raw = S.get();
    try {
        S->worker = std::thread(worker_main, raw);
    } catch (...) {
        for (auto &t : S->streams) cudaStreamDestroy(t);
        cudaStreamDestroy(S->ctrl);
        return SPMV_ERR_UNSUPPORTED;
    }
    *out = S.release();
    return SPMV_OK;
}

spmv_status spmv_server_add_matrix(spmv_server *S, const spmv_crs *A, int32_t *id) {
    if (!S || !A || !id) return SPMV_ERR_INVALID_ARG;
    std::unique_ptr<MatEntry> E(new (std::nothrow) MatEntry());
    if (!E) return SPMV_ERR_OOM;
    E->A = *A;
    spmv_at_params ap;
    memset(&ap, 0, sizeof(ap));
    ap.c = 1.0;
    ap.dstar = S->p.dstar;
    ap.mem_cap_bytes = S->p.mem_budget_bytes;
    int32_t fmt = SPMV_CRS, layout = SPMV_ROWWISE;
    spmv_stats st;
    spmv_status rc = spmv_autotune_choose(A, &ap, &fmt, &layout, &st, S->ctrl);
    if (rc != SPMV_OK) return rc;
    spmv_at_params crs;
    memset(&crs, 0, sizeof(crs));  // D* = 0: CRS
    E->uneven = st.dmat > 0.5 || st.max_row_len >= 2048;
    if (S->p.flags & SPMV_SERVER_PLAIN) {
        rc = spmv_transform(A, SPMV_CRS, SPMV_ROWWISE, 0, &E->plain, S->ctrl);
        if (rc != SPMV_OK) return rc;
        fmt = SPMV_CRS;  // no format cache in the per-matrix form
    } else {
        rc = spmv_batch_create(A, 1, &crs, nullptr, nullptr, &E->crs, S->ctrl);
        if (rc != SPMV_OK) return rc;
        if (E->uneven && fmt == SPMV_CRS) {
            rc = spmv_transform(A, SPMV_CRS, SPMV_ROWWISE, 0, &E->plain, S->ctrl);
            if (rc != SPMV_OK) {
                spmv_batch_destroy(E->crs);
                return rc;
            }
        }
    }
    if (cudaStreamSynchronize(S->ctrl) != cudaSuccess) {
        cudaGetLastError();
        if (E->crs) spmv_batch_destroy(E->crs);
        if (E->plain) spmv_destroy(E->plain);
        return SPMV_ERR_CUDA;
    }
    E->target = fmt;
    // ELL arrays, one 16-byte tile record per 32 rows, descriptors
    E->target_bytes = st.ell_bytes + 16ull * (uint64_t)((A->n_rows + 31) / 32) + kHandleSlack;
    const double n = (double)A->n_rows, nc = (double)A->n_cols;
    const double ell = 12.0 * (double)((A->n_rows + 31) / 32 * 32) * (double)st.max_row_len;
    E->bytes_crs = 12.0 * (double)A->nnz + 4.0 * (n + 1.0) + 8.0 * nc + 8.0 * n;
    E->bytes_fast = ell + 8.0 * nc + 8.0 * n;
    // Break-even of the transformation (Sec. 2.2, Eqs. (1)-(3)) with moved
    // bytes standing in for times: SP = CRS bytes / ELL bytes per product,
    // TT = transformation bytes / CRS bytes; k products pay for it once
    // k t_crs >= t_trans + k t_ell, i.e. k >= TT / (1 - 1 / SP). Never when
    // SP <= 1, nor when one transformation would take over a quarter of the
    // cache budget (it would evict everything else).
    const double trans = 12.0 * (double)A->nnz + 4.0 * (n + 1.0) + ell;
    const double sp = E->bytes_crs / E->bytes_fast, tt = trans / E->bytes_crs;
    const bool fits = S->p.mem_budget_bytes == 0 || E->target_bytes <= S->p.mem_budget_bytes / 4;
    if (fmt == SPMV_CRS) {
        E->breakeven = -1;
    } else if (S->p.flags & SPMV_SERVER_FIXED_THRESHOLD) {
        E->breakeven = S->p.amortize_products;
    } else if (sp <= 1.0 || !fits) {
        E->breakeven = -1;
    } else {
        const double k = std::ceil(tt / (1.0 - 1.0 / sp));
        E->breakeven = std::max<int64_t>(S->p.amortize_products, k < 1e15 ? (int64_t)k : (int64_t)1e15);
    }
    std::lock_guard<std::mutex> lk(S->pool_mu);
    *id = (int32_t)S->mats.size();
    S->mats.push_back(std::move(E));
    return SPMV_OK;
}

spmv_status spmv_server_submit(spmv_server *S, int32_t id, int32_t k, const double *x, double *y,
                               spmv_stream_t after, uint64_t *req) {
    if (!S || !req || k < 0 || S->stop.load()) return SPMV_ERR_INVALID_ARG;
    if (k > 0 && (!x || !y)) return SPMV_ERR_INVALID_ARG;
    if (!entry(S, id)) return SPMV_ERR_INVALID_ARG;
    std::unique_ptr<Request> r(new (std::nothrow) Request());
    if (!r) return SPMV_ERR_OOM;
    r->mat = id;
    r->k = k;
    r->x = x;
    r->y = y;
    r->srv = S;
    if (after) {
        if (cudaEventCreateWithFlags(&r->ready, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventRecord(r->ready, reinterpret_cast<cudaStream_t>(after)) != cudaSuccess) {
            cudaGetLastError();
            if (r->ready) cudaEventDestroy(r->ready);
            return SPMV_ERR_CUDA;
        }
    }
    r->t_submit = now_s();
    {
        std::lock_guard<std::mutex> lk(S->stats_mu);
        if (S->stats.submitted == 0) S->t_first = r->t_submit;
        S->stats.submitted += 1;
    }
    S->outstanding.fetch_add(1);
    {
        std::lock_guard<std::mutex> lk(S->in_mu);
        r->id = S->next_id++;
        *req = r->id;
        S->incoming.push_back(r.get());
        S->reqs.emplace(r->id, std::move(r));
    }
    poke(S);
    return SPMV_OK;
}

spmv_status spmv_server_wait(spmv_server *S, uint64_t req, int32_t timeout_ms, double *latency_ms,
                             int32_t *format) {
    if (!S) return SPMV_ERR_INVALID_ARG;
    Request *r = nullptr;
    {
        std::lock_guard<std::mutex> lk(S->in_mu);
        auto it = S->reqs.find(req);
        if (it == S->reqs.end()) return SPMV_ERR_INVALID_ARG;
        r = it->second.get();
    }
    {
        std::unique_lock<std::mutex> lk(S->done_mu);
        auto done = [r] { return r->state.load(std::memory_order_acquire) == R_REAPED; };
        if (timeout_ms < 0) S->done_cv.wait(lk, done);
        else if (!S->done_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) return SPMV_ERR_TIMEOUT;
    }
    const spmv_status st = r->status;
    if (latency_ms) *latency_ms = (r->t_done.load() - r->t_submit) * 1e3;
    if (format) *format = r->format;
    std::lock_guard<std::mutex> lk(S->in_mu);
    S->reqs.erase(req);
    return st;
}

spmv_status spmv_server_drain(spmv_server *S, int32_t timeout_ms) {
    if (!S) return SPMV_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->done_mu);
    auto done = [S] { return S->outstanding.load() == 0; };
    if (timeout_ms < 0) S->done_cv.wait(lk, done);
    else if (!S->done_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) return SPMV_ERR_TIMEOUT;
    return SPMV_OK;
}

spmv_status spmv_server_stats_get(spmv_server *S, spmv_server_stats *out, int32_t reset) {
    if (!S || !out) return SPMV_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->stats_mu);
    *out = S->stats;
    out->p50_ms = percentile(S->lat_ms, 0.50);
    out->p99_ms = percentile(S->lat_ms, 0.99);
    double sum = 0.0, mx = 0.0;
    for (double v : S->lat_ms) {
        sum += v;
        mx = std::max(mx, v);
    }
    out->mean_ms = S->lat_ms.empty() ? 0.0 : sum / (double)S->lat_ms.size();
    out->max_ms = mx;
    out->busy_s = S->t_last > S->t_first ? S->t_last - S->t_first : 0.0;
    if (reset) {
        const uint64_t cb = S->stats.cache_bytes;
        memset(&S->stats, 0, sizeof(S->stats));
        S->stats.cache_bytes = cb;
        S->stats.peak_cache_bytes = cb;
        S->lat_ms.clear();
        S->t_first = S->t_last = 0.0;
    }
    return SPMV_OK;
}

void spmv_server_destroy(spmv_server *S) {
    if (!S) return;
    S->stop.store(true);
    poke(S);
    if (S->worker.joinable()) S->worker.join();
    for (auto &e : S->mats) {
        if (e->fast) spmv_batch_destroy(e->fast);
        if (e->crs) spmv_batch_destroy(e->crs);
        if (e->plain) spmv_destroy(e->plain);
        if (e->built) cudaEventDestroy(e->built);
    }
    for (auto &s : S->streams) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
    cudaStreamSynchronize(S->ctrl);
    cudaStreamDestroy(S->ctrl);
    for (auto &kv : S->reqs)
        if (kv.second->ready) cudaEventDestroy(kv.second->ready);
    delete S;
}

}  // extern "C"
