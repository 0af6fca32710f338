// Two-stage TMA pipeline that copies a contiguous range of a float64 array
// (and the same range of up to two int32 arrays) into shared memory.
//
// One thread issues, for stage `st`, two 1-D bulk copies (cp.async.bulk) of
// the 16-byte-aligned interior of the entry range [e0, e1); the few entries
// outside it (at most one value and three indices per edge) and whole ranges
// larger than a stage are read from global memory by the consumers. Stage
// completion is an mbarrier with expected transaction bytes; every wait is
// bounded. A CTA alternates stages, so the copy for its next tile runs while
// it consumes the current one.
#pragma once

#include "common.cuh"

namespace spmvat {

struct StageMeta {
    long long e0, e1;    // the entry range of the tile
    long long a0v, b0v;  // staged value range [a0v, b0v)
    long long a0i, b0i;  // staged index range [a0i, b0i) (both index arrays)
    int staged;
    int pad;
};

// NIDX = number of int32 arrays staged with the float64 one (0, 1 or 2).
template <int CAP, int NIDX>
struct StagePipe {
    static constexpr bool WITH_IDX = NIDX > 0;
    static constexpr size_t kHeader = 128;
    static constexpr size_t kStage = (size_t)CAP * 8 + (size_t)NIDX * CAP * 4;
    static constexpr size_t kSmem = kHeader + 2 * kStage;
    static_assert(CAP % 4 == 0, "stage capacity must keep 16-byte alignment");

    uint64_t *bar;
    StageMeta *meta;
    unsigned char *base;

    __device__ void setup(unsigned char *smem) {
        bar = reinterpret_cast<uint64_t *>(smem);
        meta = reinterpret_cast<StageMeta *>(smem + 16);
        base = smem + kHeader;
        if (threadIdx.x == 0) {
            mbar_init(&bar[0], 1);
            mbar_init(&bar[1], 1);
            fence_mbar_init();
        }
        __syncthreads();
    }
    __device__ double *sval(int st) const { return reinterpret_cast<double *>(base + st * kStage); }
    __device__ int32_t *sidx(int st) const {
        return reinterpret_cast<int32_t *>(base + st * kStage + (size_t)CAP * 8);
    }
    __device__ int32_t *sidx2(int st) const {
        return reinterpret_cast<int32_t *>(base + st * kStage + (size_t)CAP * 12);
    }

    // Thread 0 only. `can_stage`: all base pointers are 16-byte aligned.
    __device__ void issue(int st, long long e0, long long e1, const double *val, const int32_t *idx,
                          bool can_stage, const int32_t *idx2 = nullptr) {
        StageMeta m;
        if (e1 < e0) e1 = e0;
        m.e0 = e0;
        m.e1 = e1;
        m.a0v = e0 & ~1ll;
        m.b0v = max(m.a0v, e1 & ~1ll);
        m.a0i = e0 & ~3ll;
        m.b0i = WITH_IDX ? max(m.a0i, e1 & ~3ll) : m.a0i;
        const unsigned bv = (unsigned)((m.b0v - m.a0v) * 8);
        const unsigned bi = (unsigned)((m.b0i - m.a0i) * 4);
        m.staged = can_stage && (m.b0v - m.a0v) <= CAP && (m.b0i - m.a0i) <= CAP && (bv + bi) > 0;
        m.pad = 0;
        meta[st] = m;
        if (m.staged) {
            mbar_arrive_expect_tx(&bar[st], bv + (unsigned)NIDX * bi);
            if (bv) bulk_g2s(sval(st), val + m.a0v, bv, &bar[st]);
            if (NIDX >= 1 && bi) bulk_g2s(sidx(st), idx + m.a0i, bi, &bar[st]);
            if (NIDX >= 2 && bi) bulk_g2s(sidx2(st), idx2 + m.a0i, bi, &bar[st]);
        } else {
            mbar_arrive_expect_tx(&bar[st], 0);
        }
    }

    // All threads. `use` counts the previous waits on this stage.
    __device__ bool wait(int st, int use) { return mbar_wait_bounded(&bar[st], (unsigned)(use & 1), kSpinLimit); }

    __device__ __forceinline__ double val_at(const StageMeta &m, int st, const double *val, long long k) const {
        return (m.staged && k >= m.a0v && k < m.b0v) ? sval(st)[k - m.a0v] : val[k];
    }
    __device__ __forceinline__ int32_t idx_at(const StageMeta &m, int st, const int32_t *idx, long long k) const {
        return (m.staged && k >= m.a0i && k < m.b0i) ? sidx(st)[k - m.a0i] : idx[k];
    }
    __device__ __forceinline__ int32_t idx2_at(const StageMeta &m, int st, const int32_t *idx2, long long k) const {
        return (m.staged && k >= m.a0i && k < m.b0i) ? sidx2(st)[k - m.a0i] : idx2[k];
    }
};

// Standard loop over tiles with the pipeline. `range(tile, &e0, &e1)` gives
// a tile's entry range (thread 0 only); `pre(tile)` returns what every thread
// loads for a tile before consuming it (for example its line pointers);
// `body(tile, st, meta, pre)` consumes it; all threads call. Both loads run
// ahead of their use: thread 0 loads the range of the tile after next while
// the current tile is consumed, and every thread loads `pre` of the next
// tile, so no tile waits for them. On a wait that runs out, sets ST_TIMEOUT,
// waits (bounded) for the copies in flight and returns false.
template <class Pipe, class RangeF, class PreF, class BodyF>
__device__ bool pipe_tiles(Pipe &P, int n_tiles, const double *val, const int32_t *idx, bool can_stage,
                           int *status, RangeF range, PreF pre, BodyF body, const int32_t *idx2 = nullptr) {
    const int G = gridDim.x;
    int tile = blockIdx.x;
    if (tile >= n_tiles) return true;
    long long f0 = 0, f1 = 0;  // thread 0: the range of the next tile to issue
    if (threadIdx.x == 0) {
        long long e0, e1;
        range(tile, &e0, &e1);
        P.issue(0, e0, e1, val, idx, can_stage, idx2);
        if (tile + G < n_tiles) range(tile + G, &f0, &f1);
    }
    auto cur = pre(tile);
    for (int it = 0; tile < n_tiles; tile += G, ++it) {
        const int st = it & 1;
        const int next = tile + G;
        if (threadIdx.x == 0 && next < n_tiles) {
            P.issue(st ^ 1, f0, f1, val, idx, can_stage, idx2);
            if (next + G < n_tiles) range(next + G, &f0, &f1);
        }
        const auto nxt = (next < n_tiles) ? pre(next) : cur;
        const bool ok = P.wait(st, it >> 1);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                atomicOr(status, ST_TIMEOUT);
                P.wait(st, it >> 1);
                if (next < n_tiles) P.wait(st ^ 1, (it + 1) >> 1);
            }
            return false;
        }
        const StageMeta m = P.meta[st];
        body(tile, st, m, cur);
        __syncthreads();
        cur = nxt;
    }
    return true;
}

}  // namespace spmvat
