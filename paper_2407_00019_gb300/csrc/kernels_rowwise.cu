// Row-wise transformations of Sec. 2.1 and the row statistics of Eq. (4).
//
//  k_analyze        : row lengths -> sum, sum of squares, max, min, empties,
//                     log2-class histogram, IRP sanity (Sec. 2.2, Eq. (4)).
//  k_validate_idx   : every index in [0, bound).
//  k_expand         : entry -> line index (COO-Row IROW, Sec. 2.1; Phase II
//                     CCS -> COO-Column, Sec. 2.1).
//  k_lines_to_ell   : compressed lines -> padded column-major ELL (Sec. 2.1,
//                     Fig. 3 indexing), TMA bulk-staged and double-buffered;
//                     optionally computes y = A x from the staged entries in
//                     the same pass (fused transformation + first SpMV).
#include <climits>

#include "common.cuh"
#include "stage_pipe.cuh"

namespace spmvat {

// ---------------------------------------------------------------- analyze
// One pass: each thread takes AN_ITEMS consecutive rows (one 16-byte load of
// IRP plus the next pointer), so all loads of a warp are in flight at once.
constexpr int AN_THREADS = 256;
constexpr int AN_ITEMS = 4;

__global__ void __launch_bounds__(AN_THREADS) k_analyze(const int32_t *__restrict__ irp, int32_t n, int64_t nnz,
                                                         AnalyzeAcc *acc) {
    __shared__ unsigned long long s_hist[32];
    __shared__ unsigned long long s_sum[AN_THREADS / 32][3];
    __shared__ int s_mm[AN_THREADS / 32][3];
    if (threadIdx.x < 32) s_hist[threadIdx.x] = 0ull;
    __syncthreads();
    unsigned long long sl = 0, sl2 = 0, ne = 0;
    int mx = 0, inv_mn = 0, bad = 0;
    {
        const long long i0 = ((long long)blockIdx.x * AN_THREADS + threadIdx.x) * AN_ITEMS;
        int p[AN_ITEMS + 1];
        if (i0 + AN_ITEMS <= n && ((reinterpret_cast<uintptr_t>(irp + i0) & 15) == 0)) {
            const int4 q = *reinterpret_cast<const int4 *>(irp + i0);
            p[0] = q.x; p[1] = q.y; p[2] = q.z; p[3] = q.w;
            p[4] = irp[i0 + 4];
        } else {
#pragma unroll
            for (int j = 0; j <= AN_ITEMS; ++j) p[j] = (i0 + j <= n) ? irp[i0 + j] : 0;
        }
#pragma unroll
        for (int j = 0; j < AN_ITEMS; ++j) {
            const long long i = i0 + j;
            const bool has = i < n;
            int len = 0;
            if (has) {
                len = p[j + 1] - p[j];
                if (len < 0 || p[j] < 0 || (long long)p[j + 1] > nnz) { bad = 1; len = len < 0 ? 0 : len; }
                if (i == 0 && p[0] != 0) bad = 1;
                if (i == n - 1 && (long long)p[j + 1] != nnz) bad = 1;
                sl += (unsigned)len;
                sl2 += (unsigned long long)len * (unsigned long long)len;
                ne += (len == 0);
                mx = max(mx, len);
                inv_mn = max(inv_mn, INT_MAX - len);
            }
            // length class histogram: one round per distinct class in the
            // warp (regular matrices have one or two)
            const int cls = has ? ((len == 0) ? 0 : 32 - __clz(len)) : 32;
            unsigned todo = __ballot_sync(0xffffffffu, has);
            while (todo) {
                const int c = __shfl_sync(0xffffffffu, cls, __ffs(todo) - 1);
                const unsigned m = __ballot_sync(0xffffffffu, has && cls == c);
                if ((int)lane_id() == __ffs(todo) - 1) atomicAdd(&s_hist[c], (unsigned long long)__popc(m));
                todo &= ~m;
            }
        }
    }
    sl = warp_sum(sl);
    sl2 = warp_sum(sl2);
    ne = warp_sum(ne);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        inv_mn = max(inv_mn, __shfl_xor_sync(0xffffffffu, inv_mn, o));
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    const int w = threadIdx.x >> 5;
    if (lane_id() == 0) {
        s_sum[w][0] = sl; s_sum[w][1] = sl2; s_sum[w][2] = ne;
        s_mm[w][0] = mx; s_mm[w][1] = inv_mn; s_mm[w][2] = bad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int j = 1; j < AN_THREADS / 32; ++j) {
            sl += s_sum[j][0]; sl2 += s_sum[j][1]; ne += s_sum[j][2];
            mx = max(mx, s_mm[j][0]); inv_mn = max(inv_mn, s_mm[j][1]); bad |= s_mm[j][2];
        }
        atomicAdd(&acc->sum_len, sl);
        atomicAdd(&acc->sum_len2, sl2);
        atomicAdd(&acc->n_empty, ne);
        atomicMax(&acc->max_len, mx);
        atomicMax(&acc->min_len, inv_mn);  // stores INT_MAX - min
        if (bad) atomicOr(&acc->status, ST_BAD_PTR);
    }
    if (threadIdx.x < 32 && s_hist[threadIdx.x]) atomicAdd(&acc->hist[threadIdx.x], s_hist[threadIdx.x]);
}

cudaError_t launch_analyze(const int32_t *irp, int32_t n_rows, int64_t nnz, AnalyzeAcc *acc, cudaStream_t s) {
    const unsigned grid = ceil_div_u(n_rows, (long long)AN_THREADS * AN_ITEMS);
    KernelScope ks("analyze", s);
    k_analyze<<<grid, AN_THREADS, 0, s>>>(irp, n_rows, nnz, acc);
    return cudaGetLastError();
}

// The pass an ELL build needs of the row pointers: the longest row and the
// same pointer checks as k_analyze (first 0, last nnz, none decreasing, all
// in [0, nnz]), nothing else. Persistent CTAs, rows in a grid-stride loop,
// one accumulator update per CTA.
constexpr int RW_CTAS_PER_SM = 4;
constexpr int RW_ITEMS = 4;  // rows a thread takes at a time (16-byte loads of IRP)
static_assert(RW_ITEMS % 4 == 0, "whole 16-byte loads");

__global__ void __launch_bounds__(AN_THREADS) k_row_width(const int32_t *__restrict__ irp, int32_t n, int64_t nnz,
                                                           AnalyzeAcc *acc) {
    __shared__ int s_mx[AN_THREADS / 32], s_bad[AN_THREADS / 32];
    int mx = 0, bad = 0;
    const long long stride = (long long)gridDim.x * AN_THREADS * RW_ITEMS;
    for (long long i0 = ((long long)blockIdx.x * AN_THREADS + threadIdx.x) * RW_ITEMS; i0 < n; i0 += stride) {
        int p[RW_ITEMS + 1];
        if (i0 + RW_ITEMS <= n && ((reinterpret_cast<uintptr_t>(irp + i0) & 15) == 0)) {
#pragma unroll
            for (int h = 0; h < RW_ITEMS / 4; ++h) {
                const int4 q = __ldcs(reinterpret_cast<const int4 *>(irp + i0) + h);
                p[4 * h] = q.x; p[4 * h + 1] = q.y; p[4 * h + 2] = q.z; p[4 * h + 3] = q.w;
            }
            p[RW_ITEMS] = irp[i0 + RW_ITEMS];
        } else {
#pragma unroll
            for (int j = 0; j <= RW_ITEMS; ++j) p[j] = (i0 + j <= n) ? irp[i0 + j] : 0;
        }
#pragma unroll
        for (int j = 0; j < RW_ITEMS; ++j) {
            const long long i = i0 + j;
            if (i < n) {
                const int len = p[j + 1] - p[j];
                if (len < 0 || p[j] < 0 || (long long)p[j + 1] > nnz) bad = 1;
                if (i == 0 && p[0] != 0) bad = 1;
                if (i == n - 1 && (long long)p[j + 1] != nnz) bad = 1;
                mx = max(mx, len);
            }
        }
    }
    mx = (int)__reduce_max_sync(0xffffffffu, (unsigned)max(mx, 0));
    bad = (int)__reduce_or_sync(0xffffffffu, (unsigned)bad);
    if (lane_id() == 0) {
        s_mx[threadIdx.x >> 5] = mx;
        s_bad[threadIdx.x >> 5] = bad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < AN_THREADS / 32; ++w) {
            mx = max(mx, s_mx[w]);
            bad |= s_bad[w];
        }
        if (mx > 0) atomicMax(&acc->max_len, mx);
        if (bad) atomicOr(&acc->status, ST_BAD_PTR);
    }
}

cudaError_t launch_row_width(const int32_t *irp, int32_t n_rows, int64_t nnz, AnalyzeAcc *acc, cudaStream_t s) {
    if (n_rows <= 0) return cudaSuccess;
    unsigned grid = ceil_div_u(n_rows, (long long)AN_THREADS * RW_ITEMS);
    if (grid > (unsigned)sm_count() * RW_CTAS_PER_SM) grid = (unsigned)sm_count() * RW_CTAS_PER_SM;
    KernelScope ks("row_width", s);
    k_row_width<<<grid, AN_THREADS, 0, s>>>(irp, n_rows, nnz, acc);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- validate
__global__ void __launch_bounds__(256) k_validate_idx(const int32_t *__restrict__ idx, int64_t n, int32_t bound,
                                                       int *status) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    int bad = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        bad |= (unsigned)__ldcs(idx + i) >= (unsigned)bound;
    if (__any_sync(0xffffffffu, bad) && lane_id() == 0) atomicOr(status, ST_BAD_INDEX);
}

cudaError_t launch_validate_idx(const int32_t *idx, int64_t n, int32_t bound, int *status, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    unsigned grid = ceil_div_u(n, 256);
    unsigned cap = (unsigned)sm_count() * 8u;
    if (grid > cap) grid = cap;
    KernelScope ks("validate_idx", s);
    k_validate_idx<<<grid, 256, 0, s>>>(idx, n, bound, status);
    return cudaGetLastError();
}

// ------------------------------------------------------------- tile lines
// out[t] = the line holding entry t*tile (the largest i with ptr[i] <= t*tile,
// which is the non-empty line containing that entry). One thread per line
// writes the tiles whose first entry falls inside it: one coalesced pass over
// ptr instead of a binary search per tile.
__global__ void __launch_bounds__(256) k_tile_lines(const int32_t *__restrict__ ptr, int32_t n_lines, int shift,
                                                     long long n_tiles, int32_t *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_lines) return;
    const int a = max(__ldg(ptr + i), 0), b = __ldg(ptr + i + 1);
    const unsigned tile = 1u << shift;
    for (unsigned t = ((unsigned)a + tile - 1u) >> shift; (long long)t << shift < (long long)b && t < n_tiles; ++t)
        out[t] = i;
}

size_t tile_lines_bytes(int64_t nnz, int tile) { return (size_t)((nnz + tile - 1) / tile + 1) * 4; }

cudaError_t launch_tile_lines(const int32_t *ptr, int32_t n_lines, int64_t nnz, int tile, int32_t *out,
                              cudaStream_t s) {
    const long long n_tiles = (nnz + tile - 1) / tile;
    if (n_tiles <= 0) return cudaSuccess;
    // zero first: with a malformed ptr some tiles would get no writer, and
    // every consumer indexes ptr with these values
    cudaError_t e = cudaMemsetAsync(out, 0, (size_t)n_tiles * sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    int shift = 0;
    while ((1 << shift) < tile) ++shift;
    if ((1 << shift) != tile) return cudaErrorInvalidValue;  // tiles are powers of two
    KernelScope ks("tile_lines", s);
    k_tile_lines<<<ceil_div_u(n_lines, 256), 256, 0, s>>>(ptr, n_lines, shift, n_tiles, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ expand
// Each warp expands the entries of 32·G consecutive lines [L0, L0 + 32G)
// (lane l holds lines L0 + lG .. L0 + lG + G - 1): one coalesced load of their
// pointers, then the warp's entry range [ptr[L0], ptr[L0 + 32G]) in passes of
// EXP_TILE = 256 entries (8 per lane). The line of entry k is the largest
// line i with ptr[i] <= k, i.e. the non-empty line holding k; lines grow with
// their starts, so within a pass it is the last line whose start lies at or
// before k, else the line of the pass's previous entry (the carry). In a
// pass every non-empty line starting inside it writes its offset i - L0
// (one byte) at its first entry in the warp's part of shared memory; a lane
// reads its 8 slots in one 8-byte load and takes running maxima from the
// carry on. Marks of earlier passes are never cleared: they hold lines at or
// below the carry, so the maxima absorb them. A lane whose slots hold a line
// above the carry is marked (ballot); the line before a lane's first slot is
// the running maximum of the last marked lane below it (one shuffle), and
// the next carry is lane 31's maximum. Passes start at the range's first
// entry rounded down to a multiple of 8, so a lane's 8 entries leave in one
// 32-byte streaming store (whole sectors per warp instruction); entries of
// neighbouring warps in a pass's first and last group are left to them. No
// global load after the pointers, no search, no CTA barrier; shared memory
// moves a byte per entry. G (1..8, so offsets fit a byte) is picked on the
// host so that a warp's range spans four passes or more.
constexpr int EXP_THREADS = 128;
constexpr int EXP_WARPS = EXP_THREADS / 32;
constexpr int EXP_ITEMS = 8;
constexpr int EXP_TILE = 32 * EXP_ITEMS;

template <int G, bool VEC>
__global__ void __launch_bounds__(EXP_THREADS) k_expand(const int32_t *__restrict__ ptr, int32_t n_lines, int32_t nnz,
                                                         int32_t *__restrict__ out) {
    static_assert(32 * G <= 256, "line offsets within a warp fit a byte");
    __shared__ __align__(16) uint8_t s_mark[EXP_WARPS][EXP_TILE];
    const unsigned lane = lane_id();
    const long long l0 = ((long long)blockIdx.x * EXP_WARPS + (threadIdx.x >> 5)) * 32 * G;
    if (l0 >= n_lines) return;  // the whole warp: nothing below waits on other warps
    const long long lf = l0 + (long long)lane * G;  // this lane's first line
    const auto at = [&](long long i) { return min(max(__ldg(ptr + min(i, (long long)n_lines)), 0), nnz); };
    int st[G + 1];  // starts of the lane's lines, then the end of its last one
#pragma unroll
    for (int g = 0; g <= G; ++g) st[g] = at(lf + g);
    const int k_lo = __shfl_sync(0xffffffffu, st[0], 0);
    const int k_hi = __shfl_sync(0xffffffffu, st[G], 31);
    uint8_t *sm = s_mark[threadIdx.x >> 5];
    const int e = (int)lane * EXP_ITEMS;  // this lane's first entry within a pass
    *reinterpret_cast<uint2 *>(sm + e) = make_uint2(0u, 0u);  // offset 0: at or below every entry's line
    const unsigned below = (1u << lane) - 1u;
    int carry = 0;
    for (int b = k_lo & ~7; b < k_hi; b += EXP_TILE) {
        __syncwarp();  // the slots written below were read in the pass before
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const unsigned a = (unsigned)(st[g] - b);
            if (st[g + 1] > st[g] && a < (unsigned)EXP_TILE) sm[a] = (uint8_t)((int)lane * G + g);
        }
        __syncwarp();
        const uint2 w = *reinterpret_cast<const uint2 *>(sm + e);
        int v[EXP_ITEMS];
#pragma unroll
        for (int j = 0; j < EXP_ITEMS; ++j) v[j] = (int)(((j < 4 ? w.x : w.y) >> (8 * (j & 3))) & 0xffu);
        v[0] = max(v[0], carry);
#pragma unroll
        for (int j = 1; j < EXP_ITEMS; ++j) v[j] = max(v[j], v[j - 1]);
        const unsigned lt = __ballot_sync(0xffffffffu, v[EXP_ITEMS - 1] > carry) & below;
        const int x = __shfl_sync(0xffffffffu, v[EXP_ITEMS - 1], lt ? 31 - __clz(lt) : (int)lane);
        if (lt) {
#pragma unroll
            for (int j = 0; j < EXP_ITEMS; ++j) v[j] = max(v[j], x);
        }
        carry = __shfl_sync(0xffffffffu, v[EXP_ITEMS - 1], 31);
        const int k = b + e;
        const int base = (int)l0;
#pragma unroll
        for (int j = 0; j < EXP_ITEMS; ++j) v[j] += base;
        if (VEC && k >= k_lo && k + EXP_ITEMS <= k_hi) {
            st_cs_v8(out + k, v);
        } else {
#pragma unroll
            for (int j = 0; j < EXP_ITEMS; ++j)
                if (k + j >= k_lo && k + j < k_hi) __stcs(out + k + j, v[j]);
        }
    }
}

cudaError_t launch_expand(const int32_t *ptr, int32_t n_lines, int64_t nnz, int32_t *out, cudaStream_t s,
                          const char *name) {
    if (nnz <= 0 || n_lines <= 0) return cudaSuccess;
    if (nnz > INT_MAX) return cudaErrorInvalidValue;  // int32 pointers bound nnz
    // lines per lane: a warp's range should span about four passes or more
    const double mean = (double)nnz / (double)n_lines;
    int g = 1;
    while (g < 8 && 32.0 * g * mean < 4.0 * EXP_TILE) g <<= 1;
    const bool vec = (reinterpret_cast<uintptr_t>(out) & 31u) == 0;
    const long long per_cta = (long long)EXP_WARPS * 32 * g;
    const unsigned grid = (unsigned)((n_lines + per_cta - 1) / per_cta);
    KernelScope ks(name, s);
#define SPMVAT_EXPAND(G)                                                                                   \
    if (vec) k_expand<G, true><<<grid, EXP_THREADS, 0, s>>>(ptr, n_lines, (int32_t)nnz, out);              \
    else k_expand<G, false><<<grid, EXP_THREADS, 0, s>>>(ptr, n_lines, (int32_t)nnz, out);
    switch (g) {
    case 1: SPMVAT_EXPAND(1) break;
    case 2: SPMVAT_EXPAND(2) break;
    case 4: SPMVAT_EXPAND(4) break;
    default: SPMVAT_EXPAND(8) break;
    }
#undef SPMVAT_EXPAND
    return cudaGetLastError();
}

// ------------------------------------------------------------ lines -> ELL
// Persistent CTAs walk tiles of ELL_LINES consecutive lines through the
// two-stage TMA pipeline (stage_pipe.cuh): the tile's values and indices
// arrive in shared memory while the previous tile is written out. Slot k of
// line i goes to k*ld + i: for a fixed k a warp writes 32 consecutive lines
// (coalesced, streaming stores). SPLIT threads per line take slots
// part, part + SPLIT, ...: two for the build alone, four when the build also
// multiplies (the x gathers then need twice the warps in flight to hide
// their latency, and a 27-slot row is one batch of gathers per thread).
constexpr int ELL_LINES = 128;
constexpr int ELL_SPLIT_BUILD = 2;
constexpr int ELL_SPLIT_FUSED = 4;
constexpr int ELL_STAGE_CAP = 4096;  // entries per stage (48 KB)
constexpr int ELL_KB_BUILD = 6;      // slots a thread handles at once
constexpr int ELL_KB_FUSED = 4;      // (fused: two CTAs of 512 threads per SM leave 64 registers)
using EllPipe = StagePipe<ELL_STAGE_CAP, 1>;

template <bool FUSED, int ELL_SPLIT>
__global__ void __launch_bounds__(ELL_LINES *ELL_SPLIT, FUSED ? 2 : 4) k_lines_to_ell(
    const int32_t *__restrict__ ptr, const int32_t *__restrict__ idx, const double *__restrict__ val,
    int32_t n_lines, int32_t idx_bound, int32_t width, int32_t ld, int32_t n_tiles, int can_stage,
    double *__restrict__ eval, int32_t *__restrict__ eidx, const double *__restrict__ x, double *__restrict__ y,
    int *status) {
    constexpr int ELL_KB = FUSED ? ELL_KB_FUSED : ELL_KB_BUILD;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ double s_acc[(ELL_SPLIT - 1) * ELL_LINES];
    EllPipe P;
    P.setup(smem);
    const int lt = threadIdx.x % ELL_LINES;
    const int part = threadIdx.x / ELL_LINES;
    int bad = 0;
    auto range = [&](int tile, long long *e0, long long *e1) {
        const long long l0 = (long long)tile * ELL_LINES;
        if (l0 >= n_lines) { *e0 = *e1 = 0; return; }
        const long long l1 = min(l0 + (long long)ELL_LINES, (long long)n_lines);
        *e0 = ptr[l0];
        *e1 = ptr[l1];
    };
    // this thread's line pointers, loaded a tile ahead
    auto pre = [&](int tile) {
        const long long l = (long long)tile * ELL_LINES + lt;
        return (l < n_lines) ? make_int2(ptr[l], ptr[l + 1]) : make_int2(0, 0);
    };
    auto body = [&](int tile, int st, const StageMeta &m, int2 se) {
        const long long l = (long long)tile * ELL_LINES + lt;
        double acc = 0.0;
        if (l < ld) {
            if (l < n_lines) {
                const long long s = se.x, e = se.y;
                int len = (int)(e - s);
                if (len < 0 || len > width) { bad = 1; len = len < 0 ? 0 : width; }
                int last = len > 0 ? P.idx_at(m, st, idx, s + len - 1) : 0;
                if ((unsigned)last >= (unsigned)idx_bound) { bad = 1; last = 0; }
                // slots in batches of ELL_KB per thread: every value, index
                // and x gather of a batch is issued before its first use
                for (int k0 = part; k0 < width; k0 += ELL_SPLIT * ELL_KB) {
                    double v[ELL_KB];
                    int32_t c[ELL_KB];
#pragma unroll
                    for (int u = 0; u < ELL_KB; ++u) {
                        const int k = k0 + u * ELL_SPLIT;
                        v[u] = 0.0;
                        c[u] = last;
                        if (k < len) {
                            v[u] = P.val_at(m, st, val, s + k);
                            c[u] = P.idx_at(m, st, idx, s + k);
                            if ((unsigned)c[u] >= (unsigned)idx_bound) { bad = 1; c[u] = 0; }
                        }
                    }
                    double xv[ELL_KB];
                    if (FUSED) {
#pragma unroll
                        for (int u = 0; u < ELL_KB; ++u) xv[u] = (k0 + u * ELL_SPLIT < len) ? __ldg(x + c[u]) : 0.0;
                    }
#pragma unroll
                    for (int u = 0; u < ELL_KB; ++u) {
                        const int k = k0 + u * ELL_SPLIT;
                        if (k < width) {
                            __stcs(eval + (long long)k * ld + l, v[u]);
                            __stcs(eidx + (long long)k * ld + l, c[u]);
                        }
                    }
                    if (FUSED) {
#pragma unroll
                        for (int u = 0; u < ELL_KB; ++u)
                            if (k0 + u * ELL_SPLIT < len) acc = fma(v[u], xv[u], acc);
                    }
                }
            } else {
                for (int k = part; k < width; k += ELL_SPLIT) {
                    __stcs(eval + (long long)k * ld + l, 0.0);
                    __stcs(eidx + (long long)k * ld + l, 0);
                }
            }
        }
        if (FUSED) {
            if (part > 0) s_acc[(part - 1) * ELL_LINES + lt] = acc;
            __syncthreads();
            if (part == 0 && l < n_lines) {
#pragma unroll
                for (int q = 1; q < ELL_SPLIT; ++q) acc += s_acc[(q - 1) * ELL_LINES + lt];
                y[l] = acc;
            }
        }
    };
    pipe_tiles(P, n_tiles, val, idx, can_stage != 0, status, range, pre, body);
    if (bad) atomicOr(status, ST_BAD_INDEX);
}

cudaError_t launch_lines_to_ell(const int32_t *ptr, const int32_t *idx, const double *val, int32_t n_lines,
                                int32_t idx_bound, int32_t width, int32_t ld, double *eval, int32_t *eidx,
                                const double *x, double *y, int *status, cudaStream_t s, const char *name) {
    if (ld <= 0 || width <= 0) return cudaSuccess;
    const int n_tiles = (int)ceil_div_u(ld, ELL_LINES);
    const int can_stage = ((reinterpret_cast<uintptr_t>(val) & 15) == 0) &&
                          ((reinterpret_cast<uintptr_t>(idx) & 15) == 0);
    const bool fused = (y != nullptr);
    cudaError_t e = fused ? set_smem_attr(k_lines_to_ell<true, ELL_SPLIT_FUSED>, EllPipe::kSmem)
                          : set_smem_attr(k_lines_to_ell<false, ELL_SPLIT_BUILD>, EllPipe::kSmem);
    if (e != cudaSuccess) return e;
    int grid = sm_count() * 2;
    if (grid > n_tiles) grid = n_tiles;
    if (fused) {
        KernelScope ks("crs_to_ell_row_fused_spmv", s);
        k_lines_to_ell<true, ELL_SPLIT_FUSED><<<grid, ELL_LINES * ELL_SPLIT_FUSED, EllPipe::kSmem, s>>>(
            ptr, idx, val, n_lines, idx_bound, width, ld, n_tiles, can_stage, eval, eidx, x, y, status);
    } else {
        KernelScope ks(name, s);
        k_lines_to_ell<false, ELL_SPLIT_BUILD><<<grid, ELL_LINES * ELL_SPLIT_BUILD, EllPipe::kSmem, s>>>(
            ptr, idx, val, n_lines, idx_bound, width, ld, n_tiles, can_stage, eval, eidx, nullptr, nullptr, status);
    }
    return cudaGetLastError();
}

}  // namespace spmvat
