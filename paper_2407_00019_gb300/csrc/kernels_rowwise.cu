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

namespace spmvat {

// ---------------------------------------------------------------- analyze
constexpr int AN_THREADS = 256;

__global__ void __launch_bounds__(AN_THREADS) k_analyze(const int32_t *__restrict__ irp, int32_t n, int64_t nnz,
                                                         AnalyzeAcc *acc) {
    __shared__ unsigned long long s_hist[32];
    __shared__ unsigned long long s_sum[AN_THREADS / 32][3];
    __shared__ int s_mm[AN_THREADS / 32][3];
    if (threadIdx.x < 32) s_hist[threadIdx.x] = 0ull;
    __syncthreads();
    unsigned long long sl = 0, sl2 = 0, ne = 0;
    int mx = 0, inv_mn = 0, bad = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        int a = irp[i], b = irp[i + 1];
        int len = b - a;
        if (len < 0 || a < 0 || (long long)b > nnz) { bad = 1; len = len < 0 ? 0 : len; }
        if (i == 0 && a != 0) bad = 1;
        if (i == n - 1 && (long long)b != nnz) bad = 1;
        sl += (unsigned)len;
        sl2 += (unsigned long long)len * (unsigned long long)len;
        ne += (len == 0);
        mx = max(mx, len);
        inv_mn = max(inv_mn, INT_MAX - len);
        int cls = (len == 0) ? 0 : 32 - __clz(len);
        unsigned act = __activemask();
        unsigned peers = __match_any_sync(act, cls);
        if ((lanemask_lt() & peers) == 0) atomicAdd(&s_hist[cls], (unsigned long long)__popc(peers));
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
    unsigned grid = ceil_div_u(n_rows, AN_THREADS);
    unsigned cap = (unsigned)sm_count() * 8u;
    if (grid > cap) grid = cap;
    if (grid == 0) grid = 1;
    KernelScope ks("analyze", s);
    k_analyze<<<grid, AN_THREADS, 0, s>>>(irp, n_rows, nnz, acc);
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

// ------------------------------------------------------------------ expand
// Tile of EXP_TILE consecutive entries; each thread writes EXP_ITEMS of them
// with one 16-byte store. The pointers of the lines that cover the tile are
// staged in shared memory when they fit, and each thread finds its first
// line by binary search there, then walks forward.
constexpr int EXP_THREADS = 256;
constexpr int EXP_ITEMS = 4;
constexpr int EXP_TILE = EXP_THREADS * EXP_ITEMS;
constexpr int EXP_WIN = 2048;

__global__ void __launch_bounds__(EXP_THREADS) k_expand(const int32_t *__restrict__ ptr, int32_t n_lines, int64_t nnz,
                                                         int32_t *__restrict__ out) {
    __shared__ int32_t s_ptr[EXP_WIN];
    __shared__ int s_lo, s_hi;
    const long long k0 = (long long)blockIdx.x * EXP_TILE;
    const long long k1 = min(k0 + (long long)EXP_TILE, (long long)nnz);
    if (threadIdx.x == 0) {
        int lo = last_le(ptr, 0, n_lines, k0);
        s_lo = lo;
        s_hi = last_le(ptr, lo, n_lines, k1 - 1);
    }
    __syncthreads();
    const int lo = s_lo, hi = s_hi;
    const int wn = hi - lo + 2;  // ptr[lo .. hi+1]
    const bool sm = wn <= EXP_WIN;
    if (sm)
        for (int i = threadIdx.x; i < wn; i += EXP_THREADS) s_ptr[i] = ptr[lo + i];
    __syncthreads();
    const long long k = k0 + (long long)threadIdx.x * EXP_ITEMS;
    if (k >= k1) return;
    int line = sm ? lo + last_le(s_ptr, 0, wn - 1, k) : last_le(ptr, lo, hi + 1, k);
    int v[EXP_ITEMS];
#pragma unroll
    for (int j = 0; j < EXP_ITEMS; ++j) {
        const long long kk = k + j;
        if (kk < k1) {
            while (line < hi && (long long)(sm ? s_ptr[line + 1 - lo] : ptr[line + 1]) <= kk) ++line;
        }
        v[j] = line;
    }
    if (k + EXP_ITEMS <= k1 && ((reinterpret_cast<uintptr_t>(out + k) & 15) == 0)) {
        *reinterpret_cast<int4 *>(out + k) = make_int4(v[0], v[1], v[2], v[3]);
    } else {
#pragma unroll
        for (int j = 0; j < EXP_ITEMS; ++j)
            if (k + j < k1) out[k + j] = v[j];
    }
}

cudaError_t launch_expand(const int32_t *ptr, int32_t n_lines, int64_t nnz, int32_t *out, cudaStream_t s,
                          const char *name) {
    if (nnz <= 0) return cudaSuccess;
    KernelScope ks(name, s);
    k_expand<<<ceil_div_u(nnz, EXP_TILE), EXP_THREADS, 0, s>>>(ptr, n_lines, nnz, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------ lines -> ELL
// Persistent CTAs walk tiles of ELL_LINES consecutive lines. For each tile
// one thread issues two TMA bulk copies (values and indices of the tile's
// entries, the 16-byte-aligned interior of the range) into one of two shared
// stages, so the copy of tile t+grid overlaps the write-out of tile t. The
// write-out stores slot k of line i at k*ld + i: for a fixed k a warp writes
// 32 consecutive lines (fully coalesced). Entries outside the staged interior
// (at most one value and three indices per tile edge), and whole tiles whose
// entries exceed a stage, are read from global memory instead.
constexpr int ELL_LINES = 128;
constexpr int ELL_SPLIT = 2;  // threads per line (they take alternate slots)
constexpr int ELL_THREADS = ELL_LINES * ELL_SPLIT;
constexpr int ELL_STAGE_CAP = 4096;  // entries per stage (48 KB)
constexpr size_t ELL_SMEM = 128 + 2 * (size_t)ELL_STAGE_CAP * 12;

struct EllMeta {
    long long a0v, b0v, a0i, b0i;
    int staged;
    int pad;
};

template <bool FUSED>
__global__ void __launch_bounds__(ELL_THREADS) k_lines_to_ell(
    const int32_t *__restrict__ ptr, const int32_t *__restrict__ idx, const double *__restrict__ val,
    int32_t n_lines, int32_t idx_bound, int32_t width, int32_t ld, int32_t n_tiles, int can_stage,
    double *__restrict__ eval, int32_t *__restrict__ eidx, const double *__restrict__ x, double *__restrict__ y,
    int *status) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    EllMeta *meta = reinterpret_cast<EllMeta *>(smem + 16);
    double *sval0 = reinterpret_cast<double *>(smem + 128);
    int32_t *sidx0 = reinterpret_cast<int32_t *>(smem + 128 + (size_t)ELL_STAGE_CAP * 8);
    double *sval1 = reinterpret_cast<double *>(smem + 128 + (size_t)ELL_STAGE_CAP * 12);
    int32_t *sidx1 = reinterpret_cast<int32_t *>(smem + 128 + (size_t)ELL_STAGE_CAP * 20);
    __shared__ double s_acc[ELL_LINES];

    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();

    auto issue = [&](int tile, int st) {
        const long long l0 = (long long)tile * ELL_LINES;
        EllMeta m;
        long long e0 = 0, e1 = 0;
        if (l0 < n_lines) {
            const long long l1 = min(l0 + (long long)ELL_LINES, (long long)n_lines);
            e0 = ptr[l0];
            e1 = ptr[l1];
            if (e1 < e0) e1 = e0;
        }
        m.a0v = e0 & ~1ll;
        m.b0v = max(m.a0v, e1 & ~1ll);
        m.a0i = e0 & ~3ll;
        m.b0i = max(m.a0i, e1 & ~3ll);
        const unsigned bv = (unsigned)((m.b0v - m.a0v) * 8), bi = (unsigned)((m.b0i - m.a0i) * 4);
        m.staged = can_stage && (m.b0v - m.a0v) <= ELL_STAGE_CAP && (m.b0i - m.a0i) <= ELL_STAGE_CAP &&
                   (bv + bi) > 0;
        m.pad = 0;
        meta[st] = m;
        if (m.staged) {
            mbar_arrive_expect_tx(&bar[st], bv + bi);
            if (bv) bulk_g2s(st ? (void *)sval1 : (void *)sval0, val + m.a0v, bv, &bar[st]);
            if (bi) bulk_g2s(st ? (void *)sidx1 : (void *)sidx0, idx + m.a0i, bi, &bar[st]);
        } else {
            mbar_arrive_expect_tx(&bar[st], 0);
        }
    };

    int it = 0;
    if (threadIdx.x == 0 && (int)blockIdx.x < n_tiles) issue(blockIdx.x, 0);
    const int lt = threadIdx.x % ELL_LINES;
    const int part = threadIdx.x / ELL_LINES;
    int bad = 0;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++it) {
        const int st = it & 1;
        const int next = tile + gridDim.x;
        if (threadIdx.x == 0 && next < n_tiles) issue(next, st ^ 1);
        const bool ok = mbar_wait_bounded(&bar[st], (unsigned)((it >> 1) & 1), kSpinLimit);
        if (__syncthreads_or(!ok)) {
            // Give up, but do not leave a copy in flight into the shared
            // memory of an exiting CTA: wait (bounded) for both stages.
            if (threadIdx.x == 0) {
                atomicOr(status, ST_TIMEOUT);
                mbar_wait_bounded(&bar[st], (unsigned)((it >> 1) & 1), kSpinLimit);
                if (next < n_tiles) mbar_wait_bounded(&bar[st ^ 1], (unsigned)(((it + 1) >> 1) & 1), kSpinLimit);
            }
            break;
        }
        const EllMeta m = meta[st];
        const double *sv = st ? sval1 : sval0;
        const int32_t *si = st ? sidx1 : sidx0;
        auto VAL = [&](long long k) -> double {
            return (m.staged && k >= m.a0v && k < m.b0v) ? sv[k - m.a0v] : val[k];
        };
        auto IDX = [&](long long k) -> int32_t {
            return (m.staged && k >= m.a0i && k < m.b0i) ? si[k - m.a0i] : idx[k];
        };
        const long long l = (long long)tile * ELL_LINES + lt;
        double acc = 0.0;
        if (l < ld) {
            if (l < n_lines) {
                const long long s = ptr[l], e = ptr[l + 1];
                int len = (int)(e - s);
                if (len < 0 || len > width) { bad = 1; len = len < 0 ? 0 : width; }
                int last = len > 0 ? IDX(s + len - 1) : 0;
                if ((unsigned)last >= (unsigned)idx_bound) { bad = 1; last = 0; }
                for (int k = part; k < width; k += ELL_SPLIT) {
                    double v;
                    int32_t c;
                    if (k < len) {
                        v = VAL(s + k);
                        c = IDX(s + k);
                        if ((unsigned)c >= (unsigned)idx_bound) { bad = 1; c = 0; }
                        if (FUSED) acc = fma(v, __ldg(x + c), acc);
                    } else {
                        v = 0.0;
                        c = last;
                    }
                    __stcs(eval + (long long)k * ld + l, v);
                    __stcs(eidx + (long long)k * ld + l, c);
                }
            } else {
                for (int k = part; k < width; k += ELL_SPLIT) {
                    __stcs(eval + (long long)k * ld + l, 0.0);
                    __stcs(eidx + (long long)k * ld + l, 0);
                }
            }
        }
        if (FUSED) {
            if (part == 1) s_acc[lt] = acc;
            __syncthreads();
            if (part == 0 && l < n_lines) y[l] = acc + s_acc[lt];
        }
        __syncthreads();
    }
    if (bad) atomicOr(status, ST_BAD_INDEX);
}

cudaError_t launch_lines_to_ell(const int32_t *ptr, const int32_t *idx, const double *val, int32_t n_lines,
                                int32_t idx_bound, int32_t width, int32_t ld, double *eval, int32_t *eidx,
                                const double *x, double *y, int *status, cudaStream_t s, const char *name) {
    if (ld <= 0 || width <= 0) return cudaSuccess;
    const int n_tiles = (int)ceil_div_u(ld, ELL_LINES);
    const int can_stage = ((reinterpret_cast<uintptr_t>(val) & 15) == 0) &&
                          ((reinterpret_cast<uintptr_t>(idx) & 15) == 0);
    static bool attr_set[64][2];
    int dev = 0;
    cudaGetDevice(&dev);
    dev &= 63;
    const bool fused = (y != nullptr);
    if (!attr_set[dev][fused]) {
        cudaError_t e = fused ? cudaFuncSetAttribute(k_lines_to_ell<true>,
                                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ELL_SMEM)
                              : cudaFuncSetAttribute(k_lines_to_ell<false>,
                                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ELL_SMEM);
        if (e != cudaSuccess) return e;
        attr_set[dev][fused] = true;
    }
    int grid = sm_count() * 2;
    if (grid > n_tiles) grid = n_tiles;
    if (fused) {
        KernelScope ks("crs_to_ell_row_fused_spmv", s);
        k_lines_to_ell<true><<<grid, ELL_THREADS, ELL_SMEM, s>>>(ptr, idx, val, n_lines, idx_bound, width, ld,
                                                                 n_tiles, can_stage, eval, eidx, x, y, status);
    } else {
        KernelScope ks(name, s);
        k_lines_to_ell<false><<<grid, ELL_THREADS, ELL_SMEM, s>>>(ptr, idx, val, n_lines, idx_bound, width, ld,
                                                                  n_tiles, can_stage, eval, eidx, nullptr,
                                                                  nullptr, status);
    }
    return cudaGetLastError();
}

}  // namespace spmvat
