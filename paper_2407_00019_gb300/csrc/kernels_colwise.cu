// Phase I of Sec. 2.1 (CRS -> CCS) on the GPU.
//
// The paper's serial Phase I counts the entries of every column, turns the
// counts into column pointers with a running sum, and then walks the CRS in
// row order, dropping each entry at its column's cursor. The result lists
// each column's rows in ascending order (repeated (i, j) entries in CRS
// order). Here:
//   k_col_count   : NC[j] by one atomicAdd per entry (warp aggregation with
//                   __match_any_sync was measured slower: on banded matrices a
//                   warp rarely holds two entries of one column, and the match
//                   instruction saturates the MIO pipe). Each entry also keeps
//                   the value its column's counter had when it was counted
//                   (its "rank"), in arbitrary order.
//   k_scan        : NC -> IRP_T in place, one pass with decoupled look-back
//                   (Merrill & Garland, 2016). Every spin is bounded; on
//                   expiry the tile publishes an error flag that ends its
//                   successors' waits, and the call reports SPMV_ERR_TIMEOUT.
//   k_col_scatter : entry k goes to IRP_T[col] + rank[k] as the pair
//                   (k, row), a permutation with no further atomics.
//   k_fixup_*     : each column's pairs are put in ascending k (= the serial
//                   order: CRS position order is row order), then
//                   ICOL_T = row and VAL_T = VAL[k] are written contiguously.
//                   Columns of <= 32 entries: one warp, bitonic network in
//                   registers. Longer: one CTA, bitonic sort in shared memory
//                   (<= 4096) or sorted chunks + merge-path merges.
// The default path for columns with >= 8 entries on average carries (row,
// value) instead of (k, row) and sorts each column by row in registers; see
// "row-value slot path" below.
#include <climits>

#include "common.cuh"

namespace spmvat {

// ------------------------------------------------------------------- count
// Thread-striped tiles: item u of thread t is entry k0 + u*256 + t, so one
// instruction of a warp covers 32 consecutive entries and the CTA issues its
// atomics in (nearly) ascending k. Ranks then mostly come out in the serial
// order and the fix-up rarely has to sort.
constexpr int CNT_THREADS = 256;
constexpr int CNT_ITEMS = 8;
constexpr int CNT_TILE = CNT_THREADS * CNT_ITEMS;

__global__ void __launch_bounds__(CNT_THREADS) k_col_count(const int32_t *__restrict__ icol, int64_t nnz,
                                                            int32_t n_cols, int32_t *__restrict__ nc,
                                                            int32_t *__restrict__ rank, int *status) {
    const long long k0 = (long long)blockIdx.x * CNT_TILE + threadIdx.x;
    int c[CNT_ITEMS];
#pragma unroll
    for (int u = 0; u < CNT_ITEMS; ++u) {
        const long long k = k0 + (long long)u * CNT_THREADS;
        c[u] = (k < nnz) ? __ldcs(icol + k) : -1;
    }
    int bad = 0;
#pragma unroll
    for (int u = 0; u < CNT_ITEMS; ++u) {
        const long long k = k0 + (long long)u * CNT_THREADS;
        const bool valid = (k < nnz) && (unsigned)c[u] < (unsigned)n_cols;
        bad |= (k < nnz) && !valid;
        const int r = valid ? atomicAdd(nc + c[u], 1) : 0;
        if (k < nnz) __stcs(rank + k, r);
    }
    if (__any_sync(0xffffffffu, bad) && lane_id() == 0) atomicOr(status, ST_BAD_INDEX);
}

cudaError_t launch_col_count(const int32_t *icol, int64_t nnz, int32_t n_cols, int32_t *nc, int32_t *rank,
                             int *status, cudaStream_t s) {
    if (nnz <= 0) return cudaSuccess;
    KernelScope ks("col_count", s);
    k_col_count<<<ceil_div_u(nnz, CNT_TILE), CNT_THREADS, 0, s>>>(icol, nnz, n_cols, nc, rank, status);
    return cudaGetLastError();
}

// -------------------------------------------------------------------- scan
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;
constexpr unsigned long long FLAG_NONE = 0ull;
constexpr unsigned long long FLAG_AGG = 1ull << 62;
constexpr unsigned long long FLAG_PRE = 2ull << 62;
constexpr unsigned long long FLAG_ERR = 3ull << 62;
constexpr unsigned long long VALUE_MASK = (1ull << 62) - 1;

size_t scan_scratch_bytes(int64_t n) {
    const long long tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    return 16 + (size_t)(tiles > 0 ? tiles : 1) * sizeof(unsigned long long);
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan(int32_t *a, int64_t n, unsigned *ticket,
                                                        unsigned long long *tile_status, int32_t *maxv,
                                                        int32_t long_thresh, int32_t *long_list,
                                                        int32_t *long_count, int *status, long long spin_limit,
                                                        int stall_first) {
    __shared__ int s_tile;
    __shared__ long long s_warp[SCAN_THREADS / 32];
    __shared__ int s_wmax[SCAN_THREADS / 32];
    __shared__ long long s_excl;
    __shared__ int s_abort;
    if (threadIdx.x == 0) {
        s_tile = (int)atomicAdd(ticket, 1u);  // tiles start in ticket order
        s_abort = 0;
    }
    __syncthreads();
    const int tile = s_tile;
    const long long base = (long long)tile * SCAN_TILE + (long long)threadIdx.x * SCAN_ITEMS;
    int v[SCAN_ITEMS];
    long long sum = 0;
    int mx = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        const long long i = base + j;
        v[j] = (i < n) ? a[i] : 0;
        sum += v[j];
        mx = max(mx, v[j]);
        if (long_list && i < n && v[j] > long_thresh) long_list[atomicAdd(long_count, 1)] = (int32_t)i;
    }
    // block-wide exclusive scan of the per-thread sums
    const unsigned lane = lane_id();
    const int w = threadIdx.x >> 5;
    long long inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long t = __shfl_up_sync(0xffffffffu, inc, o);
        if ((int)lane >= o) inc += t;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 31) s_warp[w] = inc;
    if (lane == 0) s_wmax[w] = mx;
    __syncthreads();
    long long warp_off = 0, total = 0;
    int bmax = 0;
    for (int j = 0; j < SCAN_THREADS / 32; ++j) {
        if (j < w) warp_off += s_warp[j];
        total += s_warp[j];
        bmax = max(bmax, s_wmax[j]);
    }
    const long long thread_excl = warp_off + inc - sum;
    if (threadIdx.x == 0) {
        if (maxv) atomicMax(maxv, bmax);
        if (tile == 0) {
            if (!stall_first) st_release_u64(&tile_status[0], FLAG_PRE | (unsigned long long)total);
            s_excl = 0;
        } else {
            st_release_u64(&tile_status[tile], FLAG_AGG | (unsigned long long)total);
        }
    }
    if (tile > 0 && w == 0) {
        long long excl = 0;
        long long pred = tile - 1;
        long long spins = 0;
        bool fail = false;
        while (true) {
            const long long idx = pred - (long long)lane;
            const unsigned long long st = (idx >= 0) ? ld_acquire_u64(&tile_status[idx]) : FLAG_PRE;
            const unsigned long long flag = st & ~VALUE_MASK;
            if (__ballot_sync(0xffffffffu, flag == FLAG_ERR)) { fail = true; break; }
            const unsigned pre = __ballot_sync(0xffffffffu, flag == FLAG_PRE);
            const unsigned none = __ballot_sync(0xffffffffu, flag == FLAG_NONE);
            const int first_pre = pre ? __ffs(pre) - 1 : 32;
            const unsigned window = (first_pre >= 31) ? 0xffffffffu : ((1u << (first_pre + 1)) - 1u);
            if (none & window) {
                if (++spins > spin_limit) { fail = true; break; }
                __nanosleep(spins < 64 ? 32 : 1000);
                continue;
            }
            long long contrib = ((int)lane <= first_pre) ? (long long)(st & VALUE_MASK) : 0;
            excl += warp_sum(contrib);
            if (first_pre < 32) break;
            pred -= 32;
        }
        if (lane == 0) {
            if (fail) {
                st_release_u64(&tile_status[tile], FLAG_ERR);
                atomicOr(status, ST_TIMEOUT);
                s_abort = 1;
            } else {
                st_release_u64(&tile_status[tile], FLAG_PRE | (unsigned long long)(excl + total));
                s_excl = excl;
            }
        }
    }
    __syncthreads();
    if (s_abort) return;
    long long run = s_excl + thread_excl;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        const long long i = base + j;
        if (i < n) a[i] = (int32_t)run;
        run += v[j];
        if (i == n - 1) a[n] = (int32_t)run;
    }
}

cudaError_t launch_scan(int32_t *a, int64_t n, void *scratch, int32_t *maxv, int32_t long_thresh,
                        int32_t *long_list, int32_t *long_count, int *status, long long spin_limit,
                        int debug_stall_first, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const long long tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    cudaError_t e = cudaMemsetAsync(scratch, 0, scan_scratch_bytes(n), s);
    if (e != cudaSuccess) return e;
    unsigned *ticket = reinterpret_cast<unsigned *>(scratch);
    unsigned long long *tstat = reinterpret_cast<unsigned long long *>(reinterpret_cast<char *>(scratch) + 16);
    KernelScope ks("scan_lookback", s);
    k_scan<<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(a, n, ticket, tstat, maxv, long_thresh, long_list, long_count,
                                                     status, spin_limit, debug_stall_first);
    return cudaGetLastError();
}

// ----------------------------------------------------------------- scatter
// Entry loads (ICOL, rank) are issued before the tile's row window is
// fetched, so the two round trips overlap.
constexpr int SCT_THREADS = 256;
constexpr int SCT_ITEMS = 8;
constexpr int SCT_TILE = SCT_THREADS * SCT_ITEMS;
constexpr int SCT_WIN = 2048;
constexpr int SLOT_CAP = 32;  // ranks kept in the slot-major array T

__global__ void __launch_bounds__(SCT_THREADS) k_col_scatter(const int32_t *__restrict__ irp, int32_t n_rows,
                                                              const int32_t *__restrict__ icol, int64_t nnz,
                                                              int32_t n_cols, const int32_t *__restrict__ cp,
                                                              const int32_t *__restrict__ rank,
                                                              const int32_t *__restrict__ tl, long long n_tiles,
                                                              int2 *__restrict__ pairs, int *status, int min_rank,
                                                              const int32_t *__restrict__ only_if) {
    __shared__ int32_t s_ptr[SCT_WIN];
    if (only_if && *only_if == 0) return;  // nothing to place: the whole grid returns at once
    const long long k0 = (long long)blockIdx.x * SCT_TILE;
    const long long k1 = min(k0 + (long long)SCT_TILE, (long long)nnz);
    const long long k = k0 + (long long)threadIdx.x * SCT_ITEMS;
    int c[SCT_ITEMS], r[SCT_ITEMS];
    if (k + SCT_ITEMS <= k1 && ((reinterpret_cast<uintptr_t>(icol + k) & 15) == 0) &&
        ((reinterpret_cast<uintptr_t>(rank + k) & 15) == 0)) {
#pragma unroll
        for (int h = 0; h < SCT_ITEMS / 4; ++h) {
            const int4 q = __ldcs(reinterpret_cast<const int4 *>(icol + k) + h);
            const int4 p = __ldcs(reinterpret_cast<const int4 *>(rank + k) + h);
            c[4 * h] = q.x; c[4 * h + 1] = q.y; c[4 * h + 2] = q.z; c[4 * h + 3] = q.w;
            r[4 * h] = p.x; r[4 * h + 1] = p.y; r[4 * h + 2] = p.z; r[4 * h + 3] = p.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < SCT_ITEMS; ++j) {
            c[j] = (k + j < k1) ? icol[k + j] : 0;
            r[j] = (k + j < k1) ? rank[k + j] : 0;
        }
    }
    long long pos[SCT_ITEMS];
    int bad = 0;
#pragma unroll
    for (int j = 0; j < SCT_ITEMS; ++j) {
        const bool ok = (k + j < k1) && (unsigned)c[j] < (unsigned)n_cols;
        bad |= (k + j < k1) && !ok;
        pos[j] = (ok && r[j] >= min_rank) ? (long long)__ldg(cp + c[j]) + r[j] : -1;
    }
    const int lo = tl[blockIdx.x];
    const int hi = (blockIdx.x + 1 < n_tiles) ? tl[blockIdx.x + 1] : n_rows - 1;
    const int wn = hi - lo + 2;
    const bool sm = wn <= SCT_WIN;
    if (sm)
        for (int i = threadIdx.x; i < wn; i += SCT_THREADS) s_ptr[i] = irp[lo + i];
    __syncthreads();
    if (k < k1) {
        int row = sm ? lo + last_le(s_ptr, 0, wn - 1, k) : last_le(irp, lo, hi + 1, k);
#pragma unroll
        for (int j = 0; j < SCT_ITEMS; ++j) {
            const long long kk = k + j;
            if (kk >= k1) break;
            while (row < hi && (long long)(sm ? s_ptr[row + 1 - lo] : irp[row + 1]) <= kk) ++row;
            if (pos[j] < 0) continue;
            if (pos[j] >= nnz) { bad = 1; continue; }
            pairs[pos[j]] = make_int2((int)kk, row);
        }
    }
    if (__any_sync(0xffffffffu, bad) && lane_id() == 0) atomicOr(status, ST_BAD_INDEX);
}

size_t col_scatter_scratch_bytes(int64_t nnz) { return tile_lines_bytes(nnz, SCT_TILE); }

cudaError_t launch_col_scatter(const int32_t *irp, int32_t n_rows, const int32_t *icol, int64_t nnz,
                               int32_t n_cols, const int32_t *cp, const int32_t *rank, int2 *pairs,
                               int32_t *scratch, int *status, cudaStream_t s, int min_rank,
                               const int32_t *only_if, bool have_tile_lines) {
    if (nnz <= 0) return cudaSuccess;
    if (!have_tile_lines) {
        cudaError_t e = launch_tile_lines(irp, n_rows, nnz, SCT_TILE, scratch, s);
        if (e != cudaSuccess) return e;
    }
    const long long n_tiles = (nnz + SCT_TILE - 1) / SCT_TILE;
    KernelScope ks(min_rank > 0 ? "col_overflow" : "col_scatter", s);
    k_col_scatter<<<(unsigned)n_tiles, SCT_THREADS, 0, s>>>(irp, n_rows, icol, nnz, n_cols, cp, rank, scratch,
                                                             n_tiles, pairs, status, min_rank, only_if);
    return cudaGetLastError();
}

// ------------------------------------------------------------------- claim
// Count and place in one pass (the slot path of Phase I). For entry k of row
// i in column j: r = atomicAdd(NC[j], 1) is its rank; when r < SLOT_CAP the
// pair (k, i) goes straight to T[r * n_cols + j], a slot-major array like an
// ELL over columns, so the fix-up can read a column tile with coalesced
// loads. Ranks are stored for every entry; entries with r >= SLOT_CAP are
// counted in *n_over and placed later by k_col_scatter (min_rank = SLOT_CAP).
__global__ void __launch_bounds__(SCT_THREADS) k_col_claim(const int32_t *__restrict__ irp, int32_t n_rows,
                                                            const int32_t *__restrict__ icol, int64_t nnz,
                                                            int32_t n_cols, int32_t *__restrict__ nc,
                                                            int32_t *__restrict__ rank,
                                                            const int32_t *__restrict__ tl, long long n_tiles,
                                                            int2 *__restrict__ T, int32_t *__restrict__ n_over,
                                                            int *status) {
    __shared__ int32_t s_ptr[SCT_WIN];
    const long long k0 = (long long)blockIdx.x * SCT_TILE;
    const long long k1 = min(k0 + (long long)SCT_TILE, (long long)nnz);
    const long long k = k0 + (long long)threadIdx.x * SCT_ITEMS;
    int c[SCT_ITEMS];
    if (k + SCT_ITEMS <= k1 && ((reinterpret_cast<uintptr_t>(icol + k) & 15) == 0)) {
#pragma unroll
        for (int h = 0; h < SCT_ITEMS / 4; ++h) {
            const int4 q = __ldcs(reinterpret_cast<const int4 *>(icol + k) + h);
            c[4 * h] = q.x; c[4 * h + 1] = q.y; c[4 * h + 2] = q.z; c[4 * h + 3] = q.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < SCT_ITEMS; ++j) c[j] = (k + j < k1) ? icol[k + j] : -1;
    }
    int r[SCT_ITEMS];
    int bad = 0, over = 0;
#pragma unroll
    for (int j = 0; j < SCT_ITEMS; ++j) {
        const bool has = k + j < k1;
        const bool ok = has && (unsigned)c[j] < (unsigned)n_cols;
        bad |= has && !ok;
        r[j] = ok ? atomicAdd(nc + c[j], 1) : -1;
    }
    const int lo = tl[blockIdx.x];
    const int hi = (blockIdx.x + 1 < n_tiles) ? tl[blockIdx.x + 1] : n_rows - 1;
    const int wn = hi - lo + 2;
    const bool sm = wn <= SCT_WIN;
    if (sm)
        for (int i = threadIdx.x; i < wn; i += SCT_THREADS) s_ptr[i] = irp[lo + i];
    __syncthreads();
    if (k < k1) {
        int row = sm ? lo + last_le(s_ptr, 0, wn - 1, k) : last_le(irp, lo, hi + 1, k);
#pragma unroll
        for (int j = 0; j < SCT_ITEMS; ++j) {
            const long long kk = k + j;
            if (kk >= k1) break;
            while (row < hi && (long long)(sm ? s_ptr[row + 1 - lo] : irp[row + 1]) <= kk) ++row;
            if (r[j] < 0) continue;
            if (r[j] < SLOT_CAP) T[(long long)r[j] * n_cols + c[j]] = make_int2((int)kk, row);
            else over = 1;
        }
        static_assert(SCT_ITEMS == 8, "a thread's ranks leave in one 32-byte store");
        if (k + SCT_ITEMS <= k1 && ((reinterpret_cast<uintptr_t>(rank + k) & 31) == 0)) {
            st_cs_v8(rank + k, r);
        } else {
#pragma unroll
            for (int j = 0; j < SCT_ITEMS; ++j)
                if (k + j < k1) rank[k + j] = r[j];
        }
    }
    if (__any_sync(0xffffffffu, over) && lane_id() == 0) atomicAdd(n_over, 1);
    if (__any_sync(0xffffffffu, bad) && lane_id() == 0) atomicOr(status, ST_BAD_INDEX);
}

cudaError_t launch_col_claim(const int32_t *irp, int32_t n_rows, const int32_t *icol, int64_t nnz, int32_t n_cols,
                             int32_t *nc, int32_t *rank, int2 *T, int32_t *n_over, int32_t *scratch, int *status,
                             cudaStream_t s) {
    if (nnz <= 0) return cudaSuccess;
    cudaError_t e = launch_tile_lines(irp, n_rows, nnz, SCT_TILE, scratch, s);
    if (e != cudaSuccess) return e;
    const long long n_tiles = (nnz + SCT_TILE - 1) / SCT_TILE;
    KernelScope ks("col_claim", s);
    k_col_claim<<<(unsigned)n_tiles, SCT_THREADS, 0, s>>>(irp, n_rows, icol, nnz, n_cols, nc, rank, scratch, n_tiles,
                                                           T, n_over, status);
    return cudaGetLastError();
}

// ------------------------------------------------------------------- fixup
// Short columns (<= 32 entries), one CTA per tile of FT_COLS consecutive
// columns, many CTAs per SM. The tile's (k, row) pairs are loaded into shared
// memory with coalesced loads; pass 1: warp w orders the columns it owns with
// a bitonic network in registers when they are out of order and writes them
// back; pass 2: all threads stride over the tile and write ICOL_T = row and
// VAL_T = VAL[k] contiguously, four independent VAL gathers in flight per
// thread. Columns longer than 32 are marked and left to k_fixup_block. A tile
// whose pairs exceed FT_CAP is handled column by column from global memory.
constexpr int FT_THREADS = 256;
constexpr int FT_COLS = 64;
constexpr int FT_CAP = 2048;  // pairs per tile in shared memory (16 KB)

__device__ __forceinline__ void warp_sort_pairs(int &key, int &row) {
    const unsigned lane = lane_id();
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const int ok = __shfl_xor_sync(0xffffffffu, key, stride);
            const int orow = __shfl_xor_sync(0xffffffffu, row, stride);
            const bool asc = (lane & size) == 0;
            const bool lower = (lane & stride) == 0;
            const bool take = (lower == asc) ? (ok < key) : (ok > key);
            if (take) { key = ok; row = orow; }
        }
    }
}

__device__ __forceinline__ void warp_sort_u32(unsigned &key) {
    const unsigned lane = lane_id();
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const unsigned ok = __shfl_xor_sync(0xffffffffu, key, stride);
            // keep the smaller key where the lane's stride bit equals its
            // size bit (lower half of an ascending pair, or upper half of a
            // descending one), else the larger: one min or max per stage
            const bool kmin = (((lane & size) != 0) == ((lane & stride) != 0));
            key = kmin ? min(key, ok) : max(key, ok);
        }
    }
}

__global__ void __launch_bounds__(FT_THREADS) k_fixup_tiles(const int32_t *__restrict__ cp, int32_t n_cols,
                                                             const double *__restrict__ val,
                                                             const int2 *__restrict__ pairs,
                                                             int32_t *__restrict__ trow, double *__restrict__ tval) {
    __shared__ int2 s_pr[FT_CAP];
    __shared__ int32_t s_cp[FT_COLS + 1];
    const unsigned lane = lane_id();
    const int w = threadIdx.x >> 5;
    const long long c0 = (long long)blockIdx.x * FT_COLS;
    const int nc = (int)min((long long)FT_COLS, (long long)n_cols - c0);
    for (int i = threadIdx.x; i <= nc; i += FT_THREADS) s_cp[i] = cp[c0 + i];
    __syncthreads();
    const int e0 = s_cp[0], e1 = s_cp[nc];
    const bool staged = (e1 - e0) <= FT_CAP;
    if (staged)
        for (int q = e0 + (int)threadIdx.x; q < e1; q += FT_THREADS) s_pr[q - e0] = __ldcs(pairs + q);
    __syncthreads();
    for (int j = w; j < nc; j += FT_THREADS / 32) {
        const int p0 = s_cp[j], p1 = s_cp[j + 1];
        const int len = p1 - p0;
        if (len <= 0) continue;
        if (len > 32) {
            if (staged)
                for (int q = p0 + (int)lane; q < p1; q += 32) s_pr[q - e0].x = -1;
            continue;
        }
        int key = INT_MAX, row = 0;
        if ((int)lane < len) {
            const int2 q = staged ? s_pr[p0 - e0 + lane] : pairs[p0 + lane];
            key = q.x;
            row = q.y;
        }
        const int nxt = __shfl_down_sync(0xffffffffu, key, 1);
        if (__any_sync(0xffffffffu, (int)lane + 1 < len && key > nxt)) {
            // Keys within 2^26 of the first one: sort 32-bit words
            // ((k - k0 + 2^26) << 5 | lane), one shuffle per network step,
            // then fetch each row from the lane it came from.
            const int k0 = __shfl_sync(0xffffffffu, key, 0);
            const long long rel = (long long)key - k0 + (1ll << 26);
            const bool narrow = __all_sync(0xffffffffu, (int)lane >= len || (rel >= 0 && rel < (1ll << 27)));
            if (narrow) {
                unsigned pk = ((int)lane < len) ? (((unsigned)rel << 5) | lane) : 0xffffffffu;
                warp_sort_u32(pk);
                const int src = (int)(pk & 31u);
                const int r2 = __shfl_sync(0xffffffffu, row, src);
                if ((int)lane < len) {
                    key = (int)((long long)k0 + (long long)(pk >> 5) - (1ll << 26));
                    row = r2;
                }
            } else {
                warp_sort_pairs(key, row);
            }
        }
        if ((int)lane < len) {
            if (staged) {
                s_pr[p0 - e0 + lane] = make_int2(key, row);
            } else {
                __stcs(trow + p0 + lane, row);
                __stcs(tval + p0 + lane, __ldg(val + key));
            }
        }
    }
    __syncthreads();
    if (!staged) return;
    for (int q0 = e0 + (int)threadIdx.x; q0 < e1; q0 += 4 * FT_THREADS) {
        int2 pr[4];
        double v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int q = q0 + u * FT_THREADS;
            pr[u] = (q < e1) ? s_pr[q - e0] : make_int2(-1, 0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = (pr[u].x >= 0) ? __ldg(val + pr[u].x) : 0.0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int q = q0 + u * FT_THREADS;
            if (pr[u].x >= 0) {
                __stcs(trow + q, pr[u].y);
                __stcs(tval + q, v[u]);
            }
        }
    }
}

// Short columns from the slot array T (the slot path). One CTA per 64
// columns: thread (r, c) loads T[r * n_cols + j0 + c] for r < NC[j0 + c], so
// each slot row of the tile is one coalesced 512-byte read, into a compact
// per-column layout in shared memory, together with the entry's CCS position.
// Then, as in k_fixup_tiles: a warp per column orders it (packed 32-bit
// bitonic network when out of order), and a flat pass writes ICOL_T and
// VAL_T = VAL[k] with four gathers in flight per thread. Columns longer than
// SLOT_CAP copy their slots to `pairs` at IRP_T[j] + r for k_fixup_block.
constexpr int FS_COLS = 64;

__global__ void __launch_bounds__(FT_THREADS) k_fixup_slots(const int32_t *__restrict__ cp, int32_t n_cols,
                                                             const double *__restrict__ val,
                                                             const int2 *__restrict__ T, int2 *__restrict__ pairs,
                                                             int32_t *__restrict__ trow, double *__restrict__ tval) {
    __shared__ int2 s_pr[FS_COLS * SLOT_CAP];
    __shared__ int32_t s_pos[FS_COLS * SLOT_CAP];
    __shared__ int32_t s_cp[FS_COLS + 1];
    __shared__ int32_t s_off[FS_COLS + 1];
    __shared__ int s_maxl;
    const unsigned lane = lane_id();
    const int w = threadIdx.x >> 5;
    const long long c0 = (long long)blockIdx.x * FS_COLS;
    const int nc = (int)min((long long)FS_COLS, (long long)n_cols - c0);
    for (int i = threadIdx.x; i <= nc; i += FT_THREADS) s_cp[i] = cp[c0 + i];
    __syncthreads();
    if (w == 0) {  // compact offsets of the short columns, and the longest short one
        int a = 0, b = 0, l0 = 0, l1 = 0;
        if ((int)lane < nc) { l0 = s_cp[lane + 1] - s_cp[lane]; a = (l0 <= SLOT_CAP) ? l0 : 0; }
        if ((int)lane + 32 < nc) { l1 = s_cp[lane + 33] - s_cp[lane + 32]; b = (l1 <= SLOT_CAP) ? l1 : 0; }
        int ia = a, ib = b;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int ta = __shfl_up_sync(0xffffffffu, ia, o), tb = __shfl_up_sync(0xffffffffu, ib, o);
            if ((int)lane >= o) { ia += ta; ib += tb; }
        }
        const int tot_a = __shfl_sync(0xffffffffu, ia, 31);
        s_off[lane] = ia - a;
        s_off[lane + 32] = tot_a + ib - b;
        if (lane == 31) s_off[64] = tot_a + ib;
        int m = max(min(l0, SLOT_CAP), min(l1, SLOT_CAP));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) s_maxl = m;
    }
    __syncthreads();
    const int maxl = s_maxl;
    // stage: thread t covers column t % 64 and slots t / 64 + 4 u (u < 8),
    // every load issued before the first store
    {
        constexpr int RSTEP = FT_THREADS / FS_COLS;   // 4
        constexpr int NU = SLOT_CAP / RSTEP;          // 8
        const int cc = threadIdx.x % FS_COLS;
        const int len = (cc < nc) ? s_cp[cc + 1] - s_cp[cc] : 0;
        const bool longc = len > SLOT_CAP;
        const int lim = min(min(len, SLOT_CAP), maxl);
        const int r0 = threadIdx.x / FS_COLS;
        const int2 *tp = T + (long long)r0 * n_cols + (c0 + cc);
        int2 pr[NU];
#pragma unroll
        for (int u = 0; u < NU; ++u)
            if (r0 + u * RSTEP < lim) pr[u] = __ldcs(tp + (long long)(u * RSTEP) * n_cols);
#pragma unroll
        for (int u = 0; u < NU; ++u) {
            const int rr = r0 + u * RSTEP;
            if (rr < lim) {
                if (longc) {
                    pairs[(long long)s_cp[cc] + rr] = pr[u];
                } else {
                    s_pr[s_off[cc] + rr] = pr[u];
                    s_pos[s_off[cc] + rr] = s_cp[cc] + rr;
                }
            }
        }
    }
    __syncthreads();
    for (int jj = w; jj < nc; jj += FT_THREADS / 32) {
        const int len = s_cp[jj + 1] - s_cp[jj];
        if (len <= 0 || len > SLOT_CAP) continue;
        const int o = s_off[jj];
        int key = INT_MAX, row = 0;
        if ((int)lane < len) {
            const int2 q = s_pr[o + lane];
            key = q.x;
            row = q.y;
        }
        const int nxt = __shfl_down_sync(0xffffffffu, key, 1);
        if (__any_sync(0xffffffffu, (int)lane + 1 < len && key > nxt)) {
            const int k0 = __shfl_sync(0xffffffffu, key, 0);
            const long long rel = (long long)key - k0 + (1ll << 26);
            const bool narrow = __all_sync(0xffffffffu, (int)lane >= len || (rel >= 0 && rel < (1ll << 27)));
            if (narrow) {
                unsigned pk = ((int)lane < len) ? (((unsigned)rel << 5) | lane) : 0xffffffffu;
                warp_sort_u32(pk);
                const int src = (int)(pk & 31u);
                const int r2 = __shfl_sync(0xffffffffu, row, src);
                if ((int)lane < len) {
                    key = (int)((long long)k0 + (long long)(pk >> 5) - (1ll << 26));
                    row = r2;
                }
            } else {
                warp_sort_pairs(key, row);
            }
            if ((int)lane < len) s_pr[o + lane] = make_int2(key, row);
        }
    }
    __syncthreads();
    // write-out: ns <= FS_COLS * SLOT_CAP = 8 per thread, all VAL gathers in flight at once
    constexpr int NW = FS_COLS * SLOT_CAP / FT_THREADS;
    const int ns = s_off[nc];
    double v[NW];
#pragma unroll
    for (int u = 0; u < NW; ++u) {
        const int q = threadIdx.x + u * FT_THREADS;
        v[u] = (q < ns) ? __ldg(val + s_pr[q].x) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < NW; ++u) {
        const int q = threadIdx.x + u * FT_THREADS;
        if (q < ns) {
            const int pos = s_pos[q];
            __stcs(trow + pos, s_pr[q].y);
            __stcs(tval + pos, v[u]);
        }
    }
}

// Long columns (> 32 entries): one CTA each.
constexpr int FIX_THREADS = 256;
constexpr int FIX_CHUNK = 4096;

__device__ void block_bitonic_u64(unsigned long long *s, int P) {
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < (P >> 1); i += blockDim.x) {
                const int lo = 2 * i - (i & (stride - 1));
                const int hi = lo + stride;
                const bool asc = (lo & size) == 0;
                const unsigned long long a = s[lo], b = s[hi];
                if ((a > b) == asc) { s[lo] = b; s[hi] = a; }
            }
            __syncthreads();
        }
    }
}

__device__ __forceinline__ int merge_path(const int32_t *A, int na, const int32_t *B, int nb, int d) {
    int lo = max(0, d - nb), hi = min(d, na);
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (A[mid] <= B[d - mid - 1]) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(FIX_THREADS) k_fixup_block(
    const int32_t *__restrict__ cp, const int32_t *__restrict__ irp, int32_t n_rows,
    const double *__restrict__ val, int2 *__restrict__ pairs, const int32_t *__restrict__ long_list,
    const int32_t *__restrict__ long_count, int32_t *__restrict__ keys_tmp, int32_t *__restrict__ trow,
    double *__restrict__ tval) {
    __shared__ unsigned long long s[FIX_CHUNK];
    const int nl = *long_count;
    for (int li = blockIdx.x; li < nl; li += gridDim.x) {
        const int j = long_list[li];
        const int p0 = cp[j], p1 = cp[j + 1];
        const int L = p1 - p0;
        if (L <= 32) continue;
        if (L <= FIX_CHUNK) {
            int P = 64;
            while (P < L) P <<= 1;
            for (int i = threadIdx.x; i < P; i += FIX_THREADS) {
                if (i < L) {
                    const int2 q = pairs[p0 + i];
                    s[i] = ((unsigned long long)(unsigned)q.x << 32) | (unsigned)q.y;
                } else {
                    s[i] = ~0ull;
                }
            }
            __syncthreads();
            block_bitonic_u64(s, P);
            for (int i = threadIdx.x; i < L; i += FIX_THREADS) {
                const unsigned long long q = s[i];
                trow[p0 + i] = (int32_t)(unsigned)(q & 0xffffffffu);
                tval[p0 + i] = __ldg(val + (int)(q >> 32));
            }
            __syncthreads();
            continue;
        }
        // L > FIX_CHUNK: keys only; sorted chunks, then merge passes
        // ping-ponging between keys_tmp[p0..p1) and the column's own pair
        // storage viewed as int32 (2L slots); rows are recomputed at the end.
        int32_t *bufA = keys_tmp + p0;
        int32_t *bufB = reinterpret_cast<int32_t *>(pairs + p0);
        for (int c0 = 0; c0 < L; c0 += FIX_CHUNK) {
            const int cl = min(FIX_CHUNK, L - c0);
            int P = 64;
            while (P < cl) P <<= 1;
            for (int i = threadIdx.x; i < P; i += FIX_THREADS)
                s[i] = (i < cl) ? (unsigned long long)(unsigned)pairs[p0 + c0 + i].x : ~0ull;
            __syncthreads();
            block_bitonic_u64(s, P);
            for (int i = threadIdx.x; i < cl; i += FIX_THREADS) bufA[c0 + i] = (int32_t)s[i];
            __syncthreads();
        }
        int32_t *src = bufA, *dst = bufB;
        for (int wdt = FIX_CHUNK; wdt < L; wdt <<= 1) {
            for (int r0 = 0; r0 < L; r0 += 2 * wdt) {
                const int na = min(wdt, L - r0);
                const int nb = max(0, min(wdt, L - r0 - wdt));
                const int tot = na + nb;
                const int per = (tot + FIX_THREADS - 1) / FIX_THREADS;
                const int d0 = min(tot, (int)threadIdx.x * per), d1 = min(tot, d0 + per);
                const int32_t *A = src + r0, *B = src + r0 + na;
                int ia = merge_path(A, na, B, nb, d0);
                int ib = d0 - ia;
                for (int d = d0; d < d1; ++d) {
                    if (ib >= nb || (ia < na && A[ia] <= B[ib])) dst[r0 + d] = A[ia++];
                    else dst[r0 + d] = B[ib++];
                }
            }
            __syncthreads();
            int32_t *t = src; src = dst; dst = t;
        }
        for (int i = threadIdx.x; i < L; i += FIX_THREADS) {
            const int k = src[i];
            trow[p0 + i] = last_le(irp, 0, n_rows, k);
            tval[p0 + i] = __ldg(val + k);
        }
        __syncthreads();
    }
}

cudaError_t launch_col_fixup_slots(const int32_t *cp, int32_t n_cols, const int32_t *irp, int32_t n_rows,
                                   const double *val, const int2 *T, int2 *pairs, const int32_t *long_list,
                                   int32_t *keys_tmp, int32_t *trow, double *tval, cudaStream_t s) {
    if (n_cols <= 0) return cudaSuccess;
    {
        KernelScope ks("col_fixup_slots", s);
        k_fixup_slots<<<ceil_div_u(n_cols, FS_COLS), FT_THREADS, 0, s>>>(cp, n_cols, val, T, pairs, trow, tval);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const int32_t *long_count = long_list - 1;
    KernelScope ks("col_fixup_block", s);
    k_fixup_block<<<(unsigned)sm_count() * 2u, FIX_THREADS, 0, s>>>(cp, irp, n_rows, val, pairs, long_list,
                                                                     long_count, keys_tmp, trow, tval);
    return cudaGetLastError();
}

size_t col_slot_bytes(int32_t n_cols) { return (size_t)SLOT_CAP * (size_t)n_cols * sizeof(int2); }
int col_slot_cap() { return SLOT_CAP; }

cudaError_t launch_col_fixup(const int32_t *cp, int32_t n_cols, const int32_t *irp, int32_t n_rows,
                             const double *val, int2 *pairs, const int32_t *long_list, int32_t *keys_tmp,
                             int32_t *trow, double *tval, int *status, cudaStream_t s) {
    (void)status;
    if (n_cols <= 0) return cudaSuccess;
    {
        KernelScope ks("col_fixup_tiles", s);
        k_fixup_tiles<<<ceil_div_u(n_cols, FT_COLS), FT_THREADS, 0, s>>>(cp, n_cols, val, pairs, trow, tval);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    {
        const int32_t *long_count = long_list - 1;
        KernelScope ks("col_fixup_block", s);
        k_fixup_block<<<(unsigned)sm_count() * 2u, FIX_THREADS, 0, s>>>(cp, irp, n_rows, val, pairs, long_list,
                                                                         long_count, keys_tmp, trow, tval);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------- row-position slot path
// The slot path above keeps a rank per entry, stores it, and sorts each
// column of its slots with a warp-wide network. When no (i, j) pair repeats,
// the row alone orders a column (the serial scatter lists a column's rows in
// ascending order), so a per-thread register network over (row, slot) keys
// does the sort, and no rank array is needed:
//   k_col_claim_rows: r = atomicAdd(NC[j], 1); slot (r, j) = {k, i} (8 bytes)
//                     for r < SLOT_CAP, reading only ICOL (and IRP for the
//                     rows); entries with r >= SLOT_CAP become records
//                     {k, i, j, r} in a compact list. Rows are owned by
//                     lanes (below).
//   k_fixup_net     : one thread per column sorts the column's slots by row
//                     with a register sorting network; rows and VAL[k] are
//                     written contiguously per CTA. The gathers of VAL stay
//                     local where this path is chosen (neighbouring columns:
//                     a tile's columns take their entries from the same rows).
//                     Slots of longer columns go straight to IRP_T[j] + r.
//   k_ov_place_rv   : list records to IRP_T[j] + r (value gathered from VAL[k]).
//   k_fixup_long_rv : columns of 33..RV_LONG_CAP entries sorted in place by
//                     row (CTA bitonic network on (row, position) keys).
// A repeated row within a column, a longer column or a full record list sets
// ST_REDO; the host then rebuilds the CCS on the (k, row) slot path.
constexpr int RV_LONG_CAP = 4096;

// {row, value} records of the grouped path below (pad: column within the group)
struct __align__(16) RowVal {
    int32_t row;
    int32_t pad;
    double v;
};

// One 16-byte store of a record (L2 only): a plain struct assignment may be
// split into narrower stores, each a partial sector of its own.
__device__ __forceinline__ void store_rec(RowVal *dst, const RowVal &r) {
    __stcg(reinterpret_cast<int4 *>(dst), make_int4(r.row, r.pad, __double2loint(r.v), __double2hiint(r.v)));
}

size_t col_rk_slot_bytes(int32_t n_cols) { return (size_t)SLOT_CAP * (size_t)n_cols * sizeof(int2); }
int col_rv_long_cap() { return RV_LONG_CAP; }

__device__ __forceinline__ int pad32(int e) { return e + (e >> 5); }

// Row-owned claim order: a CTA owns CR_ROWS consecutive rows, their ICOL
// range staged in shared memory with coalesced loads; lane l of warp w owns
// row r0 + 32 w + l, and step j claims the j-th entry of each lane's row. On
// banded matrices the 32 entries of one step are 32 neighbouring columns, so
// a warp's rank atomics fall into a few sectors of NC, and neighbouring
// columns tend to get equal ranks, so the slot stores of a step share
// sectors too. Four steps at a time keep four atomics in flight per lane.
// The fix-up sorts every column, so the order of the claims does not change
// the result; against thread-striped items (one warp instruction = 32
// consecutive entries, rows found per entry) this took the claim from 372 to
// 194 us on the 128^3 stencil.
constexpr int CR_ROWS = 256;
constexpr int CR_CAP = 8192;  // staged entries (32 KB)
constexpr int CR_STEP = 4;
constexpr int CR_LONG = 64;   // longest row a CTA claims row-owned

// Claim of entry k (row `row`, column c): its rank, then its slot or a
// record of the overflow list.
__device__ __forceinline__ void claim_place(int c, int k, int row, int r, int32_t n_cols, int2 *__restrict__ slots,
                                            int4 *__restrict__ ov, long long ov_cap, int32_t *__restrict__ n_ov,
                                            int &redo) {
    if (r < SLOT_CAP) {
        slots[(long long)r * n_cols + c] = make_int2(k, row);
    } else {
        const int q = atomicAdd(n_ov, 1);
        if (q < ov_cap) ov[q] = make_int4(k, row, c, r);
        else redo = 1;
    }
}

__global__ void __launch_bounds__(CR_ROWS) k_col_claim_rows(const int32_t *__restrict__ irp, int32_t n_rows,
                                                            const int32_t *__restrict__ icol, int64_t nnz,
                                                            int32_t n_cols, int32_t *__restrict__ nc,
                                                            int2 *__restrict__ slots, int4 *__restrict__ ov,
                                                            long long ov_cap, int32_t *__restrict__ n_ov,
                                                            int *status) {
    __shared__ int32_t s_c[CR_CAP];
    __shared__ int32_t s_ptr[CR_ROWS + 1];
    const long long r0 = (long long)blockIdx.x * CR_ROWS;
    const int nr = (int)min((long long)CR_ROWS, (long long)n_rows - r0);
    const int t = (int)threadIdx.x;
    const long long e0 = min(max((long long)__ldg(irp + r0), 0ll), (long long)nnz);
    const long long e1 = min(max((long long)__ldg(irp + r0 + nr), e0), (long long)nnz);
    const int n = (int)(e1 - e0);
    const bool staged = n <= CR_CAP;
    if (staged) {
        for (int q0 = t; q0 < n; q0 += 4 * CR_ROWS) {
            int v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = (q0 + u * CR_ROWS < n) ? __ldcs(icol + e0 + q0 + u * CR_ROWS) : 0;
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (q0 + u * CR_ROWS < n) s_c[q0 + u * CR_ROWS] = v[u];
        }
    }
    const long long row = r0 + t;
    long long a = e0, b = e0;
    if (t < nr) {
        a = min(max((long long)__ldg(irp + row), e0), e1);
        b = min(max((long long)__ldg(irp + row + 1), a), e1);
        s_ptr[t] = (int)(a - e0);
    }
    if (t == 0) s_ptr[nr] = n;
    const int len = (int)(b - a);
    // A CTA with a row longer than CR_LONG (or too many entries to stage)
    // claims entry-striped instead: one lane per entry, rows found in the
    // staged pointers, so one long row does not serialise its lane.
    const bool striped = __syncthreads_or(len > CR_LONG) || !staged;
    int bad = 0, redo = 0;
    if (!striped) {
        int wlen = len;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wlen = max(wlen, __shfl_xor_sync(0xffffffffu, wlen, o));
        for (int j0 = 0; j0 < wlen; j0 += CR_STEP) {
            int c[CR_STEP], r[CR_STEP];
#pragma unroll
            for (int u = 0; u < CR_STEP; ++u) {
                const int j = j0 + u;
                c[u] = -1;
                if (j < len) {
                    const int col = s_c[(int)(a - e0) + j];
                    if ((unsigned)col < (unsigned)n_cols) c[u] = col;
                    else bad = 1;
                }
            }
#pragma unroll
            for (int u = 0; u < CR_STEP; ++u) r[u] = (c[u] >= 0) ? atomicAdd(nc + c[u], 1) : -1;
#pragma unroll
            for (int u = 0; u < CR_STEP; ++u)
                if (r[u] >= 0) claim_place(c[u], (int)(a + j0 + u), (int)row, r[u], n_cols, slots, ov, ov_cap, n_ov, redo);
        }
    } else {
        for (int q0 = t; q0 < n; q0 += CR_STEP * CR_ROWS) {
            int c[CR_STEP], r[CR_STEP];
#pragma unroll
            for (int u = 0; u < CR_STEP; ++u) {
                const int q = q0 + u * CR_ROWS;
                c[u] = -1;
                if (q < n) {
                    const int col = staged ? s_c[q] : __ldcs(icol + e0 + q);
                    if ((unsigned)col < (unsigned)n_cols) c[u] = col;
                    else bad = 1;
                }
            }
#pragma unroll
            for (int u = 0; u < CR_STEP; ++u) r[u] = (c[u] >= 0) ? atomicAdd(nc + c[u], 1) : -1;
#pragma unroll
            for (int u = 0; u < CR_STEP; ++u) {
                if (r[u] < 0) continue;
                const int q = q0 + u * CR_ROWS;
                const int rr = (int)r0 + last_le(s_ptr, 0, nr, q);  // the row holding staged entry q
                claim_place(c[u], (int)(e0 + q), rr, r[u], n_cols, slots, ov, ov_cap, n_ov, redo);
            }
        }
    }
    if (__any_sync(0xffffffffu, redo) && lane_id() == 0) atomicOr(status, ST_REDO);
    if (__any_sync(0xffffffffu, bad) && lane_id() == 0) atomicOr(status, ST_BAD_INDEX);
}

cudaError_t launch_col_claim_rk(const int32_t *irp, int32_t n_rows, const int32_t *icol, int64_t nnz, int32_t n_cols,
                                int32_t *nc, void *slots, int4 *ov,
                                int64_t ov_cap, int32_t *n_ov, int32_t *scratch, int *status, cudaStream_t s) {
    if (nnz <= 0) return cudaSuccess;
    KernelScope ks("col_claim_rk", s);
    k_col_claim_rows<<<ceil_div_u(n_rows, CR_ROWS), CR_ROWS, 0, s>>>(irp, n_rows, icol, nnz, n_cols, nc,
                                                                    reinterpret_cast<int2 *>(slots), ov, ov_cap,
                                                                    n_ov, status);
    return cudaGetLastError();
}

// Sorting networks (Batcher's odd-even merge sort) with compile-time
// comparator lists, applied by one thread to keys held in registers.
template <int N>
struct SortNet {
    int n;
    unsigned char a[192], b[192];
};
template <int N>
__host__ __device__ constexpr SortNet<N> make_sort_net() {
    SortNet<N> t{};
    t.n = 0;
    for (int p = 1; p < N; p <<= 1)
        for (int k = p; k >= 1; k >>= 1)
            for (int j = k % p; j + k < N; j += 2 * k)
                for (int i = 0; i < k && i < N - j - k; ++i)
                    if ((i + j) / (2 * p) == (i + j + k) / (2 * p)) {
                        t.a[t.n] = (unsigned char)(i + j);
                        t.b[t.n] = (unsigned char)(i + j + k);
                        ++t.n;
                    }
    return t;
}
template <int N>
__device__ __forceinline__ void net_sort(uint32_t (&key)[SLOT_CAP]) {
    constexpr SortNet<N> net = make_sort_net<N>();  // 19 / 63 / 191 comparators
#pragma unroll
    for (int i = 0; i < net.n; ++i) {
        const uint32_t x = key[net.a[i]], y = key[net.b[i]];
        key[net.a[i]] = min(x, y);
        key[net.b[i]] = max(x, y);
    }
}

// One thread per column, FN_COLS columns per CTA. Thread t reads the slots of
// its column (one coalesced slot row per warp instruction), keeps the keys
// (row << 5 | slot) in registers and the values in shared memory, sorts the
// keys with the smallest network that covers the CTA's longest short column
// (8, 16 or 32 inputs; padding keys 0xffffffff), and records each sorted key
// at its compact position; then all threads write ICOL_T and VAL_T for the
// CTA's columns contiguously. A thread sorts 32 keys in 382 min/max
// instructions where a warp-wide network would spend 15 shuffle stages on one
// column. Needs n_rows < 2^27 - 1 (the host checks); repeated rows set ST_REDO.
constexpr int FN_COLS = 128;
constexpr int FN_WB = 8;

__global__ void __launch_bounds__(FN_COLS) k_fixup_net(const int32_t *__restrict__ cp, int32_t n_cols,
                                                        const int2 *__restrict__ slots, const double *__restrict__ val,
                                                        int32_t *__restrict__ trow,
                                                        double *__restrict__ tval, int *status) {
    __shared__ int32_t s_k[SLOT_CAP][FN_COLS + 1];  // the slots' CRS positions
    __shared__ uint32_t s_key[FN_COLS * SLOT_CAP];
    __shared__ uint8_t s_col[FN_COLS * SLOT_CAP];
    __shared__ int32_t s_cp[FN_COLS + 1];
    __shared__ int32_t s_off[FN_COLS + 1];
    __shared__ int s_wsum[FN_COLS / 32], s_wmax[FN_COLS / 32];
    __shared__ int s_redo;
    const int t = threadIdx.x;
    const unsigned lane = lane_id();
    const int w = t >> 5;
    const long long c0 = (long long)blockIdx.x * FN_COLS;
    const int nc = (int)min((long long)FN_COLS, (long long)n_cols - c0);
    for (int i = t; i <= nc; i += FN_COLS) s_cp[i] = cp[c0 + i];
    if (t == 0) s_redo = 0;
    __syncthreads();
    const int len = (t < nc) ? s_cp[t + 1] - s_cp[t] : 0;
    const bool shortc = len <= SLOT_CAP;
    // compact offsets of the short columns and the longest short column
    int a = shortc ? len : 0;
    int inc = a;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, inc, o);
        if ((int)lane >= o) inc += v;
    }
    int m = a;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 31) s_wsum[w] = inc;
    if (lane == 0) s_wmax[w] = m;
    __syncthreads();
    int woff = 0, maxl = 0;
#pragma unroll
    for (int j = 0; j < FN_COLS / 32; ++j) {
        if (j < w) woff += s_wsum[j];
        maxl = max(maxl, s_wmax[j]);
    }
    const int off = woff + inc - a;
    s_off[t] = off;
    if (t == FN_COLS - 1) s_off[FN_COLS] = off + a;
    const long long at0 = c0 + t;
    if (!shortc) {
        // slots of a long column go to its place in the CCS; k_fixup_long_rv sorts it
        for (int r = 0; r < SLOT_CAP; ++r) {
            const int2 q = __ldcs(slots + (long long)r * n_cols + at0);
            trow[(long long)s_cp[t] + r] = q.y;
            tval[(long long)s_cp[t] + r] = __ldg(val + q.x);
        }
    }
    uint32_t key[SLOT_CAP];
    const int lim = shortc ? len : 0;
#pragma unroll
    for (int r = 0; r < SLOT_CAP; ++r) {
        key[r] = 0xffffffffu;
        if (r < lim) {
            const int2 q = __ldcs(slots + (long long)r * n_cols + at0);
            s_k[r][t] = q.x;
            key[r] = ((uint32_t)q.y << 5) | (uint32_t)r;
        }
    }
    if (maxl <= 8) net_sort<8>(key);
    else if (maxl <= 16) net_sort<16>(key);
    else net_sort<32>(key);
    bool dup = false;
#pragma unroll
    for (int r = 0; r < SLOT_CAP; ++r) {
        if (r < lim) {
            s_key[off + r] = key[r];
            s_col[off + r] = (uint8_t)t;
            if (r > 0 && (key[r] >> 5) == (key[r - 1] >> 5)) dup = true;
        }
    }
    if (dup) s_redo = 1;
    __syncthreads();
    if (t == 0 && s_redo) atomicOr(status, ST_REDO);
    // write-out: FN_WB entries per thread per round, their VAL gathers issued
    // together before any store
    const int ns = s_off[FN_COLS];
    for (int q0 = t; q0 < ns; q0 += FN_COLS * FN_WB) {
        long long pos[FN_WB];
        int32_t rw[FN_WB];
        double v[FN_WB];
#pragma unroll
        for (int u = 0; u < FN_WB; ++u) {
            const int q = q0 + u * FN_COLS;
            pos[u] = -1;
            rw[u] = 0;
            v[u] = 0.0;
            if (q < ns) {
                const uint32_t k = s_key[q];
                const int cc = s_col[q];
                pos[u] = (long long)s_cp[cc] + (q - s_off[cc]);
                rw[u] = (int32_t)(k >> 5);
                v[u] = __ldg(val + s_k[k & 31u][cc]);
            }
        }
#pragma unroll
        for (int u = 0; u < FN_WB; ++u) {
            if (pos[u] >= 0) {
                __stcs(trow + pos[u], rw[u]);
                __stcs(tval + pos[u], v[u]);
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_ov_place_rv(const int32_t *__restrict__ cp, int32_t n_cols,
                                                      const double *__restrict__ val, const int4 *__restrict__ ov,
                                                      long long ov_cap, const int32_t *__restrict__ n_ov,
                                                      int32_t *__restrict__ trow, double *__restrict__ tval) {
    const long long cnt = min((long long)*n_ov, ov_cap);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (long long)gridDim.x * blockDim.x) {
        const int4 q = ov[i];  // {k, row, col, rank}
        if ((unsigned)q.z >= (unsigned)n_cols) continue;
        const long long pos = (long long)cp[q.z] + q.w;
        if (pos >= cp[q.z + 1]) continue;
        trow[pos] = q.y;
        tval[pos] = __ldg(val + q.x);
    }
}

// One CTA per long column (33 .. RV_LONG_CAP entries, in place): keys
// (row << 32 | position) sorted in shared memory, then every value is read
// before any is written back.
constexpr int RVL_PER = RV_LONG_CAP / FIX_THREADS;  // 16

__global__ void __launch_bounds__(FIX_THREADS) k_fixup_long_rv(const int32_t *__restrict__ cp,
                                                                const int32_t *__restrict__ long_list,
                                                                const int32_t *__restrict__ long_count,
                                                                int32_t *__restrict__ trow,
                                                                double *__restrict__ tval, int *status) {
    __shared__ unsigned long long s[RV_LONG_CAP];
    __shared__ int s_redo;
    const int nl = *long_count;
    for (int li = blockIdx.x; li < nl; li += gridDim.x) {
        const int j = long_list[li];
        const int p0 = cp[j], p1 = cp[j + 1];
        const int L = p1 - p0;
        if (L <= SLOT_CAP) continue;
        if (L > RV_LONG_CAP) {
            if (threadIdx.x == 0) atomicOr(status, ST_REDO);
            continue;
        }
        if (threadIdx.x == 0) s_redo = 0;
        int P = 64;
        while (P < L) P <<= 1;
        for (int i = threadIdx.x; i < P; i += FIX_THREADS)
            s[i] = (i < L) ? (((unsigned long long)(unsigned)trow[p0 + i] << 32) | (unsigned)i) : ~0ull;
        __syncthreads();
        block_bitonic_u64(s, P);
        double v[RVL_PER];
#pragma unroll
        for (int u = 0; u < RVL_PER; ++u) {
            const int i = threadIdx.x + u * FIX_THREADS;
            v[u] = (i < L) ? tval[p0 + (int)(s[i] & 0xffffffffu)] : 0.0;
            if (i > 0 && i < L && (s[i] >> 32) == (s[i - 1] >> 32)) s_redo = 1;
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < RVL_PER; ++u) {
            const int i = threadIdx.x + u * FIX_THREADS;
            if (i < L) {
                trow[p0 + i] = (int32_t)(s[i] >> 32);
                tval[p0 + i] = v[u];
            }
        }
        if (threadIdx.x == 0 && s_redo) atomicOr(status, ST_REDO);
        __syncthreads();
    }
}

cudaError_t launch_col_fixup_rk(const int32_t *cp, int32_t n_cols, int32_t n_rows, const double *val,
                                const void *slots, const int4 *ov, int64_t ov_cap, const int32_t *n_ov,
                                const int32_t *long_list, int32_t *trow, double *tval, int *status, cudaStream_t s) {
    if (n_cols <= 0) return cudaSuccess;
    {
        KernelScope ks("col_fixup_rk", s);
        k_fixup_net<<<ceil_div_u(n_cols, FN_COLS), FN_COLS, 0, s>>>(cp, n_cols, reinterpret_cast<const int2 *>(slots),
                                                                    val, trow, tval, status);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    {
        KernelScope ks("col_overflow_rk", s);
        k_ov_place_rv<<<(unsigned)sm_count() * 2u, 256, 0, s>>>(cp, n_cols, val, ov, ov_cap, n_ov, trow, tval);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const int32_t *long_count = long_list - 1;
    KernelScope ks("col_fixup_long_rv", s);
    k_fixup_long_rv<<<(unsigned)sm_count() * 2u, FIX_THREADS, 0, s>>>(cp, long_list, long_count, trow, tval, status);
    return cudaGetLastError();
}

// ---------------------------------------------------- grouped row-value path
// The claim above stores each entry's 16-byte record at its own slot, so a
// warp's stores scatter over many sectors. Here a record goes to the region
// of its column group (GRP_COLS consecutive columns, GRP_CAP records):
//   k_col_claim_grp : a CTA groups its tile's entries by column group in
//                     shared memory (warp match, then a small hash table),
//                     reserves one run per (CTA, group) with a single global
//                     atomicAdd on the group's count, stages the records of
//                     each run contiguously and writes them with coalesced
//                     stores. On banded matrices a tile touches a few groups
//                     with runs of ~100 records; entries whose group finds no
//                     table slot take their own atomic and store.
//   k_scan          : group counts -> the groups' first CCS positions.
//   k_fixup_grp     : one CTA per group: records in (coalesced), a counting
//                     sort by column in shared memory, IRP_T of the group's
//                     columns, each column of <= 32 entries sorted by row with
//                     the register network, the group's CCS range written
//                     contiguously; longer columns are written unsorted and
//                     listed for k_fixup_long_rv.
// A group of more than GRP_CAP entries, a repeated row within a column or a
// column over RV_LONG_CAP sets ST_REDO (the host then takes the (k, row) path).
constexpr int GRP_COLS = 64;
constexpr int GRP_CAP = GRP_COLS * SLOT_CAP;  // 2048 records (32 KB) per group
constexpr int GCL_THREADS = 256;
constexpr int GCL_ITEMS = 4;
constexpr int GCL_TILE = GCL_THREADS * GCL_ITEMS;
constexpr int GCL_WIN = 1024;
constexpr int GCL_HASH = 512;
constexpr int GCL_PROBES = 8;

long long col_grp_count(int32_t n_cols) { return ((long long)n_cols + GRP_COLS - 1) / GRP_COLS; }
size_t col_grp_scratch_bytes(int64_t nnz) { return tile_lines_bytes(nnz, GCL_TILE); }
size_t col_grp_region_bytes(int32_t n_cols) {
    return (size_t)col_grp_count(n_cols) * GRP_CAP * sizeof(RowVal);
}

__global__ void __launch_bounds__(GCL_THREADS) k_col_claim_grp(const int32_t *__restrict__ irp, int32_t n_rows,
                                                                const int32_t *__restrict__ icol,
                                                                const double *__restrict__ val, int64_t nnz,
                                                                int32_t n_cols, int32_t *__restrict__ gcnt,
                                                                const int32_t *__restrict__ tl, long long n_tiles,
                                                                RowVal *__restrict__ regions, int *status) {
    __shared__ int32_t s_ptr[GCL_WIN];
    __shared__ int32_t s_row[GCL_TILE + GCL_TILE / 32];
    __shared__ int32_t s_hkey[GCL_HASH];
    __shared__ int32_t s_hcnt[GCL_HASH];   // run length, then the run's staging offset
    __shared__ int32_t s_hbase[GCL_HASH];  // the run's first position in its group region
    __shared__ RowVal s_rec[GCL_TILE];
    __shared__ long long s_dst[GCL_TILE];
    __shared__ int s_wsum[GCL_THREADS / 32];
    __shared__ int s_total;
    const int t = threadIdx.x;
    const unsigned lane = lane_id();
    const int w = t >> 5;
    const long long k0 = (long long)blockIdx.x * GCL_TILE;
    const long long k1 = min(k0 + (long long)GCL_TILE, (long long)nnz);
    for (int i = t; i < GCL_HASH; i += GCL_THREADS) { s_hkey[i] = -1; s_hcnt[i] = 0; }
    if (t == 0) s_total = 0;  // first the tile's run count, later its record count
    int c[GCL_ITEMS];
    double v[GCL_ITEMS];
#pragma unroll
    for (int u = 0; u < GCL_ITEMS; ++u) {
        const long long k = k0 + u * GCL_THREADS + t;
        c[u] = (k < k1) ? __ldcs(icol + k) : -1;
    }
#pragma unroll
    for (int u = 0; u < GCL_ITEMS; ++u) {
        const long long k = k0 + u * GCL_THREADS + t;
        v[u] = (k < k1) ? __ldcs(val + k) : 0.0;
    }
    const int lo = tl[blockIdx.x];
    const int hi = (blockIdx.x + 1 < n_tiles) ? tl[blockIdx.x + 1] : n_rows - 1;
    const int wn = hi - lo + 2;
    const bool sm = wn <= GCL_WIN;
    if (sm)
        for (int i = t; i < wn; i += GCL_THREADS) s_ptr[i] = irp[lo + i];
    __syncthreads();
    {
        const long long kb = k0 + (long long)t * GCL_ITEMS;  // this thread's block of entries
        if (kb < k1) {
            int row = sm ? lo + last_le(s_ptr, 0, wn - 1, kb) : last_le(irp, lo, hi + 1, kb);
#pragma unroll
            for (int j = 0; j < GCL_ITEMS; ++j) {
                const long long kk = kb + j;
                while (row < hi && (long long)(sm ? s_ptr[row + 1 - lo] : irp[row + 1]) <= kk) ++row;
                s_row[pad32(t * GCL_ITEMS + j)] = row;
            }
        }
    }
    // lanes of one instruction with the same group form a run led by its
    // first lane; a tile whose runs outnumber half the table (scattered
    // columns: nearly one group per entry) skips the table and lets every
    // leader reserve its run with one global atomic and store it directly
    int grp[GCL_ITEMS];
    unsigned peers[GCL_ITEMS];
    int bad = 0, n_lead = 0;
#pragma unroll
    for (int u = 0; u < GCL_ITEMS; ++u) {
        const long long k = k0 + u * GCL_THREADS + t;
        const bool has = k < k1;
        const bool ok = has && (unsigned)c[u] < (unsigned)n_cols;
        bad |= has && !ok;
        grp[u] = ok ? (c[u] / GRP_COLS) : -1 - (int)lane;
        peers[u] = __match_any_sync(0xffffffffu, grp[u]);
        n_lead += __popc(__ballot_sync(0xffffffffu, ok && (int)lane == __ffs(peers[u]) - 1));
    }
    if (lane == 0 && n_lead) atomicAdd(&s_total, n_lead);
    __syncthreads();
    if (s_total > GCL_HASH / 2) {
        int redo = 0;
#pragma unroll
        for (int u = 0; u < GCL_ITEMS; ++u) {
            const bool ok = grp[u] >= 0;
            const int leader = __ffs(peers[u]) - 1;
            int base = 0;
            if (ok && (int)lane == leader) base = atomicAdd(gcnt + grp[u], __popc(peers[u]));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (!ok) continue;
            const int gp = base + __popc(peers[u] & lanemask_lt());
            RowVal q;
            q.row = s_row[pad32(u * GCL_THREADS + t)];
            q.pad = c[u] % GRP_COLS;
            q.v = v[u];
            if (gp < GRP_CAP) store_rec(regions + (long long)grp[u] * GRP_CAP + gp, q);
            else redo = 1;
        }
        if (__any_sync(0xffffffffu, redo) && lane == 0) atomicOr(status, ST_REDO);
        if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(status, ST_BAD_INDEX);
        return;
    }
    // banded tiles: runs of the same group share one table slot
    int slot[GCL_ITEMS], local[GCL_ITEMS];
#pragma unroll
    for (int u = 0; u < GCL_ITEMS; ++u) {
        const bool ok = grp[u] >= 0;
        const int g = grp[u];
        const int leader = __ffs(peers[u]) - 1;
        int h = -1, base = 0;
        if (ok && (int)lane == leader) {
            h = (int)(((unsigned)g * 2654435761u) >> 23);  // 9 bits
            for (int p = 0;; ++p) {
                const int old = atomicCAS(&s_hkey[h], -1, g);
                if (old == -1 || old == g) break;
                if (p + 1 >= GCL_PROBES) { h = -1; break; }
                h = (h + 1) & (GCL_HASH - 1);
            }
            if (h >= 0) base = atomicAdd(&s_hcnt[h], __popc(peers[u]));
        }
        h = __shfl_sync(0xffffffffu, h, leader);
        base = __shfl_sync(0xffffffffu, base, leader);
        slot[u] = ok ? h : -2;  // -1: no table slot, the entry goes alone
        local[u] = base + __popc(peers[u] & lanemask_lt());
    }
    __syncthreads();
    {
        // staging offsets (exclusive scan over the table, two slots per
        // thread) and one global reservation per occupied slot
        const int a0 = s_hcnt[2 * t], a1 = s_hcnt[2 * t + 1];
        int inc = a0 + a1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int x = __shfl_up_sync(0xffffffffu, inc, o);
            if ((int)lane >= o) inc += x;
        }
        if (lane == 31) s_wsum[w] = inc;
        const int b0 = a0 > 0 ? atomicAdd(gcnt + s_hkey[2 * t], a0) : 0;
        const int b1 = a1 > 0 ? atomicAdd(gcnt + s_hkey[2 * t + 1], a1) : 0;
        __syncthreads();
        int woff = 0, tot = 0;
#pragma unroll
        for (int j = 0; j < GCL_THREADS / 32; ++j) {
            if (j < w) woff += s_wsum[j];
            tot += s_wsum[j];
        }
        const int excl = woff + inc - a0 - a1;
        s_hcnt[2 * t] = excl;
        s_hcnt[2 * t + 1] = excl + a0;
        s_hbase[2 * t] = b0;
        s_hbase[2 * t + 1] = b1;
        if (t == 0) s_total = tot;
    }
    __syncthreads();
    int redo = 0;
#pragma unroll
    for (int u = 0; u < GCL_ITEMS; ++u) {
        if (slot[u] == -2) continue;
        const int e = u * GCL_THREADS + t;
        RowVal q;
        q.row = s_row[pad32(e)];
        q.pad = c[u] % GRP_COLS;
        q.v = v[u];
        const long long g = c[u] / GRP_COLS;
        if (slot[u] >= 0) {
            const int sp = s_hcnt[slot[u]] + local[u];
            const int gp = s_hbase[slot[u]] + local[u];
            s_rec[sp] = q;
            s_dst[sp] = gp < GRP_CAP ? g * GRP_CAP + gp : -1;
            redo |= gp >= GRP_CAP;
        } else {
            const int gp = atomicAdd(gcnt + g, 1);
            if (gp < GRP_CAP) store_rec(regions + g * GRP_CAP + gp, q);
            else redo = 1;
        }
    }
    __syncthreads();
    for (int q = t; q < s_total; q += GCL_THREADS) {
        const long long d = s_dst[q];
        if (d >= 0) store_rec(regions + d, s_rec[q]);
    }
    if (__any_sync(0xffffffffu, redo) && lane == 0) atomicOr(status, ST_REDO);
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(status, ST_BAD_INDEX);
}

constexpr int GFX_THREADS = 128;
// Six CTAs per SM: the column order is kept as 2-byte record indices (the
// rows are read from the records), so a group needs 36 KB of shared memory
// instead of 48, and the sorting networks are held to 80 registers
// (688 -> 592 us on the 4e6-row power law).
constexpr int GFX_CTAS_PER_SM = 6;
static_assert(GRP_CAP <= 65536, "record indices are 16-bit");
constexpr size_t GFX_SMEM = (size_t)GRP_CAP * (sizeof(RowVal) + sizeof(uint16_t));

__global__ void __launch_bounds__(GFX_THREADS, GFX_CTAS_PER_SM) k_fixup_grp(const int32_t *__restrict__ gpos, int32_t n_cols,
                                                            long long n_groups, const RowVal *__restrict__ regions,
                                                            int32_t *__restrict__ cp, int32_t *__restrict__ trow,
                                                            double *__restrict__ tval, int32_t *__restrict__ colmax,
                                                            int32_t *__restrict__ long_list,
                                                            int32_t *__restrict__ long_count, int *status) {
    extern __shared__ __align__(16) unsigned char gfx_smem[];
    RowVal *s_rec = reinterpret_cast<RowVal *>(gfx_smem);
    uint16_t *s_key = reinterpret_cast<uint16_t *>(s_rec + GRP_CAP);  // record in column order
    __shared__ int32_t s_ccnt[GRP_COLS], s_coff[GRP_COLS + 1], s_cur[GRP_COLS];
    __shared__ int s_redo;
    const int t = threadIdx.x;
    const unsigned lane = lane_id();
    const long long g = blockIdx.x;
    const int gb = gpos[g];
    const int cnt = gpos[g + 1] - gb;
    if (cnt < 0) return;  // only after a failed scan, which the host reports
    const long long c0 = g * GRP_COLS;
    const int ncl = (int)min((long long)GRP_COLS, (long long)n_cols - c0);
    if (t < GRP_COLS) { s_ccnt[t] = 0; s_cur[t] = 0; }
    if (t == 0) s_redo = 0;
    if (cnt > GRP_CAP) {  // the claim flagged it; nothing here is usable
        if (t == 0) atomicOr(status, ST_REDO);
        return;
    }
    __syncthreads();
    const RowVal *reg = regions + g * GRP_CAP;
    for (int q = t; q < cnt; q += GFX_THREADS) {
        const int4 w4 = __ldcs(reinterpret_cast<const int4 *>(reg) + q);  // {row, column in group, value}
        RowVal r;
        r.row = w4.x;
        r.pad = (unsigned)w4.y < (unsigned)ncl ? w4.y : 0;
        r.v = __hiloint2double(w4.w, w4.z);
        s_rec[q] = r;
        atomicAdd(&s_ccnt[r.pad], 1);
    }
    __syncthreads();
    if (t < 32) {  // exclusive scan of the 64 column counts, two per lane
        const int a = s_ccnt[2 * t], b = s_ccnt[2 * t + 1];
        int inc = a + b;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int x = __shfl_up_sync(0xffffffffu, inc, o);
            if ((int)lane >= o) inc += x;
        }
        s_coff[2 * t] = inc - a - b;
        s_coff[2 * t + 1] = inc - b;
        if (t == 31) s_coff[GRP_COLS] = inc;
        int m = max(a, b);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (t == 0 && m > 0) atomicMax(colmax, m);
    }
    __syncthreads();
    if (t < ncl) {
        cp[c0 + t] = gb + s_coff[t];
        if (s_ccnt[t] > SLOT_CAP) long_list[atomicAdd(long_count, 1)] = (int32_t)(c0 + t);
    }
    if (g == n_groups - 1 && t == 0) cp[n_cols] = gb + cnt;
    for (int q = t; q < cnt; q += GFX_THREADS) {
        const int j = s_rec[q].pad;
        const int p = s_coff[j] + atomicAdd(&s_cur[j], 1);
        s_key[p] = (uint16_t)q;
    }
    __syncthreads();
    if (t < ncl) {
        const int len = s_ccnt[t];
        const int off = s_coff[t];
        if (len >= 2 && len <= SLOT_CAP) {
            uint32_t key[SLOT_CAP];
#pragma unroll
            for (int r = 0; r < SLOT_CAP; ++r)
                key[r] = (r < len) ? (((uint32_t)s_rec[s_key[off + r]].row << 5) | (uint32_t)r) : 0xffffffffu;
            if (len <= 8) net_sort<8>(key);
            else if (len <= 16) net_sort<16>(key);
            else net_sort<32>(key);
            int idx[SLOT_CAP];
            bool dup = false;
#pragma unroll
            for (int r = 0; r < SLOT_CAP; ++r) {
                if (r < len) {
                    idx[r] = s_key[off + (int)(key[r] & 31u)];
                    if (r > 0 && (key[r] >> 5) == (key[r - 1] >> 5)) dup = true;
                }
            }
#pragma unroll
            for (int r = 0; r < SLOT_CAP; ++r)
                if (r < len) s_key[off + r] = (uint16_t)idx[r];
            if (dup) s_redo = 1;
        }
    }
    __syncthreads();
    if (t == 0 && s_redo) atomicOr(status, ST_REDO);
    for (int q = t; q < cnt; q += GFX_THREADS) {
        const int k = s_key[q];
        __stcs(trow + gb + q, s_rec[k].row);
        __stcs(tval + gb + q, s_rec[k].v);
    }
}

cudaError_t launch_col_claim_grp(const int32_t *irp, int32_t n_rows, const int32_t *icol, const double *val,
                                 int64_t nnz, int32_t n_cols, int32_t *gcnt, void *regions, int32_t *scratch,
                                 int *status, cudaStream_t s) {
    if (nnz <= 0) return cudaSuccess;
    cudaError_t e = launch_tile_lines(irp, n_rows, nnz, GCL_TILE, scratch, s);
    if (e != cudaSuccess) return e;
    const long long n_tiles = (nnz + GCL_TILE - 1) / GCL_TILE;
    KernelScope ks("col_claim_grp", s);
    k_col_claim_grp<<<(unsigned)n_tiles, GCL_THREADS, 0, s>>>(irp, n_rows, icol, val, nnz, n_cols, gcnt, scratch,
                                                               n_tiles, reinterpret_cast<RowVal *>(regions), status);
    return cudaGetLastError();
}

cudaError_t launch_col_fixup_grp(const int32_t *gpos, int32_t n_cols, const void *regions, int32_t *cp,
                                 int32_t *trow, double *tval, int32_t *colmax, int32_t *long_list, int *status,
                                 cudaStream_t s) {
    if (n_cols <= 0) return cudaSuccess;
    const long long n_groups = col_grp_count(n_cols);
    int32_t *long_count = long_list - 1;
    {
        cudaError_t e = set_smem_attr(k_fixup_grp, GFX_SMEM);
        if (e != cudaSuccess) return e;
        KernelScope ks("col_fixup_grp", s);
        k_fixup_grp<<<(unsigned)n_groups, GFX_THREADS, GFX_SMEM, s>>>(gpos, n_cols, n_groups,
                                                                     reinterpret_cast<const RowVal *>(regions), cp,
                                                                     trow, tval, colmax, long_list, long_count, status);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    KernelScope ks("col_fixup_long_rv", s);
    k_fixup_long_rv<<<(unsigned)sm_count() * 2u, FIX_THREADS, 0, s>>>(cp, long_list, long_count, trow, tval, status);
    return cudaGetLastError();
}

// ------------------------------------------------------- column locality
// Share of sampled neighbouring entries (k, k + 1) whose columns differ by 1
// to 8: high for banded and stencil matrices, where a row's consecutive
// entries fill neighbouring slots of the slot-major array, near zero for
// scattered columns. Samples are spread evenly over the entries.
__global__ void __launch_bounds__(256) k_col_locality(const int32_t *__restrict__ icol, int64_t nnz, int samples,
                                                       int32_t *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    int local = 0;
    if (i < samples && nnz > 1) {
        const long long k = (long long)((double)i * (double)(nnz - 1) / (double)samples);
        const long long d = (long long)__ldg(icol + k + 1) - (long long)__ldg(icol + k);
        local = (d >= 1 && d <= 8) ? 1 : 0;
    }
    local = __reduce_add_sync(0xffffffffu, (unsigned)local);
    if (lane_id() == 0 && local) atomicAdd(out, local);
}

cudaError_t launch_col_locality(const int32_t *icol, int64_t nnz, int samples, int32_t *out, cudaStream_t s) {
    if (nnz <= 1 || samples <= 0) return cudaSuccess;
    KernelScope ks("col_locality", s);
    k_col_locality<<<ceil_div_u(samples, 256), 256, 0, s>>>(icol, nnz, samples, out);
    return cudaGetLastError();
}


// ------------------------------------------------ structurally symmetric path
// A special case of Phase I (Sec. 2.1) that needs no count, no prefix sum
// and no sort. When the pattern of A equals the pattern of its transpose and
// every row lists its columns in strictly ascending order, the serial Phase
// I gives column c exactly the rows that row c lists as columns, in the same
// ascending order. Then IRP_T = IRP and ICOL_T = ICOL, and the CCS value at
// position p (row c, column i) is the value of the mirror entry (i, c):
// VAL_T[p] = VAL[q], q the position of column c in row i.
// k_ccs_sym does that in one pass. A warp takes a tile of SYM_TILE
// consecutive entries and each thread SYM_ITEMS consecutive ones (16-byte
// loads of ICOL and stores of ICOL_T, 32-byte stores of VAL_T, when the
// arrays are aligned for them):
// the thread finds the row of its first entry by a binary search of the
// tile's row pointers (staged in shared memory) and walks on from there, so
// every entry knows its row c, its place in the row and whether it is the
// row's last. Then entry p (row c, column i) reads the bounds of row i and
// ICOL at a first guess for q reflected through the row,
// q = IRP[i+1] - 1 - (p - IRP[c]) (exact for shift-invariant symmetric
// stencils), else binary-searches row i, and gathers VAL[q]. The kernel is
// bound by the latency of these dependent gathers and by the instructions
// around them, so positions are 32-bit (IRP is int32, so nnz <= 2^31 - 1)
// and the items of a thread run their gathers side by side. Every entry must
// find its mirror: since the mirror map is then one-to-one on a finite set
// of distinct entries, the pattern is symmetric. A missing mirror or a row
// out of order sets ST_REDO (the host then builds the CCS on a general path
// and drops what this kernel wrote), a column out of range ST_BAD_INDEX;
// cnt[2] receives the longest row (= the longest column).
constexpr int SYM_THREADS = 256;
constexpr int SYM_WARPS = SYM_THREADS / 32;
constexpr int SYM_ITEMS = 4;
constexpr int SYM_TILE = 32 * SYM_ITEMS;  // entries of a warp tile
constexpr int SYM_CTAS_PER_SM = 4;        // resident CTAs (up to 64 registers a thread)
// row pointers a warp stages per tile (more rows: read from global memory);
// small, so that the CTAs of an SM need little shared memory and the rest of
// the 256 KB per SM serves as L1 for the mirror gathers (see the carveout
// below)
constexpr int SYM_WIN = 64;

static_assert(SYM_ITEMS % 4 == 0, "16-byte accesses cover a thread's items");

// rows of a thread's entries [kb, kb + m) from the tile's row pointers
// rp[r - lo] = IRP[r], rows lo..hi: c[j] the row, jj[j] the place in it
// (unsigned: a malformed IRP gives a huge value, never a negative one), last
// bit j set when entry j ends its row; wmax = longest row started here.
template <int ITEMS>
__device__ __forceinline__ void sym_rows(const int32_t *rp, int lo, int hi, int kb, int m, int (&c)[ITEMS],
                                         unsigned (&jj)[ITEMS], unsigned &last, int &wmax) {
    int l = 0, h = hi - lo + 1;  // largest r - lo in [0, hi - lo] with IRP[r] <= kb
    while (h - l > 1) {
        const int mid = (l + h) >> 1;
        if (rp[mid] <= kb) l = mid; else h = mid;
    }
    int r = lo + l, rs = rp[l], re = rp[l + 1];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const int p = kb + j;
        c[j] = -1;
        jj[j] = 0;
        if (j < m) {
            while (p >= re && r < hi) {
                ++r;
                rs = re;
                re = rp[r + 1 - lo];
            }
            c[j] = r;
            jj[j] = (unsigned)p - (unsigned)rs;
            if (p + 1 >= re) last |= 1u << j;
            if (p == rs) wmax = max(wmax, re - rs);
        }
    }
}

// Persistent warps: warp w takes the tiles w, w + (warps in the grid), ...;
// a tile is SYM_TILE consecutive entries, SYM_ITEMS per lane. Nothing waits
// on another warp: the tile's row pointers go to the warp's own slice of
// shared memory, and the longest row, ST_REDO and ST_BAD_INDEX leave once
// per warp, at its end. A warp loads its next tile's columns and row range
// while it works on the current one, and that tile's row pointers (into two
// registers a lane) at the end of it, so only the dependent gathers remain on
// each tile's path.
template <bool VEC>
__global__ void __launch_bounds__(SYM_THREADS, SYM_CTAS_PER_SM) k_ccs_sym(
    const int32_t *__restrict__ irp, int32_t n, const int32_t *__restrict__ icol, const double *__restrict__ val,
    int32_t nnz, const int32_t *__restrict__ tl, int n_tiles, int32_t *__restrict__ trow,
    double *__restrict__ tval, unsigned long long *__restrict__ cnt, int *status) {
    __shared__ int32_t s_ptr[SYM_WARPS][SYM_WIN];
    const unsigned lane = lane_id();
    int32_t *sp = s_ptr[threadIdx.x >> 5];
    const int warps = (int)(gridDim.x * SYM_WARPS);
    int wmax = 0, bad = 0, redo = 0;
    // the next tile's columns and row range are loaded while this one is processed
    const auto load_tile = [&](int t, int (&ci)[SYM_ITEMS], int &nxt, int &lo, int &hi) {
        const long long kbl = (long long)t * SYM_TILE + (long long)lane * SYM_ITEMS;
        const int m = (int)max(min((long long)SYM_ITEMS, (long long)nnz - kbl), 0ll);
        const int kb = m > 0 ? (int)kbl : 0;
        if (VEC && m == SYM_ITEMS) {
            const int4 w = __ldcs(reinterpret_cast<const int4 *>(icol + kb));
            ci[0] = w.x; ci[1] = w.y; ci[2] = w.z; ci[3] = w.w;
        } else {
#pragma unroll
            for (int j = 0; j < SYM_ITEMS; ++j) ci[j] = (j < m) ? __ldcs(icol + kb + j) : 0;
        }
        nxt = (m == SYM_ITEMS && kbl + SYM_ITEMS < nnz && lane == 31) ? __ldg(icol + kb + SYM_ITEMS) : INT_MAX;
        lo = tl[t];
        hi = (t + 1 < n_tiles) ? tl[t + 1] : n - 1;
    };
    // and the next tile's row pointers (at most SYM_WIN of them: two a lane)
    const auto load_win = [&](int lo, int hi, int &w0, int &w1) {
        const int wn = hi - lo + 2;
        w0 = (wn <= SYM_WIN && (int)lane < wn) ? __ldg(irp + lo + lane) : 0;
        w1 = (wn <= SYM_WIN && (int)lane + 32 < wn) ? __ldg(irp + lo + 32 + lane) : 0;
    };
    static_assert(SYM_WIN <= 64, "two row pointers a lane");
    static_assert(SYM_ITEMS == 4, "a lane's columns are one 16-byte load");
    int t = (int)(blockIdx.x * SYM_WARPS + (threadIdx.x >> 5));
    int ci_n[SYM_ITEMS] = {0, 0, 0, 0}, nx_n = INT_MAX, lo_n = 0, hi_n = 0, w0 = 0, w1 = 0;
    if (t < n_tiles) {
        load_tile(t, ci_n, nx_n, lo_n, hi_n);
        load_win(lo_n, hi_n, w0, w1);
    }
    for (; t < n_tiles; t += warps) {
        const long long kbl = (long long)t * SYM_TILE + (long long)lane * SYM_ITEMS;
        const int m = (int)max(min((long long)SYM_ITEMS, (long long)nnz - kbl), 0ll);
        const int kb = m > 0 ? (int)kbl : 0;
        int ci[SYM_ITEMS];
#pragma unroll
        for (int j = 0; j < SYM_ITEMS; ++j) ci[j] = ci_n[j];
        int nxt = __shfl_down_sync(0xffffffffu, ci[0], 1);
        if (lane == 31 || m < SYM_ITEMS) nxt = (m == SYM_ITEMS) ? nx_n : INT_MAX;
        const int lo = lo_n, hi = hi_n;
        if (t + warps < n_tiles) load_tile(t + warps, ci_n, nx_n, lo_n, hi_n);
        const int wn = hi - lo + 2;
        const bool sm = wn <= SYM_WIN;
        __syncwarp();  // the slice was read for the tile before
        if (sm) {
            if ((int)lane < wn) sp[lane] = w0;
            if ((int)lane + 32 < wn) sp[lane + 32] = w1;
        }
        __syncwarp();
        int c[SYM_ITEMS];
        unsigned jj[SYM_ITEMS], last = 0;
        if (m > 0) {
            if (sm) sym_rows<SYM_ITEMS>(sp, lo, hi, kb, m, c, jj, last, wmax);
            else sym_rows<SYM_ITEMS>(irp + lo, lo, hi, kb, m, c, jj, last, wmax);
        } else {
#pragma unroll
            for (int j = 0; j < SYM_ITEMS; ++j) c[j] = -1, jj[j] = 0;
        }
        int a[SYM_ITEMS], b[SYM_ITEMS];
#pragma unroll
        for (int j = 0; j < SYM_ITEMS; ++j) {
            a[j] = b[j] = 0;
            if (c[j] < 0) continue;
            const int i = ci[j];
            if ((unsigned)i >= (unsigned)n) {
                bad = 1;
                c[j] = -1;
                continue;
            }
            const int after = (j + 1 < SYM_ITEMS) ? ci[j + 1] : nxt;
            if (!((last >> j) & 1u) && after <= i) redo = 1;
            a[j] = min(max(__ldg(irp + i), 0), nnz);
            b[j] = min(max(__ldg(irp + i + 1), a[j]), nnz);
        }
        int q[SYM_ITEMS], g[SYM_ITEMS];
#pragma unroll
        for (int j = 0; j < SYM_ITEMS; ++j) {
            q[j] = 0;
            g[j] = -1;
            if (c[j] >= 0 && jj[j] < (unsigned)(b[j] - a[j])) {
                q[j] = b[j] - 1 - (int)jj[j];
                g[j] = __ldg(icol + q[j]);
            }
        }
#pragma unroll
        for (int j = 0; j < SYM_ITEMS; ++j) {
            if (c[j] < 0 || g[j] == c[j]) continue;
            int l = a[j], h = b[j];
            while (h - l > 1) {
                const int mid = l + ((h - l) >> 1);
                if (__ldg(icol + mid) <= c[j]) l = mid; else h = mid;
            }
            if (l < b[j] && __ldg(icol + l) == c[j]) q[j] = l;
            else redo = 1, c[j] = -1;
        }
        double v[SYM_ITEMS];
#pragma unroll
        for (int j = 0; j < SYM_ITEMS; ++j) v[j] = (c[j] >= 0) ? __ldg(val + q[j]) : 0.0;
        // every entry is stored: a failed one leaves ST_REDO or ST_BAD_INDEX set,
        // and the host then discards both arrays
        if (VEC && m == SYM_ITEMS) {
#pragma unroll
            for (int h = 0; h < SYM_ITEMS / 4; ++h)
                __stcs(reinterpret_cast<int4 *>(trow + kb) + h, make_int4(ci[4 * h], ci[4 * h + 1], ci[4 * h + 2], ci[4 * h + 3]));
#pragma unroll
            for (int h = 0; h < SYM_ITEMS / 4; ++h)
                st_cs_v4d(tval + kb + 4 * h, v[4 * h], v[4 * h + 1], v[4 * h + 2], v[4 * h + 3]);
        } else {
#pragma unroll
            for (int j = 0; j < SYM_ITEMS; ++j)
                if (j < m) {
                    __stcs(trow + kb + j, ci[j]);
                    __stcs(tval + kb + j, v[j]);
                }
        }
        if (t + warps < n_tiles) load_win(lo_n, hi_n, w0, w1);
    }
    // once per warp (a few thousand warps: no single L2 slice saturates)
    wmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)max(wmax, 0));
    if (lane == 0 && wmax > 0) atomicMax(cnt + 2, (unsigned long long)wmax);
    if (__any_sync(0xffffffffu, redo) && lane == 0) atomicOr(status, ST_REDO);
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(status, ST_BAD_INDEX);
}

size_t ccs_sym_scratch_bytes(int64_t nnz) { return tile_lines_bytes(nnz, SYM_TILE); }

cudaError_t launch_ccs_sym(const int32_t *irp, int32_t n, const int32_t *icol, const double *val, int64_t nnz,
                           int32_t *scratch, int32_t *trow, double *tval, unsigned long long *cnt, int *status,
                           cudaStream_t s) {
    if (nnz <= 0) return cudaSuccess;
    if (nnz > INT_MAX) return cudaErrorInvalidValue;  // int32 row pointers bound nnz
    cudaError_t e = launch_tile_lines(irp, n, nnz, SYM_TILE, scratch, s);
    if (e != cudaSuccess) return e;
    const int n_tiles = (int)((nnz + SYM_TILE - 1) / SYM_TILE);
    // 16-byte loads of ICOL and stores of ICOL_T, 32-byte stores of VAL_T
    const bool vec = ((reinterpret_cast<uintptr_t>(icol) | reinterpret_cast<uintptr_t>(trow)) & 15u) == 0 &&
                     (reinterpret_cast<uintptr_t>(tval) & 31u) == 0;
    // the smallest shared-memory carveout that holds the resident CTAs (2 KB
    // each), so that the rest of the SM's 256 KB is L1, where the gathers of a
    // mirror row by its three neighbouring output rows meet; a cheap host
    // call, made before every launch like set_smem_attr
    e = vec ? cudaFuncSetAttribute(k_ccs_sym<true>, cudaFuncAttributePreferredSharedMemoryCarveout, 8)
            : cudaFuncSetAttribute(k_ccs_sym<false>, cudaFuncAttributePreferredSharedMemoryCarveout, 8);
    if (e != cudaSuccess) return e;
    const long long want = ((long long)n_tiles + SYM_WARPS - 1) / SYM_WARPS;
    const unsigned grid = (unsigned)std::min<long long>(want, (long long)sm_count() * SYM_CTAS_PER_SM);
    KernelScope ks("ccs_sym", s);
    if (vec)
        k_ccs_sym<true><<<grid, SYM_THREADS, 0, s>>>(irp, n, icol, val, (int32_t)nnz, scratch, n_tiles, trow, tval,
                                                     cnt, status);
    else
        k_ccs_sym<false><<<grid, SYM_THREADS, 0, s>>>(irp, n, icol, val, (int32_t)nnz, scratch, n_tiles, trow, tval,
                                                      cnt, status);
    return cudaGetLastError();
}

// Sample for the symmetric path: one entry (at a hashed position) of each of
// `samples` evenly spread rows (no search for the row of an entry: a handful
// of dependent loads); an
// entry counts as a failure when its column is out of range, the next entry
// of its row does not have a larger column, or its mirror (i, c) is missing.
// Empty rows are skipped. The count goes to *fails.
__global__ void __launch_bounds__(256) k_sym_sample(const int32_t *__restrict__ irp, int32_t n,
                                                     const int32_t *__restrict__ icol, int64_t nnz, int samples,
                                                     int32_t *__restrict__ fails) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    int fail = 0;
    if (s < samples) {
        const int c = (int)((long long)s * n / samples);
        const long long ra = min(max((long long)__ldg(irp + c), 0ll), (long long)nnz);
        const long long rb = min(max((long long)__ldg(irp + c + 1), ra), (long long)nnz);
        if (rb > ra) {
            // a spread entry of the row (not always the middle one, which in a
            // stencil is the diagonal, its own mirror)
            const long long p = ra + (long long)(((unsigned)s * 2654435761u) % (unsigned long long)(rb - ra));
            const int i = __ldg(icol + p);
            if ((unsigned)i >= (unsigned)n) {
                fail = 1;
            } else {
                if (p + 1 < rb && __ldg(icol + p + 1) <= i) fail = 1;
                const long long ma = min(max((long long)__ldg(irp + i), 0ll), (long long)nnz);
                const long long mb = min(max((long long)__ldg(irp + i + 1), ma), (long long)nnz);
                // the reflected guess first (as in k_ccs_sym), a search only if it misses
                const long long gq = mb - 1 - (p - ra);
                if (!(gq >= ma && __ldg(icol + gq) == c)) {
                    int l = (int)ma, h = (int)mb;
                    while (h - l > 1) {
                        const int m = l + ((h - l) >> 1);
                        if (__ldg(icol + m) <= c) l = m; else h = m;
                    }
                    if (!(l < (int)mb && __ldg(icol + l) == c)) fail = 1;
                }
            }
        }
    }
    fail = (int)__reduce_add_sync(0xffffffffu, (unsigned)fail);
    if (lane_id() == 0 && fail) atomicAdd(fails, fail);
}

cudaError_t launch_sym_sample(const int32_t *irp, int32_t n, const int32_t *icol, int64_t nnz, int samples,
                              int32_t *fails, cudaStream_t s) {
    if (nnz <= 0 || samples <= 0) return cudaSuccess;
    KernelScope ks("sym_sample", s);
    k_sym_sample<<<ceil_div_u(samples, 256), 256, 0, s>>>(irp, n, icol, nnz, samples, fails);
    return cudaGetLastError();
}

}  // namespace spmvat

