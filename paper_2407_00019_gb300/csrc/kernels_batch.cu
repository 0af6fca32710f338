// Batches of independent matrices: the row statistics of Eq. (4), the
// CRS -> ELL-Row transformation of Sec. 2.1 and the SpMV of Sec. 3, run for
// every matrix of a batch in one persistent launch each.
//
// Work items are row tiles of at most 32 rows that never cross a matrix,
// recorded as {matrix, first row, first entry, entries} and ordered by
// matrix; every warp of the persistent grid takes items w, w + (number of
// warps), ... and loads the record of its next item while it works on the
// current one. A matrix's descriptor says how its tiles run:
//  - CRS with short rows: the tile's n entries are contiguous, so the 32
//    lanes split them into equal runs of m = ceil(n / 32) (merge-path
//    split): lane j loads entries [j m, j m + m), their columns, then the x
//    values, and sums them with one FMA per entry. Rows that cross a run
//    boundary are closed by the lane that holds their start, adding the
//    other lanes' partial sums in lane order. Every FMA then runs on full
//    lanes: FP64 issue (2 FMA / clock / SM) is as scarce as HBM bandwidth
//    for SpMV on this GPU, and one lane per row would idle most lanes on
//    rows shorter than the longest in the warp;
//  - CRS with long rows: 8 or 32 lanes per row, partial sums combined by a
//    fixed butterfly;
//  - ELL-Row, one lane per row: slot k of consecutive rows is contiguous
//    (Fig. 3 layout), so each slot is one coalesced load.
#include <climits>

#include "common.cuh"

namespace spmvat {
namespace {

constexpr int T = kBatchThreads;

// ---- warp-level tiles of the product and build launches -------------------
// Every warp owns one tile; a CTA is 8 independent warps (no block barrier).
constexpr int WCAP = 256;  // entries a warp stages at once (8 per lane)
constexpr int WU = WCAP / 32;
constexpr int MMAX = 8;    // merge-path: entries per lane, so tiles of up to 256 entries
// Greedy tiles of several rows stop at 224 entries (m <= 7): lane j reads
// slot j * m + u of the shared arrays, and m = 8 would put 8 lanes on each
// bank; m = 5 and 7, the usual sizes, give at most 2.
constexpr int kTileCap = 224;
struct WarpSmem {          // staging of the ELL build and the long-tile product
    double v[WCAP];
    double xv[WCAP];       // x at the staged entries' columns, or their column indices
};
struct RowSmem {           // merge-path bookkeeping of one warp
    double run[32 * MMAX]; // running sum of each lane's run at each entry (reset after a row's last entry)
    uint32_t last[8];      // bit k: entry k is the last entry of its row
};
union BuildSmem {
    WarpSmem ws;
    RowSmem rs;
};

// Entries [c0, c0 + cn) of val / icol (cn <= WCAP) into the warp's shared
// memory; with GATHER also x at their columns. Every load of a phase is
// issued before its first use.
template <bool GATHER>
__device__ __forceinline__ void warp_stage(WarpSmem &ws, const double *__restrict__ val,
                                           const int32_t *__restrict__ icol, int c0, int cn,
                                           const double *__restrict__ x) {
    const int lane = (int)lane_id();
    double v[WU];
    int32_t c[WU];
#pragma unroll
    for (int u = 0; u < WU; ++u) {
        const int q = lane + 32 * u;
        v[u] = (q < cn) ? __ldcs(val + c0 + q) : 0.0;
        c[u] = (q < cn) ? __ldcs(icol + c0 + q) : 0;
    }
    if (GATHER) {
        double xv[WU];
#pragma unroll
        for (int u = 0; u < WU; ++u) xv[u] = (lane + 32 * u < cn) ? __ldg(x + c[u]) : 0.0;
#pragma unroll
        for (int u = 0; u < WU; ++u) {
            const int q = lane + 32 * u;
            if (q < cn) {
                ws.v[q] = v[u];
                ws.xv[q] = xv[u];
            }
        }
    } else {
        int32_t *sc = reinterpret_cast<int32_t *>(ws.xv);
#pragma unroll
        for (int u = 0; u < WU; ++u) {
            const int q = lane + 32 * u;
            if (q < cn) {
                ws.v[q] = v[u];
                sc[q] = c[u];
            }
        }
    }
    __syncwarp();
}

// CRS rows [row0, row0 + nr), nr <= 32 / V, V lanes per row: lane j of a
// row sums entries j, j + V, ... in storage order; the V partial sums are
// combined by a fixed butterfly.
template <int V>
__device__ __forceinline__ void vector_tile(const int32_t *__restrict__ irp, const int32_t *__restrict__ icol,
                                            const double *__restrict__ val, int row0, int nr,
                                            const double *__restrict__ x, double *__restrict__ y) {
    const int lane = (int)lane_id(), sub = lane / V, j = lane % V;
    double acc = 0.0;
    if (sub < nr) {
        const int a = __ldg(irp + row0 + sub), b = __ldg(irp + row0 + sub + 1);
        int k = a + j;
        for (; k + 3 * V < b; k += 4 * V) {
            const int32_t c0 = __ldcs(icol + k), c1 = __ldcs(icol + k + V), c2 = __ldcs(icol + k + 2 * V),
                          c3 = __ldcs(icol + k + 3 * V);
            const double v0 = __ldcs(val + k), v1 = __ldcs(val + k + V), v2 = __ldcs(val + k + 2 * V),
                         v3 = __ldcs(val + k + 3 * V);
            const double x0 = __ldg(x + c0), x1 = __ldg(x + c1), x2 = __ldg(x + c2), x3 = __ldg(x + c3);
            acc = fma(v0, x0, acc);
            acc = fma(v1, x1, acc);
            acc = fma(v2, x2, acc);
            acc = fma(v3, x3, acc);
        }
        for (; k < b; k += V) acc = fma(__ldcs(val + k), __ldg(x + __ldcs(icol + k)), acc);
    }
#pragma unroll
    for (int o = V / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (j == 0 && sub < nr) y[row0 + sub] = acc;
}

// A lane's run of M entries: running sum in storage order, one FMA per
// entry, restarted after each row's last entry (bit u of `ends`).
template <int M>
__device__ __forceinline__ void run_fma(const double (&v)[MMAX], const double (&xv)[MMAX], int beg, int end,
                                        uint32_t ends, double *run) {
    double s = 0.0;
#pragma unroll
    for (int u = 0; u < M; ++u) {
        if (beg + u < end) {
            s = fma(v[u], xv[u], s);
            run[beg + u] = s;
            if ((ends >> u) & 1u) s = 0.0;
        }
    }
}

// The arithmetic of a merge-path tile (see the top of this file): lane j
// holds the values v and x values xv of its run [beg, end) of the tile's n
// entries (m = ceil(n / 32) per lane); lane r < nr holds the start rb and end
// re of row r relative to the tile's first entry. Lane j sums its run with
// one FMA per entry, restarting after each row's last entry, and leaves the
// running sums in run[]; lane r then adds row r's pieces in lane order and
// writes yr[r]. Each row is thus summed in storage order with one extra
// addition per run boundary it crosses.
//
// merge_ends marks each row's last entry (a bitmap in `last`) and returns the
// bits of the lane's own run; merge_run sums and assembles one product.
__device__ __forceinline__ uint32_t merge_ends(uint32_t *last, int beg, int nr, int rb, int re) {
    const int lane = (int)lane_id();
    if (lane < 8) last[lane] = 0u;
    __syncwarp();
    if (lane < nr && re > rb) atomicOr(&last[(re - 1) >> 5], 1u << ((re - 1) & 31));
    __syncwarp();
    // bits beg .. beg + m - 1 of the last-entry map (m <= 8: at most two words)
    const int w0 = beg >> 5, sh = beg & 31;
    uint64_t two = last[min(w0, 7)];
    if (w0 + 1 < 8) two |= (uint64_t)last[w0 + 1] << 32;
    return (uint32_t)(two >> sh);
}

__device__ __forceinline__ void merge_run(double *run, int m, int beg, int end, int nr, int rb, int re, uint32_t ends,
                                          const double (&v)[MMAX], const double (&xv)[MMAX],
                                          double *__restrict__ yr) {
    const int lane = (int)lane_id();
    // exactly m steps: an FP64 instruction whose lanes are all switched off
    // still takes its issue slot on the (narrow) FP64 pipe
    switch (m) {
        case 1: run_fma<1>(v, xv, beg, end, ends, run); break;
        case 2: run_fma<2>(v, xv, beg, end, ends, run); break;
        case 3: run_fma<3>(v, xv, beg, end, ends, run); break;
        case 4: run_fma<4>(v, xv, beg, end, ends, run); break;
        case 5: run_fma<5>(v, xv, beg, end, ends, run); break;
        case 6: run_fma<6>(v, xv, beg, end, ends, run); break;
        case 7: run_fma<7>(v, xv, beg, end, ends, run); break;
        case 8: run_fma<8>(v, xv, beg, end, ends, run); break;
        default: break;
    }
    __syncwarp();
    if (lane < nr) {
        double t = 0.0;
        if (re > rb) {
            const int j0 = rb / m, j1 = (re - 1) / m;
            t = run[min(re, (j0 + 1) * m) - 1];
            for (int j = j0 + 1; j <= j1; ++j) t += run[min(re, (j + 1) * m) - 1];
        }
        yr[lane] = t;
    }
    __syncwarp();
}

__device__ __forceinline__ void merge_sum(uint32_t *last, double *run, int m, int beg, int end, int nr, int rb,
                                          int re, const double (&v)[MMAX], const double (&xv)[MMAX],
                                          double *__restrict__ yr) {
    const uint32_t ends = merge_ends(last, beg, nr, rb, re);
    merge_run(run, m, beg, end, nr, rb, re, ends, v, xv, yr);
}

// Row bounds of a tile relative to its first entry e0: lane r < nr gets the
// start and end of row r.
__device__ __forceinline__ void tile_bounds(const int32_t *__restrict__ irp, int row0, int nr, int e0, int n,
                                            int *rb, int *re) {
    const int lane = (int)lane_id();
    *rb = 0;
    *re = 0;
    if (lane < nr) {
        *rb = __ldg(irp + row0 + lane) - e0;
        *re = lane + 1 < nr ? __ldg(irp + row0 + lane + 1) - e0 : n;
    }
}

// CRS rows [row0, row0 + nr) whose n <= 32 * MMAX entries start at entry e0,
// loaded straight into registers.
__device__ __forceinline__ void merge_tile(RowSmem &rs, const int32_t *__restrict__ irp,
                                           const int32_t *__restrict__ icol, const double *__restrict__ val,
                                           int row0, int nr, int e0, int n, const double *__restrict__ x,
                                           double *__restrict__ y) {
    const int lane = (int)lane_id();
    const int m = (n + 31) >> 5;  // warp-uniform
    const int beg = min(n, lane * m), end = min(n, beg + m);
    const double *vp = val + e0 + beg;
    const int32_t *cp = icol + e0 + beg;
    double v[MMAX], xv[MMAX];
    int32_t c[MMAX];
#pragma unroll
    for (int u = 0; u < MMAX; ++u) {
        v[u] = 0.0;
        c[u] = 0;
        if (u < m && beg + u < end) {
            v[u] = __ldcs(vp + u);
            c[u] = __ldcs(cp + u);
        }
    }
    int rb, re;
    tile_bounds(irp, row0, nr, e0, n, &rb, &re);
#pragma unroll
    for (int u = 0; u < MMAX; ++u) xv[u] = (u < m && beg + u < end) ? __ldg(x + c[u]) : 0.0;
    merge_sum(rs.last, rs.run, m, beg, end, nr, rb, re, v, xv, y + row0);
}

// A CRS tile of one lane per entry with more than 32 * MMAX entries: by
// construction a single row, summed by the whole warp.
__device__ __forceinline__ void long_rows(const int32_t *__restrict__ irp, const int32_t *__restrict__ icol,
                                          const double *__restrict__ val, int row0, int nr,
                                          const double *__restrict__ x, double *__restrict__ y) {
    for (int r = 0; r < nr; ++r) vector_tile<32>(irp, icol, val, row0 + r, 1, x, y);
}

// ELL-Row rows [row0, row0 + nr), nr <= 32, one lane per row, slots summed in
// slot order (padding slots included, as in the single-matrix ELL-Row SpMV).
__device__ __forceinline__ void ell_tile(const double *__restrict__ ev, const int32_t *__restrict__ ec, int ld,
                                         int width, int row0, int nr, const double *__restrict__ x,
                                         double *__restrict__ y) {
    const int r = (int)lane_id();
    if (r >= nr) return;
    const double *pv = ev + row0 + r;
    const int32_t *pc = ec + row0 + r;
    const size_t L = (size_t)ld;
    double acc = 0.0;
    int k = 0;
    for (; k + 4 <= width; k += 4) {
        const int32_t c0 = __ldcs(pc + k * L), c1 = __ldcs(pc + (k + 1) * L), c2 = __ldcs(pc + (k + 2) * L),
                      c3 = __ldcs(pc + (k + 3) * L);
        const double v0 = __ldcs(pv + k * L), v1 = __ldcs(pv + (k + 1) * L), v2 = __ldcs(pv + (k + 2) * L),
                     v3 = __ldcs(pv + (k + 3) * L);
        const double x0 = __ldg(x + c0), x1 = __ldg(x + c1), x2 = __ldg(x + c2), x3 = __ldg(x + c3);
        acc = fma(v0, x0, acc);
        acc = fma(v1, x1, acc);
        acc = fma(v2, x2, acc);
        acc = fma(v3, x3, acc);
    }
    for (; k < width; ++k) acc = fma(__ldcs(pv + k * L), __ldg(x + __ldcs(pc + k * L)), acc);
    y[row0 + r] = acc;
}

// CRS rows [row0, row0 + nr) -> ELL-Row slots (Sec. 2.1, Fig. 3): slot k of
// row i at k * ld + i; padding slots get value +0.0 and the row's last column
// (0 for an empty row). With MUL, also y for these rows in ELL slot order
// (the order of ell_tile, so the results agree bit for bit).
template <bool MUL>
__device__ __forceinline__ void ell_build_tile(WarpSmem &ws, const BatchMat *__restrict__ M, int row0, int nr,
                                               const double *__restrict__ x, double *__restrict__ y) {
    const int32_t *irp = M->irp, *icol = M->icol;
    const double *val = M->val;
    const int lane = (int)lane_id();
    int a = 0, b = 0;
    if (lane < nr) {
        a = __ldg(irp + row0 + lane);
        b = __ldg(irp + row0 + lane + 1);
    }
    const int e0 = __shfl_sync(0xffffffffu, a, 0), e1 = __shfl_sync(0xffffffffu, b, nr - 1);
    const bool staged = e1 - e0 <= WCAP;
    if (staged) warp_stage<false>(ws, val, icol, e0, e1 - e0, nullptr);
    if (lane < nr) {
        const int len = b - a;
        const double *sv = staged ? ws.v + (a - e0) : val + a;
        const int32_t *sc = staged ? reinterpret_cast<const int32_t *>(ws.xv) + (a - e0) : icol + a;
        const int32_t last = len > 0 ? sc[len - 1] : 0;
        const int width = M->width;
        const size_t L = (size_t)M->ld;
        double *pv = M->eval + row0 + lane;
        int32_t *pc = M->ecol + row0 + lane;
        double acc = 0.0;
        for (int k = 0; k < width; ++k) {
            const bool real = k < len;
            const double v = real ? sv[k] : 0.0;
            const int32_t c = real ? sc[k] : last;
            __stcs(pv + k * L, v);
            __stcs(pc + k * L, c);
            if (MUL) acc = fma(v, __ldg(x + c), acc);
        }
        if (MUL) y[row0 + lane] = acc;
    }
    __syncwarp();
}

// One CRS tile of matrix M by its schedule: rows [row0, row0 + nr), entries
// [e0, e0 + n).
__device__ __forceinline__ void crs_tile(RowSmem &rs, const BatchMat *__restrict__ M, int row0, int nr, int e0,
                                         int n, const double *x, double *y) {
    const int32_t *irp = M->irp, *icol = M->icol;
    const double *val = M->val;
    switch (M->tpr) {
        case 8: vector_tile<8>(irp, icol, val, row0, nr, x, y); break;
        case 32: vector_tile<32>(irp, icol, val, row0, nr, x, y); break;
        default:
            if (n <= 32 * MMAX) merge_tile(rs, irp, icol, val, row0, nr, e0, n, x, y);
            else long_rows(irp, icol, val, row0, nr, x, y);
            break;
    }
}

__global__ void __launch_bounds__(T) k_batch_analyze(const BatchMat *__restrict__ mats,
                                                     const int2 *__restrict__ chunks, long long n_chunks,
                                                     BatchAcc *__restrict__ acc) {
    __shared__ unsigned long long s_a[T / 32], s_b[T / 32];
    __shared__ int s_mx[T / 32], s_mn[T / 32], s_em[T / 32];
    for (long long ci = blockIdx.x; ci < n_chunks; ci += gridDim.x) {
        const int2 ch = __ldg(chunks + ci);
        const BatchMat *M = mats + ch.x;
        const int n = M->n_rows;
        const long long nnz = M->nnz;
        const int32_t *irp = M->irp;
        const int r0 = ch.y, nr = min(kBatchChunk, n - r0);
        unsigned long long s1 = 0, s2 = 0;
        int mx = 0, mn = 0, em = 0, bad = 0;
        for (int i = threadIdx.x; i < nr; i += T) {
            const int a = __ldg(irp + r0 + i), b = __ldg(irp + r0 + i + 1);
            if (a < 0 || b < a || (long long)b > nnz) {
                bad = 1;
            } else {
                const int len = b - a;
                s1 += (unsigned long long)len;
                s2 += (unsigned long long)len * (unsigned long long)len;
                mx = max(mx, len);
                mn = max(mn, INT_MAX - len);
                em += (len == 0);
            }
        }
        if (threadIdx.x == 0) {
            if (r0 == 0 && __ldg(irp) != 0) bad = 1;
            if (r0 + nr == n && (long long)__ldg(irp + n) != nnz) bad = 1;
        }
        bad = __syncthreads_or(bad);
        unsigned badidx = 0;
        if (!bad && nnz > 0) {
            // the chunk's entries: [irp[r0], irp[r0 + nr]) lies in [0, nnz] here
            const int ea = __ldg(irp + r0), eb = __ldg(irp + r0 + nr);
            const int32_t *icol = M->icol;
            const unsigned nc = (unsigned)M->n_cols;
            for (int k = ea + (int)threadIdx.x; k < eb; k += T) badidx |= (unsigned)__ldcs(icol + k) >= nc;
        }
        s1 = warp_sum(s1);
        s2 = warp_sum(s2);
        mx = __reduce_max_sync(0xffffffffu, mx);
        mn = __reduce_max_sync(0xffffffffu, mn);
        em = __reduce_add_sync(0xffffffffu, em);
        const int w = threadIdx.x >> 5;
        if (lane_id() == 0) {
            s_a[w] = s1;
            s_b[w] = s2;
            s_mx[w] = mx;
            s_mn[w] = mn;
            s_em[w] = em;
        }
        const int anybad = __syncthreads_or((int)badidx);
        if (threadIdx.x == 0) {
            unsigned long long a = 0, b = 0;
            int x1 = 0, x2 = 0, e = 0;
            for (int j = 0; j < T / 32; ++j) {
                a += s_a[j];
                b += s_b[j];
                x1 = max(x1, s_mx[j]);
                x2 = max(x2, s_mn[j]);
                e += s_em[j];
            }
            BatchAcc *A = acc + ch.x;
            atomicAdd(&A->sum_len, a);
            atomicAdd(&A->sum_len2, b);
            atomicMax(&A->max_len, x1);
            atomicMax(&A->min_len, x2);
            atomicAdd(&A->n_empty, e);
            if (bad) atomicOr(&A->status, ST_BAD_PTR);
            if (anybad) atomicOr(&A->status, ST_BAD_INDEX);
        }
        __syncthreads();
    }
}

// .x of a tile record: the matrix index (below 2^26) and the row count
// (1..32, stored minus one in the top bits).
__device__ __forceinline__ int tile_key(int mat, int nr) { return mat | ((nr - 1) << kBatchMatBits); }
__device__ __forceinline__ int tile_mat(int key) { return key & ((1 << kBatchMatBits) - 1); }
__device__ __forceinline__ int tile_rows(int key) { return (int)((unsigned)key >> kBatchMatBits) + 1; }

// Tiles of every matrix, one warp per matrix, in row order. CRS matrices
// with one lane per entry: greedy runs of whole rows, at most 32 rows and
// kTileCap entries each (a longer row is a tile of its own: a merge tile up
// to 32 * MMAX entries, else summed by the whole warp). Other matrices: rpt rows per tile. Without FILL, writes the
// tile count of each matrix to cnt[i]; with FILL, writes the records
// {matrix, first row, first entry, entries} from tiles[cnt[i]] on.
template <bool FILL>
__global__ void __launch_bounds__(T) k_batch_tiles(const BatchMat *__restrict__ mats, int m,
                                                   long long *__restrict__ cnt, int4 *__restrict__ tiles,
                                                   const long long *__restrict__ d_nt) {
    if (FILL && d_nt && *d_nt == 0) return;  // planned on the device: no records, or more than allocated
    const int lane = (int)lane_id();
    const int nwarps = (int)(gridDim.x * (T / 32));
    for (int i = (int)(blockIdx.x * (T / 32) + (threadIdx.x >> 5)); i < m; i += nwarps) {
        const BatchMat *M = mats + i;
        const int n = M->n_rows;
        const int32_t *irp = M->irp;
        const long long out = FILL ? cnt[i] : 0;
        long long count = 0;
        if (M->fmt == BATCH_CRS && M->tpr == 1) {
            int r = 0;
            while (r < n) {
                const int rows = min(32, n - r);
                const int e0 = __ldg(irp + r);
                const int end_l = lane < rows ? __ldg(irp + r + lane + 1) : INT_MAX;
                const unsigned fit = __ballot_sync(0xffffffffu, lane < rows && end_l - e0 <= kTileCap);
                const int k = max(1, __popc(fit));  // row ends grow with the lane: rows r .. r + k - 1 fit
                const int e1 = __shfl_sync(0xffffffffu, end_l, k - 1);
                if (FILL && lane == 0) tiles[out + count] = make_int4(tile_key(i, k), r, e0, e1 - e0);
                ++count;
                r += k;
            }
        } else {
            const int rpt = M->rpt;
            count = (n + rpt - 1) / rpt;
            if (FILL) {
                for (long long k = lane; k < count; k += 32) {
                    const int r = (int)k * rpt, nr = min(rpt, n - r);
                    const int a = __ldg(irp + r), b = __ldg(irp + r + nr);
                    tiles[out + k] = make_int4(tile_key(i, nr), r, a, b - a);
                }
            }
        }
        if (!FILL && lane == 0) cnt[i] = count;
    }
}

template <bool MUL>
__global__ void __launch_bounds__(T) k_batch_build(const BatchMat *__restrict__ mats, const int4 *__restrict__ tiles,
                                                   long long n_tiles, const long long *__restrict__ d_nt,
                                                   const double *__restrict__ x, double *__restrict__ y) {
    if (d_nt) n_tiles = *d_nt;  // a batch planned on the device
    __shared__ BuildSmem sm_all[T / 32];  // a warp uses one member per tile
    WarpSmem &ws = sm_all[threadIdx.x >> 5].ws;
    RowSmem &rs = sm_all[threadIdx.x >> 5].rs;
    const long long nw = (long long)gridDim.x * (T / 32);
    for (long long t = (long long)blockIdx.x * (T / 32) + (threadIdx.x >> 5); t < n_tiles; t += nw) {
        const int4 tl = __ldg(tiles + t);
        const BatchMat *M = mats + tile_mat(tl.x);
        const int nr = tile_rows(tl.x);
        const double *xm = MUL ? x + M->xoff : nullptr;
        double *ym = MUL ? y + M->yoff : nullptr;
        if (M->fmt == BATCH_ELL) ell_build_tile<MUL>(ws, M, tl.y, nr, xm, ym);
        else if (MUL) crs_tile(rs, M, tl.y, nr, tl.z, tl.w, xm, ym);
    }
}

// ---- the product launch: merge-path tiles double-buffered with cp.async ----
constexpr int AT = 128;  // threads per CTA of the product launch
struct PipeSmem {        // one warp: two stages of tile entries
    double v[2][WCAP];   // values; a lane's run sums later overwrite its own entries
    int32_t c[2][WCAP];  // column indices
    uint32_t last[8];
};


__device__ __forceinline__ bool is_merge(const BatchMat *__restrict__ M, int n) {
    return M->fmt == BATCH_CRS && M->tpr == 1 && n <= 32 * MMAX;
}

// Copies of a merge tile's n entries from e0 into stage st, coalesced (lane
// q copies entries q, q + 32, ...).
__device__ __forceinline__ void stage_issue(PipeSmem &ps, int st, const BatchMat *__restrict__ M, int e0, int n) {
    const double *val = M->val + e0;
    const int32_t *icol = M->icol + e0;
    for (int q = (int)lane_id(); q < n; q += 32) {
        cp_async_8(&ps.v[st][q], val + q);
        cp_async_4(&ps.c[st][q], icol + q);
    }
}

// Every warp walks its tiles; the entries of its next merge tile are copied
// into the other stage while it works on the current one, so only the x
// gathers (and the row bounds, loaded alongside) wait on memory.
__global__ void __launch_bounds__(AT) k_batch_apply(const BatchMat *__restrict__ mats, const int4 *__restrict__ tiles,
                                                    long long n_tiles, const long long *__restrict__ d_nt,
                                                    const double *__restrict__ x, double *__restrict__ y) {
    if (d_nt) n_tiles = *d_nt;  // a batch planned on the device
    __shared__ PipeSmem ps_all[AT / 32];
    PipeSmem &ps = ps_all[threadIdx.x >> 5];
    const int lane = (int)lane_id();
    const long long nw = (long long)gridDim.x * (AT / 32);
    long long t = (long long)blockIdx.x * (AT / 32) + (threadIdx.x >> 5);
    if (t >= n_tiles) return;
    int4 cur = __ldg(tiles + t);
    if (is_merge(mats + tile_mat(cur.x), cur.w)) stage_issue(ps, 0, mats + tile_mat(cur.x), cur.z, cur.w);
    cp_async_commit();
    int4 nxt = t + nw < n_tiles ? __ldg(tiles + t + nw) : cur;
    for (int it = 0; t < n_tiles; t += nw, ++it) {
        const int st = it & 1;
        if (t + nw < n_tiles && is_merge(mats + tile_mat(nxt.x), nxt.w))
            stage_issue(ps, st ^ 1, mats + tile_mat(nxt.x), nxt.z, nxt.w);
        cp_async_commit();
        const int4 after = t + 2 * nw < n_tiles ? __ldg(tiles + t + 2 * nw) : nxt;
        const BatchMat *M = mats + tile_mat(cur.x);
        const int nr = tile_rows(cur.x);
        const double *xm = x + M->xoff;
        double *ym = y + M->yoff;
        if (M->fmt == BATCH_ELL) {
            ell_tile(M->eval, M->ecol, M->ld, M->width, cur.y, nr, xm, ym);
        } else if (is_merge(M, cur.w)) {
            const int n = cur.w, m = (n + 31) >> 5;
            const int beg = min(n, lane * m), end = min(n, beg + m);
            int rb, re;
            tile_bounds(M->irp, cur.y, nr, cur.z, n, &rb, &re);
            cp_async_wait_prev();  // this tile's copies (all groups but the newest)
            __syncwarp();
            double v[MMAX], xv[MMAX];
#pragma unroll
            for (int u = 0; u < MMAX; ++u) {
                const bool ok = u < m && beg + u < end;
                const int32_t c = ok ? ps.c[st][beg + u] : 0;
                xv[u] = ok ? __ldg(xm + c) : 0.0;
                v[u] = ok ? ps.v[st][beg + u] : 0.0;
            }
            merge_sum(ps.last, ps.v[st], m, beg, end, nr, rb, re, v, xv, ym + cur.y);
        } else {
            const int32_t *irp = M->irp, *icol = M->icol;
            const double *val = M->val;
            if (M->tpr == 8) vector_tile<8>(irp, icol, val, cur.y, nr, xm, ym);
            else if (M->tpr == 32) vector_tile<32>(irp, icol, val, cur.y, nr, xm, ym);
            else long_rows(irp, icol, val, cur.y, nr, xm, ym);
        }
        cur = nxt;
        nxt = after;
    }
    cp_async_wait_all();
}

// ---- several products per launch: y_j = A x_j, j < nvec ------------------
// Work items are (tile, vector) pairs, tile-major, dealt round robin to the
// warps: the nvec products of one tile run on neighbouring warps at the same
// time, so the tile's entries come from DRAM once and from L1/L2 for the
// other vectors, and a request with few tiles still fills the GPU. Each item
// runs exactly the arithmetic of k_batch_apply, so every product has the same
// bits as a single-product launch. Vector j of the concatenated x starts at
// x + j * ldx, of y at y + j * ldy.
__global__ void __launch_bounds__(AT) k_batch_apply_multi(const BatchMat *__restrict__ mats,
                                                          const int4 *__restrict__ tiles, long long n_tiles,
                                                          const long long *__restrict__ d_nt,
                                                          const double *__restrict__ x, long long ldx,
                                                          double *__restrict__ y, long long ldy, int nvec) {
    if (d_nt) n_tiles = *d_nt;  // a batch planned on the device
    __shared__ RowSmem rs_all[AT / 32];
    RowSmem &rs = rs_all[threadIdx.x >> 5];
    const long long nw = (long long)gridDim.x * (AT / 32);
    const long long n_items = n_tiles * nvec;
    for (long long it = (long long)blockIdx.x * (AT / 32) + (threadIdx.x >> 5); it < n_items; it += nw) {
        const long long t = it / nvec;
        const int j = (int)(it - t * nvec);
        const int4 tl = __ldg(tiles + t);
        const BatchMat *M = mats + tile_mat(tl.x);
        const int nr = tile_rows(tl.x);
        const double *xm = x + j * ldx + M->xoff;
        double *ym = y + j * ldy + M->yoff;
        if (M->fmt == BATCH_ELL) ell_tile(M->eval, M->ecol, M->ld, M->width, tl.y, nr, xm, ym);
        else crs_tile(rs, M, tl.y, nr, tl.z, tl.w, xm, ym);
    }
}

int g_grid[64][5] = {};

}  // namespace

int batch_grid(int kernel) {
    int dev = 0;
    cudaGetDevice(&dev);
    int &g = g_grid[dev & 63][kernel % 5];
    if (!g) {
        int occ = 0;
        cudaError_t e = cudaErrorInvalidValue;
        switch (kernel) {
            case 0: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_analyze, T, 0); break;
            case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_build<false>, T, 0); break;
            case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_build<true>, T, 0); break;
            case 3: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_apply, AT, 0); break;
            default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_apply_multi, AT, 0); break;
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            occ = 1;
        }
        g = (occ > 0 ? occ : 1) * sm_count();
    }
    return g;
}

cudaError_t launch_batch_analyze(const BatchMat *mats, const int2 *chunks, long long n_chunks, BatchAcc *acc,
                                 cudaStream_t s) {
    if (n_chunks <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)std::min<long long>(n_chunks, batch_grid(0));
    KernelScope ks("batch_analyze", s);
    k_batch_analyze<<<grid, T, 0, s>>>(mats, chunks, n_chunks, acc);
    return cudaGetLastError();
}

cudaError_t launch_batch_tiles(const BatchMat *mats, int m, long long *cnt, int4 *tiles, cudaStream_t s,
                               const long long *d_nt) {
    if (m <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)std::min<long long>((m + T / 32 - 1) / (T / 32), (long long)sm_count() * 8);
    if (tiles) {
        KernelScope ks("batch_tiles", s);
        k_batch_tiles<true><<<grid, T, 0, s>>>(mats, m, cnt, tiles, d_nt);
    } else {
        KernelScope ks("batch_tile_count", s);
        k_batch_tiles<false><<<grid, T, 0, s>>>(mats, m, cnt, nullptr, nullptr);
    }
    return cudaGetLastError();
}

cudaError_t launch_batch_build(const BatchMat *mats, const int4 *tiles, long long n_tiles, const double *x,
                               double *y, cudaStream_t s, const long long *d_nt) {
    if (n_tiles <= 0) return cudaSuccess;
    if (x) {
        const unsigned grid = (unsigned)std::min<long long>(n_tiles, batch_grid(2));
        KernelScope ks("batch_build_apply", s);
        k_batch_build<true><<<grid, T, 0, s>>>(mats, tiles, n_tiles, d_nt, x, y);
    } else {
        const unsigned grid = (unsigned)std::min<long long>(n_tiles, batch_grid(1));
        KernelScope ks("batch_build", s);
        k_batch_build<false><<<grid, T, 0, s>>>(mats, tiles, n_tiles, d_nt, nullptr, nullptr);
    }
    return cudaGetLastError();
}

cudaError_t launch_batch_apply(const BatchMat *mats, const int4 *tiles, long long n_tiles, const double *x,
                               double *y, cudaStream_t s, const long long *d_nt) {
    if (n_tiles <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)std::min<long long>((n_tiles + AT / 32 - 1) / (AT / 32), batch_grid(3));
    KernelScope ks("batch_apply", s);
    k_batch_apply<<<grid, AT, 0, s>>>(mats, tiles, n_tiles, d_nt, x, y);
    return cudaGetLastError();
}

}  // namespace spmvat

namespace spmvat {

cudaError_t launch_batch_apply_multi(const BatchMat *mats, const int4 *tiles, long long n_tiles, const double *x,
                                     long long ldx, double *y, long long ldy, int nvec, cudaStream_t s,
                                     const long long *d_nt) {
    if (n_tiles <= 0 || nvec <= 0) return cudaSuccess;
    if (nvec == 1) return launch_batch_apply(mats, tiles, n_tiles, x, y, s, d_nt);
    const unsigned grid = (unsigned)std::min<long long>((n_tiles + AT / 32 - 1) / (AT / 32), batch_grid(4));
    KernelScope ks("batch_apply_multi", s);
    k_batch_apply_multi<<<grid, AT, 0, s>>>(mats, tiles, n_tiles, d_nt, x, ldx, y, ldy, nvec);
    return cudaGetLastError();
}

// ------------------------------------------------- plan on the device
// The build of a batch without host work between its launches (so that one
// CUDA graph can hold it): the on-line rule of Sec. 2.2 per matrix, the ELL
// arrays placed in a pool allocated beforehand, and the tile records counted,
// offset and written by kernels.
//
// k_batch_plan (one CTA): Eq. (4) per matrix from the analysis sums (the
// numerator of sigma^2 exact in 128-bit integers, as on the host); ELL-Row
// iff D_mat < D* and the ELL arrays of the matrices chosen before it, in
// matrix order, plus its own fit the cap (a block-wide scan of the
// candidates' bytes; only if they do not all fit, one thread takes them in
// order and skips those that do not fit); then the descriptors (format,
// width, leading dimension, ELL pointers into the pool, and for ELL members
// one lane per row in 32-row tiles; CRS members keep the lanes per row the
// host set from the schedule table) and the plan records for the host.
constexpr int PLAN_T = 1024;
constexpr unsigned long long kCand = 1ull << 63;  // flag: the rule picks ELL-Row (bytes below it)

__device__ unsigned long long block_excl_scan_u64(unsigned long long v, unsigned long long *s_w,
                                                  unsigned long long *total) {
    const int lane = (int)lane_id(), w = (int)(threadIdx.x >> 5);
    unsigned long long inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) s_w[w] = inc;
    __syncthreads();
    unsigned long long pre = 0, tot = 0;
    for (int j = 0; j < PLAN_T / 32; ++j) {
        if (j < w) pre += s_w[j];
        tot += s_w[j];
    }
    __syncthreads();
    *total = tot;
    return pre + inc - v;
}

__global__ void __launch_bounds__(PLAN_T) k_batch_plan(BatchMat *__restrict__ mats, const BatchAcc *__restrict__ acc,
                                                       int m, double dstar, unsigned long long cap,
                                                       unsigned char *__restrict__ pool,
                                                       unsigned long long *__restrict__ bytes,
                                                       BatchPlanOut *__restrict__ plans,
                                                       unsigned long long *__restrict__ tot, int *status) {
    __shared__ unsigned long long s_w[PLAN_T / 32];
    __shared__ int s_greedy;
    int bad = 0;
    // statistics and the candidates' ELL bytes
    for (int i = threadIdx.x; i < m; i += PLAN_T) {
        const BatchAcc a = acc[i];
        const BatchMat &D = mats[i];
        BatchPlanOut P;
        const int st = a.status;
        if (st) bad |= st;
        if ((long long)a.sum_len != D.nnz) bad |= ST_BAD_PTR;
        const double n = (double)D.n_rows;
        const unsigned __int128 num = (unsigned __int128)(unsigned long long)D.n_rows * a.sum_len2 -
                                      (unsigned __int128)a.sum_len * a.sum_len;
        P.mu = (double)a.sum_len / n;
        P.sigma = sqrt((double)num) / n;
        P.dmat = a.sum_len == 0 ? 0.0 : P.sigma / P.mu;
        P.max_row_len = a.max_len;
        plans[i] = P;
        const unsigned long long eb = (unsigned long long)((D.n_rows + 31) / 32 * 32) * (unsigned long long)a.max_len * 12ull;
        bytes[i] = (P.dmat < dstar) ? (kCand | eb) : 0ull;  // a candidate may need 0 bytes (no entries)
    }
    if (bad) atomicOr(status, bad);
    __syncthreads();
    // matrix-order offsets of the candidates
    unsigned long long carry = 0;
    for (int base = 0; base < m; base += PLAN_T) {
        const int i = base + (int)threadIdx.x;
        const unsigned long long v = i < m ? (bytes[i] & ~kCand) : 0ull;
        unsigned long long t = 0;
        const unsigned long long ex = block_excl_scan_u64(v, s_w, &t);
        if (i < m) bytes[m + i] = carry + ex;  // offset if every candidate before it is taken
        carry += t;
    }
    if (threadIdx.x == 0) s_greedy = carry > cap;
    __syncthreads();
    if (s_greedy && threadIdx.x == 0) {
        // the cap binds: candidates in matrix order, each taken if it still fits
        unsigned long long used = 0;
        for (int i = 0; i < m; ++i) {
            const unsigned long long eb = bytes[i] & ~kCand;
            if ((bytes[i] & kCand) && used + eb <= cap) {
                bytes[m + i] = used;
                used += eb;
            } else {
                bytes[i] = 0;
            }
        }
    }
    __syncthreads();
    unsigned long long n_ell = 0, ell_bytes = 0;
    for (int i = threadIdx.x; i < m; i += PLAN_T) {
        BatchMat &D = mats[i];
        const BatchPlanOut &P = plans[i];
        const unsigned long long eb = bytes[i] & ~kCand;
        if (bytes[i] & kCand) {
            D.fmt = BATCH_ELL;
            D.width = P.max_row_len;
            D.ld = (D.n_rows + 31) / 32 * 32;
            D.tpr = 1;
            D.rpt = 32;
            unsigned char *b = pool + bytes[m + i];
            D.eval = reinterpret_cast<double *>(b);
            D.ecol = reinterpret_cast<int32_t *>(b + (unsigned long long)D.ld * D.width * 8ull);
            n_ell += 1;
            ell_bytes += eb;
        } else {
            D.fmt = BATCH_CRS;
            D.width = D.ld = 0;
            D.eval = nullptr;
            D.ecol = nullptr;
        }
    }
    n_ell = warp_sum(n_ell);
    ell_bytes = warp_sum(ell_bytes);
    if (lane_id() == 0 && n_ell) {
        atomicAdd(tot, n_ell);
        atomicAdd(tot + 1, ell_bytes);
    }
}

// Exclusive scan of the per-matrix tile counts in place; the total into
// *n_tiles. A total above `cap` (the records allocated) sets ST_REDO and
// leaves *n_tiles = 0, so that no later launch writes or reads past them; so
// does a malformed member.
__global__ void __launch_bounds__(PLAN_T) k_batch_tile_offsets(long long *__restrict__ cnt, int m, long long cap,
                                                               long long *__restrict__ n_tiles, int *status) {
    __shared__ unsigned long long s_w[PLAN_T / 32];
    unsigned long long carry = 0;
    for (int base = 0; base < m; base += PLAN_T) {
        const int i = base + (int)threadIdx.x;
        const unsigned long long v = i < m ? (unsigned long long)cnt[i] : 0ull;
        unsigned long long t = 0;
        const unsigned long long ex = block_excl_scan_u64(v, s_w, &t);
        if (i < m) cnt[i] = (long long)(carry + ex);
        carry += t;
    }
    if (threadIdx.x == 0) {
        // a malformed member (reported by the plan) or more records than
        // allocated: no records, so the later launches do nothing
        const bool malformed = (*status & (ST_BAD_PTR | ST_BAD_INDEX)) != 0;
        const bool over = (long long)carry > cap;
        *n_tiles = (over || malformed) ? 0 : (long long)carry;
        if (over) atomicOr(status, ST_REDO);
    }
}

cudaError_t launch_batch_plan(BatchMat *mats, const BatchAcc *acc, int m, double dstar, unsigned long long cap,
                              unsigned char *pool, unsigned long long *bytes, BatchPlanOut *plans,
                              unsigned long long *tot, int *status, cudaStream_t s) {
    KernelScope ks("batch_plan", s);
    k_batch_plan<<<1, PLAN_T, 0, s>>>(mats, acc, m, dstar, cap, pool, bytes, plans, tot, status);
    return cudaGetLastError();
}

cudaError_t launch_batch_tile_offsets(long long *cnt, int m, long long cap, long long *n_tiles, int *status,
                                      cudaStream_t s) {
    KernelScope ks("batch_tile_offsets", s);
    k_batch_tile_offsets<<<1, PLAN_T, 0, s>>>(cnt, m, cap, n_tiles, status);
    return cudaGetLastError();
}

}  // namespace spmvat
