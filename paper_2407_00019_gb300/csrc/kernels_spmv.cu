// SpMV y = A x in each format of Sec. 2.1 (Sec. 3 gives the paper's OpenMP
// loops; these are GB300 designs of the same products).
//
//  CRS      : regular rows: 128-row tiles staged in shared memory, SPLIT
//             threads per row with lanes on consecutive rows (coalesced x
//             gathers on banded matrices), fixed-order partial sums; rows too
//             long for a staged tile: V lanes per row with a fixed shuffle
//             tree; uneven rows: the entry-split product (below).
//  ELL-Row  : one thread per two rows, 128-bit loads of the column-major
//             slots (values and indices), FMA in slot order (Fig. 3 order).
//  COO-Row  : row-aligned 128-row tiles staged in shared memory (bounds
//             from the row pointers), as CRS; tiles too large for shared
//             memory: the entry-split product. The allocation-free entry
//             point uses 2048-entry tiles whose rows crossing tile edges are
//             finished by a second, per-tile kernel in tile order.
//  COO-Col, ELL-Col, CCS : the column-major products of Fig. 1: each entry
//             adds val * x[col] into y[row] with FP64 atomics.
#include <climits>

#include "common.cuh"

namespace spmvat {

// ===================================================================== CRS
template <int V>
__global__ void __launch_bounds__(256) k_spmv_crs_vector(const int32_t *__restrict__ irp,
                                                          const int32_t *__restrict__ icol,
                                                          const double *__restrict__ val,
                                                          const int32_t *__restrict__ rows, int64_t count,
                                                          const double *__restrict__ x, double *__restrict__ y) {
    constexpr int G = 32 / V;  // rows per warp and iteration
    const unsigned lane = lane_id();
    const int sub = (int)lane % V;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long g0 = warp * G; g0 < count; g0 += nwarps * G) {
        const long long g = g0 + (lane / V);
        const bool valid = g < count;
        const int r = valid ? (rows ? __ldg(rows + g) : (int)g) : 0;
        const int s = valid ? __ldg(irp + r) : 0;
        const int e = valid ? __ldg(irp + r + 1) : 0;
        double acc = 0.0;
        int k = s + sub;
        for (; k + V < e; k += 2 * V) {
            const double v0 = __ldcs(val + k), v1 = __ldcs(val + k + V);
            const int c0 = __ldcs(icol + k), c1 = __ldcs(icol + k + V);
            acc = fma(v0, __ldg(x + c0), acc);
            acc = fma(v1, __ldg(x + c1), acc);
        }
        if (k < e) acc = fma(__ldcs(val + k), __ldg(x + __ldcs(icol + k)), acc);
#pragma unroll
        for (int o = V / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, V);
        if (valid && sub == 0) y[r] = acc;
    }
}

cudaError_t launch_spmv_crs_vector(int v, const int32_t *irp, const int32_t *icol, const double *val,
                                   const int32_t *rows, int64_t count, const double *x, double *y,
                                   cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    const long long warps_needed = (count * v + 31) / 32;
    unsigned grid = ceil_div_u(warps_needed, 8);
    const unsigned cap = (unsigned)sm_count() * 16u;
    if (grid > cap) grid = cap;
    switch (v) {
#define SPMV_CASE(VV)                                                                            \
    case VV: {                                                                                   \
        KernelScope ks("spmv_crs_v" #VV, s);                                                     \
        k_spmv_crs_vector<VV><<<grid, 256, 0, s>>>(irp, icol, val, rows, count, x, y);           \
        break;                                                                                   \
    }
        SPMV_CASE(1)
        SPMV_CASE(2)
        SPMV_CASE(4)
        SPMV_CASE(8)
        SPMV_CASE(16)
        SPMV_CASE(32)
#undef SPMV_CASE
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Rows of a tile in ELL order: a CTA stages 128 consecutive rows' VAL and
// ICOL in shared memory with coalesced loads (eight per thread in flight),
// then SPLIT threads per row walk the row's entries; for a fixed slot the
// lanes of a warp handle consecutive rows, so their x gathers land on
// neighbouring columns for banded matrices, as in ELL-Row. FMA chains in
// storage order (strided by part), partials of the SPLIT threads added in a
// fixed order.
constexpr int CRS_ROWS_R = 128;

// One thread's share of a staged row: entries k0, k0 + SPLIT, ... below e,
// FMA chain in that order; the x gathers of up to eight entries are issued
// together before their FMAs (a 27-entry row at SPLIT = 4 waits for one
// gather latency instead of four).
template <int SPLIT>
__device__ __forceinline__ double staged_row_dot(const double *s_v, const int32_t *s_c, int k0, int e,
                                                 const double *__restrict__ x) {
    double acc = 0.0;
    for (; k0 < e; k0 += 8 * SPLIT) {
        double xv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int k = k0 + u * SPLIT;
            xv[u] = (k < e) ? __ldg(x + s_c[k]) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int k = k0 + u * SPLIT;
            if (k < e) acc = fma(s_v[k], xv[u], acc);
        }
    }
    return acc;
}

template <int SPLIT>
__global__ void __launch_bounds__(CRS_ROWS_R *SPLIT) k_spmv_crs_rows(const int32_t *__restrict__ irp,
                                                                     const int32_t *__restrict__ icol,
                                                                     const double *__restrict__ val, int32_t n_rows,
                                                                     int cap, const double *__restrict__ x,
                                                                     double *__restrict__ y) {
    constexpr int R = CRS_ROWS_R;
    constexpr int T = R * SPLIT;
    extern __shared__ __align__(16) unsigned char smem[];
    double *s_v = reinterpret_cast<double *>(smem);
    int32_t *s_c = reinterpret_cast<int32_t *>(s_v + cap);
    __shared__ int32_t s_ptr[R + 1];
    __shared__ double s_part[SPLIT > 1 ? (SPLIT - 1) * R : 1];
    const long long r0 = (long long)blockIdx.x * R;
    const int nr = (int)min((long long)R, (long long)n_rows - r0);
    const int e0 = __ldg(irp + r0), e1 = __ldg(irp + r0 + nr);
    const int n = e1 - e0;
    const bool staged = n <= cap;
    for (int i = threadIdx.x; i <= nr; i += T) s_ptr[i] = irp[r0 + i];
    if (staged) {
        for (int q0 = threadIdx.x; q0 < n; q0 += 8 * T) {
            double v[8];
            int c[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int q = q0 + u * T;
                v[u] = (q < n) ? __ldcs(val + e0 + q) : 0.0;
                c[u] = (q < n) ? __ldcs(icol + e0 + q) : 0;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int q = q0 + u * T;
                if (q < n) {
                    s_v[q] = v[u];
                    s_c[q] = c[u];
                }
            }
        }
    }
    __syncthreads();
    const int r = threadIdx.x % R, part = threadIdx.x / R;
    double acc = 0.0;
    if (r < nr) {
        const int s = s_ptr[r] - e0, e = s_ptr[r + 1] - e0;
        if (staged) {
            acc = staged_row_dot<SPLIT>(s_v, s_c, s + part, e, x);
        } else {
            for (int k = e0 + s + part; k < e0 + e; k += SPLIT)
                acc = fma(__ldcs(val + k), __ldg(x + __ldcs(icol + k)), acc);
        }
    }
    if (SPLIT > 1) {
        if (part > 0) s_part[(part - 1) * R + r] = acc;
        __syncthreads();
        if (part == 0)
            for (int p = 1; p < SPLIT; ++p) acc += s_part[(p - 1) * R + r];
    }
    if (part == 0 && r < nr) y[r0 + r] = acc;
}

// Shared-memory capacity (entries) for 128-row tiles of rows up to
// max_row_len long; 0 when that would leave fewer than two CTAs per SM.
int crs_rows_cap(int max_row_len) {
    const long long cap = (long long)CRS_ROWS_R * (max_row_len > 0 ? max_row_len : 1);
    return cap * 12 <= 96 * 1024 ? (int)((cap + 3) & ~3ll) : 0;
}

cudaError_t launch_spmv_crs_rows(int split, int cap, const int32_t *irp, const int32_t *icol, const double *val,
                                 int32_t n_rows, const double *x, double *y, cudaStream_t s) {
    if (n_rows <= 0) return cudaSuccess;
    if (cap <= 0) return cudaErrorInvalidValue;
    const unsigned grid = ceil_div_u(n_rows, CRS_ROWS_R);
    const size_t smem = (size_t)cap * 12;
    switch (split) {
#define ROWS_CASE(SP)                                                                         \
    case SP: {                                                                                \
        cudaError_t e = set_smem_attr(k_spmv_crs_rows<SP>, smem);                             \
        if (e != cudaSuccess) return e;                                                       \
        KernelScope ks("spmv_crs_rows_p" #SP, s);                                             \
        k_spmv_crs_rows<SP><<<grid, CRS_ROWS_R * SP, smem, s>>>(irp, icol, val, n_rows, cap, x, y); \
        break;                                                                                \
    }
        ROWS_CASE(1)
        ROWS_CASE(2)
        ROWS_CASE(4)
        ROWS_CASE(8)
#undef ROWS_CASE
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ================================================================= ELL-Row
template <int UNROLL>
__global__ void __launch_bounds__(256) k_spmv_ell_row(const double *__restrict__ eval,
                                                       const int32_t *__restrict__ eidx, int32_t n_rows,
                                                       int32_t width, int32_t ld, const double *__restrict__ x,
                                                       double *__restrict__ y, bool y16) {
    const long long pairs = ((long long)n_rows + 1) >> 1;
    const long long step = (long long)ld >> 1;  // one slot column, in double2 / int2
    const double2 *pv = reinterpret_cast<const double2 *>(eval);
    const int2 *pc = reinterpret_cast<const int2 *>(eidx);
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < pairs;
         p += (long long)gridDim.x * blockDim.x) {
        double a0 = 0.0, a1 = 0.0;
        int k = 0;
        for (; k + UNROLL <= width; k += UNROLL) {
            double2 v[UNROLL];
            int2 c[UNROLL];
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                v[u] = __ldcs(pv + (long long)(k + u) * step + p);
                c[u] = __ldcs(pc + (long long)(k + u) * step + p);
            }
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                a0 = fma(v[u].x, __ldg(x + c[u].x), a0);
                a1 = fma(v[u].y, __ldg(x + c[u].y), a1);
            }
        }
        for (; k < width; ++k) {
            const double2 v = __ldcs(pv + (long long)k * step + p);
            const int2 c = __ldcs(pc + (long long)k * step + p);
            a0 = fma(v.x, __ldg(x + c.x), a0);
            a1 = fma(v.y, __ldg(x + c.y), a1);
        }
        const long long i = 2 * p;
        if (y16 && i + 1 < n_rows) {
            __stcs(reinterpret_cast<double2 *>(y + i), make_double2(a0, a1));
        } else {
            y[i] = a0;
            if (i + 1 < n_rows) y[i + 1] = a1;
        }
    }
}

cudaError_t launch_spmv_ell_row(const double *eval, const int32_t *eidx, int32_t n_rows, int32_t width,
                                int32_t ld, const double *x, double *y, cudaStream_t s) {
    if (n_rows <= 0) return cudaSuccess;
    const bool y16 = (reinterpret_cast<uintptr_t>(y) & 15) == 0;  // else two 8-byte stores per pair
    const long long pairs = ((long long)n_rows + 1) >> 1;
    const unsigned grid = ceil_div_u(pairs, 256);
    KernelScope ks("spmv_ell_row", s);
    k_spmv_ell_row<4><<<grid, 256, 0, s>>>(eval, eidx, n_rows, width, ld, x, y, y16);
    return cudaGetLastError();
}

// ================================================================= ELL-Col
// One column per thread: slot k of column j is at k*ld + j, so a warp loads
// 32 consecutive columns (coalesced) and its atomic adds go to the k-th rows
// of 32 consecutive columns, which in banded matrices are consecutive rows:
// a few sectors of y per warp instruction.
// SKIP (chosen when padding is at least a quarter of the slots): a slot
// holding +-0 (the padding of a short column, Fig. 3) adds +-0 when x_j is
// finite, which leaves y unchanged (y starts at +0, so no element is ever
// -0), and such adds are left out; with x_j infinite or NaN every slot is
// added, so the padding still turns y into NaN as the padded product does.
// A warp whose four slots of a batch hold no zero adds them unconditionally.
// Without SKIP the loop has no test at all (the test costs matrices with
// little padding more than it saves).
template <bool SKIP>
__global__ void __launch_bounds__(256) k_spmv_ell_col(const double *__restrict__ eval,
                                                       const int32_t *__restrict__ eidx, int32_t n_cols,
                                                       int32_t width, int32_t ld, const double *__restrict__ x,
                                                       double *__restrict__ y) {
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n_cols;
         j += (long long)gridDim.x * blockDim.x) {
        const double xj = __ldg(x + j);
        const bool all = !SKIP || !isfinite(xj);
        const double *pv = eval + j;
        const int32_t *pr = eidx + j;
        int k = 0;
        for (; k + 4 <= width; k += 4) {
            double v[4];
            int r[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                v[u] = __ldcs(pv + (long long)(k + u) * ld);
                r[u] = __ldcs(pr + (long long)(k + u) * ld);
            }
            if (!SKIP) {
#pragma unroll
                for (int u = 0; u < 4; ++u) atomicAdd(y + r[u], v[u] * xj);
                continue;
            }
            bool keep[4], every = true;
#pragma unroll
            for (int u = 0; u < 4; ++u) every &= keep[u] = all || v[u] != 0.0;
            if (__all_sync(__activemask(), every)) {  // lanes past n_cols have left the loop
#pragma unroll
                for (int u = 0; u < 4; ++u) atomicAdd(y + r[u], v[u] * xj);
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (keep[u]) atomicAdd(y + r[u], v[u] * xj);
            }
        }
        for (; k < width; ++k) {
            const double v = __ldcs(pv + (long long)k * ld);
            if (all || v != 0.0) atomicAdd(y + __ldcs(pr + (long long)k * ld), v * xj);
        }
    }
}

cudaError_t launch_spmv_ell_col(const double *eval, const int32_t *eidx, int32_t n_rows, int32_t n_cols,
                                int32_t width, int32_t ld, int64_t nnz, const double *x, double *y, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(y, 0, sizeof(double) * (size_t)n_rows, s);
    if (e != cudaSuccess || n_cols <= 0) return e;
    const bool skip = 4.0 * (double)nnz <= 3.0 * (double)width * (double)n_cols;  // >= 1/4 of the slots padding
    KernelScope ks("spmv_ell_col", s);
    if (skip)
        k_spmv_ell_col<true><<<ceil_div_u(n_cols, 256), 256, 0, s>>>(eval, eidx, n_cols, width, ld, x, y);
    else
        k_spmv_ell_col<false><<<ceil_div_u(n_cols, 256), 256, 0, s>>>(eval, eidx, n_cols, width, ld, x, y);
    return cudaGetLastError();
}

// ---- the ceiling of the column-wise products: FP64 atomic adds alone -------
// n_adds adds of 1.0 into y[0..n), lanes on consecutive elements and each
// pass over y shifted by a fixed offset: the best case of the atomic adds of
// COO-Column and ELL-Column on banded matrices, with no other memory traffic.
__global__ void __launch_bounds__(256) k_atomic_ceiling(double *__restrict__ y, long long n, long long n_adds) {
    const long long nt = (long long)gridDim.x * blockDim.x;
    for (long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x; a < n_adds; a += nt) {
        const long long pass = a / n;
        atomicAdd(y + (a + pass * 16384) % n, 1.0);
    }
}

cudaError_t launch_atomic_ceiling(double *y, long long n, long long n_adds, cudaStream_t s) {
    if (n <= 0 || n_adds <= 0) return cudaSuccess;
    KernelScope ks("atomic_ceiling", s);
    k_atomic_ceiling<<<(unsigned)sm_count() * 8u, 256, 0, s>>>(y, n, n_adds);
    return cudaGetLastError();
}

// ================================================================= COO-Row
constexpr int COO_ROWS_R = 128;  // rows per tile of the row-aligned COO-Row kernel
constexpr int COO_THREADS = 256;
constexpr int COO_ITEMS = 8;
constexpr int COO_TILE = COO_THREADS * COO_ITEMS;

size_t coo_row_scratch_bytes(int64_t nnz) {
    const long long tiles = (nnz + COO_TILE - 1) / COO_TILE;
    return (size_t)(tiles > 0 ? tiles : 1) * sizeof(double2) + 16;  // carries + a status word
}

// One CTA per 2048-entry tile, several CTAs per SM. Phase A: coalesced loads
// of IROW / ICOL / VAL (eight per thread in flight) into shared memory.
// Segments (runs of one row) are then found with integer work only (a head
// flag per entry, one block scan). Phase B: consecutive threads take
// consecutive segments, so for a fixed position the x gathers of a warp hit
// neighbouring columns on banded matrices; when a tile has few segments,
// SPLIT threads share each one (entries strided by part, partials added in a
// fixed order); segments longer than COO_LONG are summed by a warp. One FMA
// per entry, storage order within each part. A segment that continues from
// the previous tile or into the next one leaves its partial in `carry` for
// k_coo_row_carry.
constexpr int COO_LONG = 64;

__global__ void __launch_bounds__(COO_THREADS) k_coo_row_tiles(const int32_t *__restrict__ irow,
                                                                const int32_t *__restrict__ icol,
                                                                const double *__restrict__ val, int64_t nnz,
                                                                int32_t n_rows, int32_t n_cols,
                                                                const double *__restrict__ x,
                                                                double *__restrict__ y, double2 *__restrict__ carry) {
    __shared__ double s_v[COO_TILE];
    __shared__ int32_t s_c[COO_TILE];
    __shared__ int32_t s_r[COO_TILE];
    __shared__ int32_t s_seg[COO_TILE + 1];
    __shared__ double s_part[COO_THREADS];
    __shared__ int s_wc[COO_THREADS / 32];
    __shared__ int s_nseg, s_prev, s_next;
    const unsigned lane = lane_id();
    const int w = threadIdx.x >> 5;
    const long long e0 = (long long)blockIdx.x * COO_TILE;
    const int n = (int)min((long long)COO_TILE, (long long)nnz - e0);
    if (threadIdx.x == 0) {
        s_prev = (e0 > 0) ? __ldg(irow + e0 - 1) : -1;
        s_next = (e0 + n < nnz) ? __ldg(irow + e0 + n) : -1;
    }
    {
        int r[COO_ITEMS], c[COO_ITEMS];
        double v[COO_ITEMS];
#pragma unroll
        for (int u = 0; u < COO_ITEMS; ++u) {
            const int q = u * COO_THREADS + threadIdx.x;
            const bool h = q < n;
            r[u] = h ? __ldcs(irow + e0 + q) : 0;
            c[u] = h ? __ldcs(icol + e0 + q) : 0;
            v[u] = h ? __ldcs(val + e0 + q) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < COO_ITEMS; ++u) {
            const int q = u * COO_THREADS + threadIdx.x;
            if (q < n) {
                const bool okc = (unsigned)c[u] < (unsigned)n_cols;
                s_r[q] = r[u];
                s_c[q] = okc ? c[u] : 0;
                s_v[q] = okc ? v[u] : 0.0;
            }
        }
    }
    __syncthreads();
    // segment starts: thread t looks at entries 8t .. 8t+7
    const int qb = (int)threadIdx.x * COO_ITEMS;
    int rr[COO_ITEMS + 1];
#pragma unroll
    for (int j = 0; j <= COO_ITEMS; ++j) {
        const int q = qb + j - 1;
        rr[j] = (q >= 0 && q < n) ? s_r[q] : -2;
    }
    int cnt = 0;
#pragma unroll
    for (int j = 1; j <= COO_ITEMS; ++j) cnt += (qb + j - 1 < n) && (qb + j - 1 == 0 || rr[j] != rr[j - 1]);
    int inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, inc, o);
        if ((int)lane >= o) inc += t;
    }
    if (lane == 31) s_wc[w] = inc;
    __syncthreads();
    int off = inc - cnt, tot = 0;
    for (int j = 0; j < COO_THREADS / 32; ++j) {
        if (j < w) off += s_wc[j];
        tot += s_wc[j];
    }
#pragma unroll
    for (int j = 1; j <= COO_ITEMS; ++j)
        if ((qb + j - 1 < n) && (qb + j - 1 == 0 || rr[j] != rr[j - 1])) s_seg[off++] = qb + j - 1;
    if (threadIdx.x == 0) {
        s_seg[tot] = n;
        s_nseg = tot;
    }
    __syncthreads();
    const int nseg = s_nseg;
    const int prev_row = s_prev, next_row = s_next;
    const bool last_tile = e0 + n >= nnz;
    auto emit = [&](int g, int row, double sum) {
        const bool cin = (g == 0) && prev_row == row;
        const bool cout = (g == nseg - 1) && next_row == row;
        if (cin || cout) {
            if (cin) carry[blockIdx.x].x = sum;
            if (cout) carry[blockIdx.x].y = sum;
        } else if ((unsigned)row < (unsigned)n_rows) {
            y[row] = sum;
        }
        if (g == 0)
            for (int q = prev_row + 1; q < row && q < n_rows; ++q) y[q] = 0.0;
        const int upto = (g + 1 < nseg) ? s_r[s_seg[g + 1]] : (last_tile ? n_rows : row + 1);
        for (int q = row + 1; q < upto && q < n_rows; ++q) y[q] = 0.0;
    };
    // threads per segment
    int ns = 1;
    while (ns < nseg && ns < COO_THREADS) ns <<= 1;
    const int split = (ns >= COO_THREADS) ? 1 : min(8, COO_THREADS / ns);
    const int gs = (split == 1) ? COO_THREADS : ns;
    const int part = (int)threadIdx.x / gs;
    for (int g0 = 0; g0 < nseg; g0 += gs) {
        const int g = g0 + (int)threadIdx.x % gs;
        double acc = 0.0;
        bool mine = part < split && g < nseg;
        int q0 = 0, q1 = 0;
        if (mine) {
            q0 = s_seg[g];
            q1 = s_seg[g + 1];
            if (q1 - q0 > COO_LONG) mine = false;
        }
        if (mine)
            for (int q = q0 + part; q < q1; q += split) acc = fma(s_v[q], __ldg(x + s_c[q]), acc);
        if (split > 1) {
            if (mine && part > 0) s_part[threadIdx.x] = acc;
            __syncthreads();
            if (mine && part == 0)
                for (int p = 1; p < split; ++p) acc += s_part[p * gs + threadIdx.x];
            __syncthreads();
        }
        if (mine && part == 0) emit(g, s_r[q0], acc);
    }
    // long segments: one warp each
    for (int g = w; g < nseg; g += COO_THREADS / 32) {
        const int q0 = s_seg[g], q1 = s_seg[g + 1];
        if (q1 - q0 <= COO_LONG) continue;
        double acc = 0.0;
        for (int q = q0 + (int)lane; q < q1; q += 32) acc = fma(s_v[q], __ldg(x + s_c[q]), acc);
        acc = warp_sum(acc);
        if (lane == 0) emit(g, s_r[q0], acc);
    }
}

// ---- COO over line-aligned tiles -----------------------------------------
// Tile bounds of the 128-line schedules of COO-Row and COO-Column: tb[t] =
// ptr[min(128 t, n_lines)], the first entry of line 128 t in the line-sorted
// COO (ptr: the pointers of the compressed format the COO is made from), and
// the largest tile's entry count into *maxn when given. Bounds are clamped to
// [0, nnz], so the products stay in bounds even on malformed pointers. The
// largest count is reduced per warp first (one atomic per warp, not per tile).
__global__ void __launch_bounds__(256) k_line_tile_bounds(const int32_t *__restrict__ ptr, int32_t n_lines,
                                                           int64_t nnz, long long n_tiles, int32_t *__restrict__ tb,
                                                           int32_t *__restrict__ maxn) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const auto bound = [&](long long u) {
        return (int32_t)min(max((long long)__ldg(ptr + min(u * COO_ROWS_R, (long long)n_lines)), 0ll), (long long)nnz);
    };
    int32_t m = 0;
    if (t <= n_tiles) {
        const int32_t a = bound(t);
        tb[t] = a;
        if (t < n_tiles) m = bound(t + 1) - a;
    }
    if (maxn) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane_id() == 0 && m > 0) atomicMax(maxn, m);
    }
}

cudaError_t launch_line_tile_bounds(const int32_t *ptr, int32_t n_lines, int64_t nnz, int32_t *tb, int32_t *maxn,
                                    const char *name, cudaStream_t s) {
    const long long n_tiles = ((long long)n_lines + COO_ROWS_R - 1) / COO_ROWS_R;
    KernelScope ks(name, s);
    k_line_tile_bounds<<<ceil_div_u(n_tiles + 1, 256), 256, 0, s>>>(ptr, n_lines, nnz, n_tiles, tb, maxn);
    return cudaGetLastError();
}

// A CTA takes 128 consecutive rows: their entries [tb[t], tb[t+1]) are
// loaded into shared memory with coalesced loads (VAL, ICOL, and IROW as a
// one-byte offset from the tile's first row: 13 bytes an entry, so four CTAs
// of 512 threads fit an SM), each row finds its first entry by binary search
// over the staged offsets, then SPLIT threads per row run the FMA chains with
// lanes on consecutive rows (as k_spmv_crs_rows). Rows never cross tiles, so
// no partial sums are carried.
// entries a thread loads at once while staging: three for the row tiles (a
// batch of four took 200 against 187 us on the 27-point stencil, 128^3), four
// for the column tiles (three took 199 against 195 us)
constexpr int COO_ROW_STAGE_U = 3;
constexpr int COO_COL_STAGE_U = 4;

__host__ __device__ constexpr size_t coo_tile_smem(int cap) { return ((size_t)cap * 13 + 15) & ~(size_t)15; }

template <int SPLIT>
__global__ void __launch_bounds__(COO_ROWS_R *SPLIT, 2048 / (COO_ROWS_R * SPLIT)) k_coo_row_rows(
    const int32_t *__restrict__ irow, const int32_t *__restrict__ icol, const double *__restrict__ val,
    const int32_t *__restrict__ tb, int32_t n_rows, int32_t n_cols, int cap, const double *__restrict__ x,
    double *__restrict__ y) {
    constexpr int R = COO_ROWS_R;
    constexpr int T = R * SPLIT;
    constexpr int U = COO_ROW_STAGE_U;
    extern __shared__ __align__(16) unsigned char smem[];
    double *s_v = reinterpret_cast<double *>(smem);
    int32_t *s_c = reinterpret_cast<int32_t *>(s_v + cap);
    uint8_t *s_r = reinterpret_cast<uint8_t *>(s_c + cap);  // row - r0, clamped to [0, R]
    __shared__ int32_t s_ptr[R + 1];
    __shared__ double s_part[SPLIT > 1 ? (SPLIT - 1) * R : 1];
    const long long r0 = (long long)blockIdx.x * R;
    const int nr = (int)min((long long)R, (long long)n_rows - r0);
    const int e0 = __ldg(tb + blockIdx.x), e1 = __ldg(tb + blockIdx.x + 1);
    const int n = e1 - e0;  // <= cap by construction of the schedule
    for (int q0 = threadIdx.x; q0 < n; q0 += U * T) {
        double v[U];
        int c[U], r[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int q = q0 + u * T;
            v[u] = (q < n) ? __ldcs(val + e0 + q) : 0.0;
            c[u] = (q < n) ? __ldcs(icol + e0 + q) : 0;
            r[u] = (q < n) ? __ldcs(irow + e0 + q) : 0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int q = q0 + u * T;
            if (q < n) {
                const bool ok = (unsigned)c[u] < (unsigned)n_cols;
                s_v[q] = ok ? v[u] : 0.0;
                s_c[q] = ok ? c[u] : 0;
                s_r[q] = (uint8_t)min(max((long long)r[u] - r0, 0ll), (long long)R);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) s_ptr[nr] = n;  // every staged entry belongs to a row below r0 + nr
    if (threadIdx.x < (unsigned)nr) {  // first entry of row r0 + i: lower bound in s_r
        const int key = (int)threadIdx.x;
        int lo = 0, hi = n;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if ((int)s_r[mid] < key) lo = mid + 1; else hi = mid;
        }
        s_ptr[threadIdx.x] = lo;
    }
    __syncthreads();
    const int r = threadIdx.x % R, part = threadIdx.x / R;
    double acc = 0.0;
    if (r < nr) {
        const int s = s_ptr[r], e = s_ptr[r + 1];
        acc = staged_row_dot<SPLIT>(s_v, s_c, s + part, e, x);
    }
    if (SPLIT > 1) {
        if (part > 0) s_part[(part - 1) * R + r] = acc;
        __syncthreads();
        if (part == 0)
            for (int p = 1; p < SPLIT; ++p) acc += s_part[(p - 1) * R + r];
    }
    if (part == 0 && r < nr) y[r0 + r] = acc;
}

// shared-memory entries for row tiles whose largest tile has max_n entries
// (0: would leave fewer than two CTAs per SM)
int coo_rows_cap(int max_n) {
    const long long cap = ((long long)(max_n > 0 ? max_n : 1) + 3) & ~3ll;
    return cap * 16 <= 96 * 1024 ? (int)cap : 0;
}

cudaError_t launch_spmv_coo_row_rows(int split, int cap, const int32_t *irow, const int32_t *icol,
                                     const double *val, const int32_t *tb, int32_t n_rows, int32_t n_cols,
                                     const double *x, double *y, cudaStream_t s) {
    if (n_rows <= 0) return cudaSuccess;
    if (cap <= 0) return cudaErrorInvalidValue;
    const unsigned grid = ceil_div_u(n_rows, COO_ROWS_R);
    const size_t smem = coo_tile_smem(cap);
    switch (split) {
#define COOR_CASE(SP)                                                                                  \
    case SP: {                                                                                         \
        cudaError_t e = set_smem_attr(k_coo_row_rows<SP>, smem);                                       \
        if (e != cudaSuccess) return e;                                                                \
        KernelScope ks("spmv_coo_row_rows_p" #SP, s);                                                  \
        k_coo_row_rows<SP><<<grid, COO_ROWS_R * SP, smem, s>>>(irow, icol, val, tb, n_rows, n_cols, cap, x, y); \
        break;                                                                                         \
    }
        COOR_CASE(2)
        COOR_CASE(4)
#undef COOR_CASE
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Rows that cross tile edges: the tile where the row starts walks forward
// and adds the partials in tile order.
__global__ void __launch_bounds__(256) k_coo_row_carry(const int32_t *__restrict__ irow, int64_t nnz,
                                                        long long n_tiles, int32_t n_rows,
                                                        const double2 *__restrict__ carry, double *__restrict__ y) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tiles) return;
    const long long t0 = t * COO_TILE;
    const long long t1 = min(t0 + (long long)COO_TILE, (long long)nnz);
    const int ra = irow[t0], rb = irow[t1 - 1];
    const bool cin = (t0 > 0) && irow[t0 - 1] == ra;
    const bool cout = (t1 < nnz) && irow[t1] == rb;
    if (!cout || (cin && ra == rb)) return;
    double sum = carry[t].y;
    for (long long u = t + 1; u < n_tiles; ++u) {
        sum += carry[u].x;
        const long long u0 = u * COO_TILE;
        const long long u1 = min(u0 + (long long)COO_TILE, (long long)nnz);
        const bool middle = (irow[u1 - 1] == rb) && (u1 < nnz) && irow[u1] == rb;
        if (!middle) break;
    }
    if ((unsigned)rb < (unsigned)n_rows) y[rb] = sum;
}

cudaError_t launch_spmv_coo_row(const int32_t *irow, const int32_t *icol, const double *val, int64_t nnz,
                                int32_t n_rows, int32_t n_cols, const double *x, double *y, void *scratch,
                                int *status, cudaStream_t s) {
    (void)status;  // no device-side waits in this kernel
    if (nnz <= 0) return cudaMemsetAsync(y, 0, sizeof(double) * (size_t)n_rows, s);
    const long long tiles = (nnz + COO_TILE - 1) / COO_TILE;
    double2 *carry = reinterpret_cast<double2 *>(scratch);
    {
        KernelScope ks("spmv_coo_row", s);
        k_coo_row_tiles<<<(unsigned)tiles, COO_THREADS, 0, s>>>(irow, icol, val, nnz, n_rows, n_cols, x, y, carry);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    KernelScope ks("spmv_coo_row_carry", s);
    k_coo_row_carry<<<ceil_div_u(tiles, 256), 256, 0, s>>>(irow, nnz, tiles, n_rows, carry, y);
    return cudaGetLastError();
}

// ================================================================= COO-Col
constexpr int COOC_ITEMS = 4;
__global__ void __launch_bounds__(256) k_spmv_coo_col(const int32_t *__restrict__ row,
                                                       const int32_t *__restrict__ col,
                                                       const double *__restrict__ val, int64_t nnz,
                                                       const double *__restrict__ x, double *__restrict__ y) {
    const long long k = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * COOC_ITEMS;
    if (k >= nnz) return;
    if (k + COOC_ITEMS <= nnz && ((reinterpret_cast<uintptr_t>(row + k) & 15) == 0) &&
        ((reinterpret_cast<uintptr_t>(col + k) & 15) == 0) && ((reinterpret_cast<uintptr_t>(val + k) & 15) == 0)) {
        const int4 r = __ldcs(reinterpret_cast<const int4 *>(row + k));
        const int4 c = __ldcs(reinterpret_cast<const int4 *>(col + k));
        const double2 v0 = __ldcs(reinterpret_cast<const double2 *>(val + k));
        const double2 v1 = __ldcs(reinterpret_cast<const double2 *>(val + k) + 1);
        atomicAdd(y + r.x, v0.x * __ldg(x + c.x));
        atomicAdd(y + r.y, v0.y * __ldg(x + c.y));
        atomicAdd(y + r.z, v1.x * __ldg(x + c.z));
        atomicAdd(y + r.w, v1.y * __ldg(x + c.w));
    } else {
        for (long long j = k; j < min(k + COOC_ITEMS, (long long)nnz); ++j)
            atomicAdd(y + row[j], val[j] * __ldg(x + col[j]));
    }
}

// COO-Column over column-aligned tiles: a CTA takes 128 consecutive columns,
// stages their entries (TVAL, TROW, and TCOL as a one-byte offset from the
// tile's first column) in shared memory with coalesced loads, finds each
// column's first entry by binary search over the staged offsets, and SPLIT
// threads per column add VAL * x[col] into y[row] with lanes
// on consecutive columns. Lanes then hold the m-th entries of neighbouring
// columns, which in banded matrices lie in neighbouring rows, so the 32
// atomic adds of a warp instruction fall into a few sectors of y instead of
// 32. `tb` are the tiles' first entries (tile t starts at column 128 t).
template <int SPLIT>
__global__ void __launch_bounds__(COO_ROWS_R *SPLIT, 2048 / (COO_ROWS_R * SPLIT)) k_coo_col_cols(
    const int32_t *__restrict__ trow, const int32_t *__restrict__ tcol, const double *__restrict__ tval,
    const int32_t *__restrict__ tb, int32_t n_rows, int32_t n_cols, int cap, const double *__restrict__ x,
    double *__restrict__ y) {
    constexpr int R = COO_ROWS_R;
    constexpr int T = R * SPLIT;
    constexpr int U = COO_COL_STAGE_U;
    extern __shared__ __align__(16) unsigned char smem[];
    double *s_v = reinterpret_cast<double *>(smem);
    int32_t *s_r = reinterpret_cast<int32_t *>(s_v + cap);
    uint8_t *s_c = reinterpret_cast<uint8_t *>(s_r + cap);  // column - c0, clamped to [0, R]
    __shared__ int32_t s_ptr[R + 1];
    const long long c0 = (long long)blockIdx.x * R;
    const int nc = (int)min((long long)R, (long long)n_cols - c0);
    const int e0 = __ldg(tb + blockIdx.x), e1 = __ldg(tb + blockIdx.x + 1);
    const int n = e1 - e0;  // <= cap by construction of the schedule
    for (int q0 = threadIdx.x; q0 < n; q0 += U * T) {
        double v[U];
        int c[U], r[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int q = q0 + u * T;
            v[u] = (q < n) ? __ldcs(tval + e0 + q) : 0.0;
            c[u] = (q < n) ? __ldcs(tcol + e0 + q) : 0;
            r[u] = (q < n) ? __ldcs(trow + e0 + q) : 0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int q = q0 + u * T;
            if (q < n) {
                const bool ok = (unsigned)r[u] < (unsigned)n_rows;
                s_v[q] = ok ? v[u] : 0.0;
                s_r[q] = ok ? r[u] : 0;
                s_c[q] = (uint8_t)min(max((long long)c[u] - c0, 0ll), (long long)R);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) s_ptr[nc] = n;  // every staged entry belongs to a column below c0 + nc
    if (threadIdx.x < (unsigned)nc) {  // first entry of column c0 + i: lower bound in the staged offsets
        const int key = (int)threadIdx.x;
        int lo = 0, hi = n;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if ((int)s_c[mid] < key) lo = mid + 1; else hi = mid;
        }
        s_ptr[threadIdx.x] = lo;
    }
    __syncthreads();
    const int j = threadIdx.x % R, part = threadIdx.x / R;
    if (j >= nc) return;
    const int st = s_ptr[j], en = s_ptr[j + 1];
    if (st >= en) return;
    const double xj = __ldg(x + c0 + j);
    int k = st + part;
    for (; k + 3 * SPLIT < en; k += 4 * SPLIT) {
        const int r0 = s_r[k], r1 = s_r[k + SPLIT], r2 = s_r[k + 2 * SPLIT], r3 = s_r[k + 3 * SPLIT];
        atomicAdd(y + r0, s_v[k] * xj);
        atomicAdd(y + r1, s_v[k + SPLIT] * xj);
        atomicAdd(y + r2, s_v[k + 2 * SPLIT] * xj);
        atomicAdd(y + r3, s_v[k + 3 * SPLIT] * xj);
    }
    for (; k < en; k += SPLIT) atomicAdd(y + s_r[k], s_v[k] * xj);
}

cudaError_t launch_spmv_coo_col_cols(int split, int cap, const int32_t *trow, const int32_t *tcol, const double *tval,
                                     const int32_t *tb, int32_t n_rows, int32_t n_cols, const double *x, double *y,
                                     cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(y, 0, sizeof(double) * (size_t)n_rows, s);
    if (e != cudaSuccess || n_cols <= 0) return e;
    if (cap <= 0) return cudaErrorInvalidValue;
    const unsigned grid = ceil_div_u(n_cols, COO_ROWS_R);
    const size_t smem = coo_tile_smem(cap);
    switch (split) {
#define COOC_CASE(SP)                                                                                           \
    case SP: {                                                                                                  \
        e = set_smem_attr(k_coo_col_cols<SP>, smem);                                                            \
        if (e != cudaSuccess) return e;                                                                         \
        KernelScope ks("spmv_coo_col_cols_p" #SP, s);                                                           \
        k_coo_col_cols<SP><<<grid, COO_ROWS_R * SP, smem, s>>>(trow, tcol, tval, tb, n_rows, n_cols, cap, x, y); \
        break;                                                                                                  \
    }
        COOC_CASE(1)
        COOC_CASE(2)
        COOC_CASE(4)
#undef COOC_CASE
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_spmv_coo_col(const int32_t *row, const int32_t *col, const double *val, int64_t nnz,
                                int32_t n_rows, const double *x, double *y, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(y, 0, sizeof(double) * (size_t)n_rows, s);
    if (e != cudaSuccess || nnz <= 0) return e;
    KernelScope ks("spmv_coo_col", s);
    k_spmv_coo_col<<<ceil_div_u(nnz, 256 * COOC_ITEMS), 256, 0, s>>>(row, col, val, nnz, x, y);
    return cudaGetLastError();
}

// ===================================================================== CCS
// Eight lanes per column; each adds its entries into y[row].
__global__ void __launch_bounds__(256) k_spmv_ccs(const int32_t *__restrict__ cp, const int32_t *__restrict__ trow,
                                                   const double *__restrict__ tval, int32_t n_cols,
                                                   const double *__restrict__ x, double *__restrict__ y) {
    constexpr int V = 8;
    const long long g = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / V;
    const int sub = threadIdx.x % V;
    if (g >= n_cols) return;
    const double xj = __ldg(x + g);
    const int s = __ldg(cp + g), e = __ldg(cp + g + 1);
    for (int p = s + sub; p < e; p += V) atomicAdd(y + __ldcs(trow + p), __ldcs(tval + p) * xj);
}

cudaError_t launch_spmv_ccs(const int32_t *cp, const int32_t *trow, const double *tval, int32_t n_rows,
                            int32_t n_cols, const double *x, double *y, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(y, 0, sizeof(double) * (size_t)n_rows, s);
    if (e != cudaSuccess || n_cols <= 0) return e;
    KernelScope ks("spmv_ccs", s);
    k_spmv_ccs<<<ceil_div_u((long long)n_cols * 8, 256), 256, 0, s>>>(cp, trow, tval, n_cols, x, y);
    return cudaGetLastError();
}

// ===================================================== entry-split products
// For rows of very uneven length (power-law rows): every thread multiplies 8
// consecutive entries, one FMA each in storage order, restarting at each row
// start; it stores the sum of every row that starts and ends inside its 8
// entries and adds the partial sums of rows that cross its edges into y with
// atomicAdd (y is zeroed first). Every thread issues the same FMAs whatever
// the row lengths, where lanes that own rows would wait for the longest row
// of their warp on the narrow FP64 pipe. CRS finds each entry's row from the
// tile's row pointers (staged in shared memory, as the expansions do); COO
// reads IROW.
constexpr int SEG_THREADS = 256;
constexpr int SEG_ITEMS = 8;
constexpr int SEG_TILE = SEG_THREADS * SEG_ITEMS;
constexpr int SEG_WIN = 2048;

size_t spmv_seg_scratch_bytes(int64_t nnz) { return tile_lines_bytes(nnz, SEG_TILE); }

template <bool COO>
__global__ void __launch_bounds__(SEG_THREADS) k_spmv_seg(const int32_t *__restrict__ lines,
                                                           const int32_t *__restrict__ icol,
                                                           const double *__restrict__ val, int64_t nnz,
                                                           int32_t n_rows, int32_t n_cols,
                                                           const int32_t *__restrict__ tl, long long n_tiles,
                                                           const double *__restrict__ x, double *__restrict__ y) {
    __shared__ int32_t s_ptr[COO ? 1 : SEG_WIN];
    const long long k0 = (long long)blockIdx.x * SEG_TILE;
    const long long k1 = min(k0 + (long long)SEG_TILE, (long long)nnz);
    const long long k = k0 + (long long)threadIdx.x * SEG_ITEMS;
    const int cnt = (int)max(0ll, min((long long)SEG_ITEMS, k1 - k));
    int c[SEG_ITEMS], r[SEG_ITEMS];
    double v[SEG_ITEMS];
    const bool vec = cnt == SEG_ITEMS && ((reinterpret_cast<uintptr_t>(icol + k) & 15) == 0) &&
                     ((reinterpret_cast<uintptr_t>(val + k) & 15) == 0) &&
                     (!COO || ((reinterpret_cast<uintptr_t>(lines + k) & 15) == 0));
    if (vec) {
#pragma unroll
        for (int h = 0; h < SEG_ITEMS / 4; ++h) {
            const int4 q = __ldcs(reinterpret_cast<const int4 *>(icol + k) + h);
            c[4 * h] = q.x; c[4 * h + 1] = q.y; c[4 * h + 2] = q.z; c[4 * h + 3] = q.w;
            if (COO) {
                const int4 p = __ldcs(reinterpret_cast<const int4 *>(lines + k) + h);
                r[4 * h] = p.x; r[4 * h + 1] = p.y; r[4 * h + 2] = p.z; r[4 * h + 3] = p.w;
            }
        }
#pragma unroll
        for (int h = 0; h < SEG_ITEMS / 2; ++h) {
            const double2 q = __ldcs(reinterpret_cast<const double2 *>(val + k) + h);
            v[2 * h] = q.x; v[2 * h + 1] = q.y;
        }
    } else {
#pragma unroll
        for (int j = 0; j < SEG_ITEMS; ++j) {
            c[j] = (j < cnt) ? icol[k + j] : 0;
            v[j] = (j < cnt) ? val[k + j] : 0.0;
            if (COO) r[j] = (j < cnt) ? lines[k + j] : -1;
        }
    }
    bool starts, ends;  // does the first row start, the last row end, inside these entries
    if (COO) {
        int last = r[0];
#pragma unroll
        for (int j = 1; j < SEG_ITEMS; ++j)
            if (j < cnt) last = r[j];
        const int prev = (cnt > 0 && k > 0) ? __ldg(lines + k - 1) : -1;
        const int next = (cnt > 0 && k + cnt < nnz) ? __ldg(lines + k + cnt) : -1;
        starts = prev != r[0];
        ends = next != last;
    } else {
        const int lo = tl[blockIdx.x];
        const int hi = (blockIdx.x + 1 < n_tiles) ? tl[blockIdx.x + 1] : n_rows - 1;
        const int wn = hi - lo + 2;  // lines[lo .. hi+1]
        const bool sm = wn <= SEG_WIN;
        if (sm)
            for (int i = threadIdx.x; i < wn; i += SEG_THREADS) s_ptr[i] = lines[lo + i];
        __syncthreads();
        starts = ends = true;
        if (cnt > 0) {
            auto P = [&](int row) -> long long { return sm ? s_ptr[row - lo] : lines[row]; };
            int row = sm ? lo + last_le(s_ptr, 0, wn - 1, k) : last_le(lines, lo, hi + 1, k);
            starts = P(row) == k;
            long long nb = (row < hi) ? P(row + 1) : LLONG_MAX;
            int last = row;
#pragma unroll
            for (int j = 0; j < SEG_ITEMS; ++j) {
                const long long kk = k + j;
                while (kk >= nb && row < hi) {
                    ++row;
                    nb = (row < hi) ? P(row + 1) : LLONG_MAX;
                }
                r[j] = row;
                if (j < cnt) last = row;
            }
            ends = (last < hi ? P(last + 1) : (long long)lines[last + 1]) <= k + cnt;
        }
    }
    if (cnt == 0) return;
    double xv[SEG_ITEMS];
#pragma unroll
    for (int j = 0; j < SEG_ITEMS; ++j)
        xv[j] = (j < cnt && (unsigned)c[j] < (unsigned)n_cols) ? __ldg(x + c[j]) : 0.0;
    auto flush = [&](int row, double a, bool whole) {
        if ((unsigned)row >= (unsigned)n_rows) return;
        if (whole) y[row] = a;
        else atomicAdd(y + row, a);
    };
    double acc = 0.0;
    int cur = r[0];
    bool first = true;
#pragma unroll
    for (int j = 0; j < SEG_ITEMS; ++j) {
        if (j < cnt) {
            if (r[j] != cur) {
                flush(cur, acc, !first || starts);
                acc = 0.0;
                cur = r[j];
                first = false;
            }
            acc = fma(v[j], xv[j], acc);
        }
    }
    flush(cur, acc, (!first || starts) && ends);
}

cudaError_t launch_spmv_seg(bool coo, const int32_t *lines, const int32_t *icol, const double *val, int64_t nnz,
                            int32_t n_rows, int32_t n_cols, const int32_t *tl, const double *x, double *y,
                            cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(y, 0, sizeof(double) * (size_t)n_rows, s);
    if (e != cudaSuccess || nnz <= 0) return e;
    const long long n_tiles = (nnz + SEG_TILE - 1) / SEG_TILE;
    if (coo) {
        KernelScope ks("spmv_coo_row_seg", s);
        k_spmv_seg<true><<<(unsigned)n_tiles, SEG_THREADS, 0, s>>>(lines, icol, val, nnz, n_rows, n_cols, nullptr,
                                                                   n_tiles, x, y);
    } else {
        KernelScope ks("spmv_crs_seg", s);
        k_spmv_seg<false><<<(unsigned)n_tiles, SEG_THREADS, 0, s>>>(lines, icol, val, nnz, n_rows, n_cols, tl,
                                                                    n_tiles, x, y);
    }
    return cudaGetLastError();
}

// Tile lines of the CRS entry-split product (kept in the CRS handle).
cudaError_t launch_spmv_seg_lines(const int32_t *irp, int32_t n_rows, int64_t nnz, int32_t *tl, cudaStream_t s) {
    return launch_tile_lines(irp, n_rows, nnz, SEG_TILE, tl, s);
}

}  // namespace spmvat
