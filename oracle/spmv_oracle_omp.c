/*
 * Multi-core build of part of the CPU oracle (OpenMP over the host cores).
 *
 * TEST INFRASTRUCTURE ONLY, like spmv_oracle.c: it exists so that the
 * benchmark can time the oracle on all of the host's cores next to its
 * single-thread time. It shares nothing with the CUDA library. The tests
 * check every function here bit for bit against the serial functions of
 * spmv_oracle.c, which stay the definition.
 *
 * What runs in parallel, and why the results are the serial bits:
 *  - SpMV in CRS and ELL-Row: rows are split into contiguous blocks, one per
 *    thread; each row is summed in the same storage (CRS) or slot (ELL,
 *    Fig. 3) order as the serial loop, so every y[i] is the same sum.
 *  - Phase I (Sec. 2.1) count and column pointers: each thread counts the
 *    columns of its block of rows into its own count array; the counts are
 *    added column by column (integers, so the order does not matter), and
 *    the running sum over the columns is taken in two passes (per-thread
 *    sums of column blocks, then each block's pointers from its offset).
 *  - The Phase I scatter stays serial: its row order is what defines the
 *    order of the entries within each column.
 * Compiled with -O2 -ffp-contract=off -fopenmp.
 */
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

int32_t orc_omp_threads(void) { return (int32_t)omp_get_max_threads(); }

static int threads_of(int32_t nthreads) { return nthreads > 0 ? nthreads : omp_get_max_threads(); }

/* CRS SpMV, one plain FP64 sum per row in storage order. */
void orc_omp_spmv_crs(int32_t n_rows, const int32_t *irp, const int32_t *icol, const double *val,
                      const double *x, double *y, int32_t nthreads) {
#pragma omp parallel for schedule(static) num_threads(threads_of(nthreads))
    for (int32_t i = 0; i < n_rows; ++i) {
        double s = 0.0;
        for (int32_t k = irp[i]; k < irp[i + 1]; ++k) s += val[k] * x[icol[k]];
        y[i] = s;
    }
}

/* ELL-Row SpMV: each thread takes a block of rows and sums them slot by
 * slot (slot loop outside, row loop inside, as in Fig. 3). */
void orc_omp_spmv_ell_row(int32_t n_rows, int32_t width, const double *eval, const int32_t *ecol,
                          const double *x, double *y, int32_t nthreads) {
#pragma omp parallel num_threads(threads_of(nthreads))
    {
        const int t = omp_get_thread_num(), T = omp_get_num_threads();
        const int32_t lo = (int32_t)((int64_t)n_rows * t / T), hi = (int32_t)((int64_t)n_rows * (t + 1) / T);
        for (int32_t i = lo; i < hi; ++i) y[i] = 0.0;
        for (int32_t k = 0; k < width; ++k) {
            const int64_t base = (int64_t)k * n_rows;
            for (int32_t i = lo; i < hi; ++i) y[i] += eval[base + i] * x[ecol[base + i]];
        }
    }
}

/* Phase I (Sec. 2.1): parallel count and column pointers, serial scatter in
 * row order. Returns 0, or -1 if the per-thread counts cannot be allocated. */
int32_t orc_omp_crs_to_ccs(int32_t n_rows, int32_t n_cols, const int32_t *irp, const int32_t *icol,
                           const double *val, int32_t *irp_t, int32_t *icol_t, double *val_t, int32_t nthreads) {
    const int T = threads_of(nthreads);
    const size_t nc = (size_t)(n_cols > 0 ? n_cols : 1);
    int32_t *cnt = (int32_t *)calloc((size_t)T * nc, sizeof(int32_t));
    int64_t *part = (int64_t *)calloc((size_t)T + 1, sizeof(int64_t));
    if (!cnt || !part) {
        free(cnt);
        free(part);
        return -1;
    }
    /* count: thread t counts the columns of its rows into cnt[t] */
#pragma omp parallel num_threads(T)
    {
        const int t = omp_get_thread_num(), TT = omp_get_num_threads();
        const int32_t lo = (int32_t)((int64_t)n_rows * t / TT), hi = (int32_t)((int64_t)n_rows * (t + 1) / TT);
        int32_t *c = cnt + (size_t)t * nc;
        for (int32_t i = lo; i < hi; ++i)
            for (int32_t k = irp[i]; k < irp[i + 1]; ++k) c[icol[k]] += 1;
    }
    /* per-column totals into cnt[0], and the sum of each thread's column block */
#pragma omp parallel num_threads(T)
    {
        const int t = omp_get_thread_num(), TT = omp_get_num_threads();
        const int32_t lo = (int32_t)((int64_t)n_cols * t / TT), hi = (int32_t)((int64_t)n_cols * (t + 1) / TT);
        int64_t s = 0;
        for (int32_t j = lo; j < hi; ++j) {
            int32_t v = cnt[j];
            for (int u = 1; u < TT; ++u) v += cnt[(size_t)u * nc + j];
            cnt[j] = v;
            s += v;
        }
        part[t + 1] = s;
#pragma omp barrier
#pragma omp single
        for (int u = 1; u <= TT; ++u) part[u] += part[u - 1];
        /* column pointers of this block from its offset */
        int64_t p = part[t];
        for (int32_t j = lo; j < hi; ++j) {
            irp_t[j] = (int32_t)p;
            p += cnt[j];
        }
        if (t == TT - 1) irp_t[n_cols] = (int32_t)p;
    }
    /* cursors, then the serial scatter in row order */
    for (int32_t j = 0; j < n_cols; ++j) cnt[j] = irp_t[j];
    for (int32_t i = 0; i < n_rows; ++i) {
        for (int32_t k = irp[i]; k < irp[i + 1]; ++k) {
            const int32_t j = icol[k];
            const int32_t p = cnt[j];
            cnt[j] = p + 1;
            val_t[p] = val[k];
            icol_t[p] = i;
        }
    }
    free(cnt);
    free(part);
    return 0;
}
