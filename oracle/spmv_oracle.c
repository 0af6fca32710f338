/*
 * CPU oracle for run-time sparse-format transformation and SpMV
 * (Katagiri & Sato, "An Auto-tuning Method for Run-time Data Transformation
 * for Sparse Matrix-Vector Multiplication").
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, plain, obviously correct
 * definition that the CUDA library is checked against. Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg load it. It shares no
 * code, header, table or constant with the CUDA library, and the library never
 * calls it.
 *
 * Conventions: 0-based indices (the paper's Fortran is 1-based), int32 index
 * arrays, float64 values, serial loops in the paper's order, compiled with
 * -O2 -ffp-contract=off so that no multiply-add is contracted. Outputs are
 * written out of place (the paper's Phase I copies back over its input).
 *
 * Readings of the paper that this file fixes (each is listed with its reason
 * in the design notes of the repository):
 *  - ELL "nz" (Sec. 2.1) is the largest row length W; slot k of line i is
 *    stored at k*n + i (Fig. 3 indexing J_PTR = N*(K-1)+I, 0-based).
 *  - A missing slot holds value +0.0 (Sec. 2.1) and the index of the last
 *    stored entry of its line, or 0 for an empty line.
 *  - Phase I scatters in row order, so each column lists its rows in
 *    ascending order and repeated (i, j) entries in CRS order.
 *  - sigma in Eq. (4) is the population deviation (divide by n).
 *  - Eq. (2) is read as TT_ell = t_trans / t_crs (the printed form is the
 *    reciprocal), so Eq. (3) gives R_ell = t_crs^2 / (t_ell * t_trans).
 *
 * Parity pins: every function here is pinned by a CPU test (dense brute force,
 * library sort, closed forms, Table 1, the Sec. 2.2 worked example) except
 * orc_dstar_from_points for inputs that only GB300 timings would produce:
 * its rule is pinned on hand-built point sets only.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- Eq. (4): D_mat = sigma / mu of the per-row nonzero counts ---------- */
/* mu = mean row length, sigma = population standard deviation, written out
 * in two passes from the definition. W = the largest row length. For nnz = 0
 * (mu = 0), D_mat is reported as 0. */
void orc_analyze(int32_t n_rows, const int32_t *irp, double *mu, double *sigma,
                 double *dmat, int32_t *wmax) {
    double s = 0.0;
    int32_t w = 0;
    for (int32_t i = 0; i < n_rows; ++i) {
        int32_t len = irp[i + 1] - irp[i];
        s += (double)len;
        if (len > w) w = len;
    }
    double m = s / (double)n_rows;
    double q = 0.0;
    for (int32_t i = 0; i < n_rows; ++i) {
        double d = (double)(irp[i + 1] - irp[i]) - m;
        q += d * d;
    }
    double sg = sqrt(q / (double)n_rows);
    *mu = m;
    *sigma = sg;
    *dmat = (m == 0.0) ? 0.0 : sg / m;
    *wmax = w;
}

/* ---- Sec. 2.1: CRS -> COO-Row. VAL and ICOL are the CRS arrays; IROW(k)
 * holds the row of entry k. ---------------------------------------------- */
void orc_crs_to_coo_row(int32_t n_rows, const int32_t *irp, int32_t *irow) {
    for (int32_t i = 0; i < n_rows; ++i)
        for (int32_t k = irp[i]; k < irp[i + 1]; ++k) irow[k] = i;
}

/* ---- Sec. 2.1 / Fig. 3: compressed lines -> ELL, slot k of line i at
 * k*n_lines + i. Used for row-wise ELL (lines = rows, over the CRS) and for
 * column-wise ELL (lines = columns, over the CCS from Phase I). ----------- */
void orc_lines_to_ell(int32_t n_lines, const int32_t *ptr, const int32_t *idx,
                      const double *val, int32_t width, double *eval,
                      int32_t *eidx) {
    for (int32_t k = 0; k < width; ++k) {
        for (int32_t i = 0; i < n_lines; ++i) {
            int32_t len = ptr[i + 1] - ptr[i];
            int64_t slot = (int64_t)k * n_lines + i;
            if (k < len) {
                eval[slot] = val[ptr[i] + k];
                eidx[slot] = idx[ptr[i] + k];
            } else {
                eval[slot] = 0.0;
                eidx[slot] = (len > 0) ? idx[ptr[i + 1] - 1] : 0;
            }
        }
    }
}

/* ---- Sec. 2.1, Phase I: CRS -> CCS by the three serial steps of the paper:
 * count the entries of every column, set the column pointers by a running
 * sum and copy them into per-column cursors, then walk the CRS in row order
 * and drop each entry at its column's cursor. nc (optional) receives the
 * per-column counts. ------------------------------------------------------ */
void orc_crs_to_ccs(int32_t n_rows, int32_t n_cols, const int32_t *irp,
                    const int32_t *icol, const double *val, int32_t *irp_t,
                    int32_t *icol_t, double *val_t, int32_t *nc) {
    int32_t *cnt = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_cols > 0 ? n_cols : 1));
    /* count */
    for (int32_t j = 0; j < n_cols; ++j) cnt[j] = 0;
    for (int32_t i = 0; i < n_rows; ++i)
        for (int32_t k = irp[i]; k < irp[i + 1]; ++k) cnt[icol[k]] += 1;
    if (nc) memcpy(nc, cnt, sizeof(int32_t) * (size_t)n_cols);
    /* column pointers, then cursors */
    irp_t[0] = 0;
    for (int32_t j = 1; j <= n_cols; ++j) irp_t[j] = irp_t[j - 1] + cnt[j - 1];
    for (int32_t j = 0; j < n_cols; ++j) cnt[j] = irp_t[j];
    /* scatter in row order */
    for (int32_t i = 0; i < n_rows; ++i) {
        for (int32_t k = irp[i]; k < irp[i + 1]; ++k) {
            int32_t j = icol[k];
            int32_t p = cnt[j];
            cnt[j] = p + 1;
            val_t[p] = val[k];
            icol_t[p] = i;
        }
    }
    free(cnt);
}

/* ---- Sec. 2.1, Phase II: CCS -> COO-Column. The column of CCS entry p. --- */
void orc_ccs_to_coo_col(int32_t n_cols, const int32_t *irp_t, int32_t *jcol) {
    for (int32_t j = 0; j < n_cols; ++j)
        for (int32_t p = irp_t[j]; p < irp_t[j + 1]; ++p) jcol[p] = j;
}

/* ---- SpMV y = A x, one plain FP64 sum per row in storage order ---------- */

/* CRS (the baseline t_crs of Eq. (1)). */
void orc_spmv_crs(int32_t n_rows, const int32_t *irp, const int32_t *icol,
                  const double *val, const double *x, double *y) {
    for (int32_t i = 0; i < n_rows; ++i) {
        double s = 0.0;
        for (int32_t k = irp[i]; k < irp[i + 1]; ++k) s += val[k] * x[icol[k]];
        y[i] = s;
    }
}

/* COO triplets (Figs. 1 and 2 without the per-thread copies): y starts at
 * zero and every entry adds val * x[col] into y[row] in storage order. */
void orc_spmv_coo(int32_t n_rows, int64_t nnz, const int32_t *row,
                  const int32_t *col, const double *val, const double *x,
                  double *y) {
    for (int32_t i = 0; i < n_rows; ++i) y[i] = 0.0;
    for (int64_t k = 0; k < nnz; ++k) y[row[k]] += val[k] * x[col[k]];
}

/* ELL-Row (Fig. 3 loop order: slot loop outside, row loop inside). */
void orc_spmv_ell_row(int32_t n_rows, int32_t width, const double *eval,
                      const int32_t *ecol, const double *x, double *y) {
    for (int32_t i = 0; i < n_rows; ++i) y[i] = 0.0;
    for (int32_t k = 0; k < width; ++k) {
        int64_t base = (int64_t)k * n_rows;
        for (int32_t i = 0; i < n_rows; ++i)
            y[i] += eval[base + i] * x[ecol[base + i]];
    }
}

/* ELL-Column: slot k of column j holds (value, row); it adds into y[row]. */
void orc_spmv_ell_col(int32_t n_rows, int32_t n_cols, int32_t width,
                      const double *eval, const int32_t *erow, const double *x,
                      double *y) {
    for (int32_t i = 0; i < n_rows; ++i) y[i] = 0.0;
    for (int32_t k = 0; k < width; ++k) {
        int64_t base = (int64_t)k * n_cols;
        for (int32_t j = 0; j < n_cols; ++j)
            y[erow[base + j]] += eval[base + j] * x[j];
    }
}

/* CCS: column j's entries add val * x[j] into y[row]. */
void orc_spmv_ccs(int32_t n_rows, int32_t n_cols, const int32_t *irp_t,
                  const int32_t *icol_t, const double *val_t, const double *x,
                  double *y) {
    for (int32_t i = 0; i < n_rows; ++i) y[i] = 0.0;
    for (int32_t j = 0; j < n_cols; ++j)
        for (int32_t p = irp_t[j]; p < irp_t[j + 1]; ++p)
            y[icol_t[p]] += val_t[p] * x[j];
}

/* ---- Tolerance reference: for each row, y_ref = sum a_ij x_j with every
 * product split exactly (p + e, e = fma(a, x, -p)) and both parts summed with
 * Neumaier's compensated summation; s_ref = sum |a_ij x_j| the same way. The
 * acceptance rule for any SpMV is |y - y_ref| <= tol * s_ref per row. ----- */
static inline void neumaier_add(double *sum, double *c, double t) {
    double s2 = *sum + t;
    if (fabs(*sum) >= fabs(t))
        *c += (*sum - s2) + t;
    else
        *c += (t - s2) + *sum;
    *sum = s2;
}

void orc_spmv_ref(int32_t n_rows, const int32_t *irp, const int32_t *icol,
                  const double *val, const double *x, double *y_ref,
                  double *s_ref) {
    for (int32_t i = 0; i < n_rows; ++i) {
        double s = 0.0, c = 0.0, a = 0.0, ca = 0.0;
        for (int32_t k = irp[i]; k < irp[i + 1]; ++k) {
            double v = val[k], xv = x[icol[k]];
            double p = v * xv;
            double e = fma(v, xv, -p);
            neumaier_add(&s, &c, p);
            neumaier_add(&s, &c, e);
            neumaier_add(&a, &ca, fabs(p));
        }
        y_ref[i] = s + c;
        s_ref[i] = a + ca;
    }
}

/* ---- Sec. 2.2, Eqs. (1)-(3): SP = t_crs / t_ell, TT = t_trans / t_crs
 * (Eq. (2) read as printed-reciprocal), R_ell = SP / TT. -------------------- */
double orc_r_ell(double t_crs, double t_ell, double t_trans) {
    double sp = t_crs / t_ell;
    double tt = t_trans / t_crs;
    return sp / tt;
}

/* ---- Sec. 2.2, off-line step (4): D* from the (D_mat^i, R_ell^i) points.
 * rule 0 (prefix): visit the points by ascending D_mat (ties keep input
 *   order); D* is the D_mat of the first point with R_ell < c; +inf when no
 *   point fails; 0 when the smallest-D_mat point already fails.
 * rule 1 (max-pass): D* is the largest D_mat among points with R_ell >= c,
 *   or 0 if there is none.
 * The on-line test of the paper is strict: ELL iff D_mat < D*. ----------- */
double orc_dstar_from_points(int32_t m, const double *dmat, const double *rell,
                             double c, int32_t rule) {
    if (rule == 1) {
        double best = 0.0;
        int found = 0;
        for (int32_t i = 0; i < m; ++i)
            if (rell[i] >= c && (!found || dmat[i] > best)) {
                best = dmat[i];
                found = 1;
            }
        return found ? best : 0.0;
    }
    /* insertion sort of indices by D_mat (stable) */
    int32_t *ord = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    for (int32_t i = 0; i < m; ++i) {
        int32_t j = i;
        while (j > 0 && dmat[ord[j - 1]] > dmat[i]) {
            ord[j] = ord[j - 1];
            --j;
        }
        ord[j] = i;
    }
    double d = INFINITY;
    for (int32_t t = 0; t < m; ++t) {
        if (rell[ord[t]] < c) {
            d = (t == 0) ? 0.0 : dmat[ord[t]];
            break;
        }
    }
    free(ord);
    return d;
}
