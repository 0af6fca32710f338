"""Pins for the CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each check goes through an
independent route (dense brute force, exact rational arithmetic, a library
sort, a closed form derived from the grid, the paper's printed Table 1 and its
worked example in Sec. 2.2, hand-evaluated rule cases).
"""

import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import spmv_synth as synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dense_from_triplets(n_rows, n_cols, rows, cols, vals):
    A = np.zeros((n_rows, n_cols))
    np.add.at(A, (np.asarray(rows, np.int64), np.asarray(cols, np.int64)), vals)
    return A


def crs_rows(A):
    return np.repeat(np.arange(A.n_rows), np.diff(A.irp))


def small_cases():
    yield synth.random_crs(37, 37, 3, seed=1)
    yield synth.random_crs(64, 50, 6, seed=2, empty_frac=0.3)
    yield synth.random_crs(20, 64, 10, seed=3)
    yield synth.random_crs(1, 1, 1, seed=4)
    yield synth.random_crs(48, 48, 2, seed=5, long_rows=2, long_len=48)
    yield synth.laplacian_2d_5pt(7, 5)


# ---------------------------------------------------------------- transforms


@pytest.mark.parametrize("case", list(range(6)))
def test_every_format_rebuilds_the_dense_matrix(case):
    A = list(small_cases())[case]
    D = dense_from_triplets(A.n_rows, A.n_cols, crs_rows(A), A.icol, A.val)
    # COO-Row
    irow = oracle.crs_to_coo_row(A.n_rows, A.irp)
    assert np.array_equal(dense_from_triplets(A.n_rows, A.n_cols, irow, A.icol, A.val), D)
    # ELL-Row: slot k of row i at k*n + i
    ev, ec, W = oracle.crs_to_ell_row(A.n_rows, A.irp, A.icol, A.val)
    assert W == int(np.diff(A.irp).max())
    rows = np.tile(np.arange(A.n_rows), W)
    assert np.array_equal(dense_from_triplets(A.n_rows, A.n_cols, rows, ec, ev), D)
    # Phase I (CCS) and Phase II (COO-Column)
    irp_t, icol_t, val_t, nc = oracle.crs_to_ccs(A.n_rows, A.n_cols, A.irp, A.icol, A.val)
    jcol = oracle.ccs_to_coo_col(A.n_cols, irp_t)
    assert np.array_equal(dense_from_triplets(A.n_rows, A.n_cols, icol_t, jcol, val_t), D)
    # ELL-Column
    ev2, er2, W2 = oracle.ccs_to_ell_col(A.n_cols, irp_t, icol_t, val_t)
    cols = np.tile(np.arange(A.n_cols), W2)
    assert np.array_equal(dense_from_triplets(A.n_rows, A.n_cols, er2, cols, ev2), D)


def test_phase1_equals_a_stable_library_sort_by_column():
    for A in list(small_cases()) + [synth.random_crs(300, 200, 7, seed=9, dup=True)]:
        irp_t, icol_t, val_t, nc = oracle.crs_to_ccs(A.n_rows, A.n_cols, A.irp, A.icol, A.val)
        perm = np.argsort(A.icol, kind="stable")
        assert np.array_equal(icol_t, crs_rows(A)[perm])
        assert np.array_equal(val_t.view(np.uint64), A.val[perm].view(np.uint64))
        assert np.array_equal(irp_t, np.searchsorted(A.icol[perm], np.arange(A.n_cols + 1)))
        assert np.array_equal(nc, np.bincount(A.icol, minlength=A.n_cols))
        assert int(nc.sum()) == A.nnz


def test_phase1_twice_returns_the_crs():
    for A in list(small_cases()) + [synth.random_crs(300, 200, 7, seed=9, dup=True)]:
        irp_t, icol_t, val_t, _ = oracle.crs_to_ccs(A.n_rows, A.n_cols, A.irp, A.icol, A.val)
        irp2, icol2, val2, _ = oracle.crs_to_ccs(A.n_cols, A.n_rows, irp_t, icol_t, val_t)
        assert np.array_equal(irp2, A.irp)
        assert np.array_equal(icol2, A.icol)
        assert np.array_equal(val2.view(np.uint64), A.val.view(np.uint64))


def test_ell_padding_is_positive_zero_and_reconstructs_crs():
    A = synth.random_crs(200, 150, 5, seed=11, empty_frac=0.1)
    ev, ec, W = oracle.crs_to_ell_row(A.n_rows, A.irp, A.icol, A.val)
    lens = np.diff(A.irp)
    ev2 = ev.reshape(W, A.n_rows)
    ec2 = ec.reshape(W, A.n_rows)
    pad = np.arange(W)[:, None] >= lens[None, :]
    assert np.all(ev2[pad].view(np.uint64) == 0)  # +0.0 exactly
    # padding index: last stored column of the row, 0 for an empty row
    last = np.where(lens > 0, A.icol[np.maximum(A.irp[1:] - 1, 0)], 0)
    assert np.array_equal(ec2[pad], np.broadcast_to(last, ec2.shape)[pad])
    # first len_i slots of each row, in slot order, give back the CRS row
    rec_c = np.concatenate([ec2[:l, i] for i, l in enumerate(lens)])
    rec_v = np.concatenate([ev2[:l, i] for i, l in enumerate(lens)])
    assert np.array_equal(rec_c, A.icol)
    assert np.array_equal(rec_v.view(np.uint64), A.val.view(np.uint64))
    assert int(pad.sum()) == W * A.n_rows - A.nnz


def test_coo_row_is_the_row_of_each_entry():
    A = synth.random_crs(500, 500, 4, seed=12, empty_frac=0.2)
    assert np.array_equal(oracle.crs_to_coo_row(A.n_rows, A.irp), crs_rows(A))


# ------------------------------------------------------------------ SpMV


def exact_spmv(A, x):
    """A x in exact rational arithmetic (tiny inputs only)."""
    out = []
    for i in range(A.n_rows):
        s = Fraction(0)
        for k in range(int(A.irp[i]), int(A.irp[i + 1])):
            s += Fraction(float(A.val[k])) * Fraction(float(x[A.icol[k]]))
        out.append(s)
    return out


def test_compensated_reference_is_correctly_rounded_on_tiny_inputs():
    for A in [synth.random_crs(30, 30, 8, seed=21), synth.random_crs(12, 40, 30, seed=22)]:
        x = synth.vector_pm1(A.n_cols, seed=23)
        y_ref, s_ref = oracle.spmv_ref(A.n_rows, A.irp, A.icol, A.val, x)
        ex = exact_spmv(A, x)
        for i in range(A.n_rows):
            # within one unit in the last place of the exact value
            assert abs(Fraction(float(y_ref[i])) - ex[i]) <= Fraction(2.0 ** -52) * abs(ex[i]) + Fraction(2.0 ** -1074)
            sa = sum(abs(Fraction(float(A.val[k])) * Fraction(float(x[A.icol[k]])))
                     for k in range(int(A.irp[i]), int(A.irp[i + 1])))
            assert abs(Fraction(float(s_ref[i])) - sa) <= Fraction(2.0 ** -50) * sa


@pytest.mark.parametrize("case", list(range(6)))
def test_every_format_spmv_matches_dense_product(case):
    A = list(small_cases())[case]
    x = synth.vector_pm1(A.n_cols, seed=31)
    D = dense_from_triplets(A.n_rows, A.n_cols, crs_rows(A), A.icol, A.val)
    y_dense = D @ x
    y_ref, s = oracle.spmv_ref(A.n_rows, A.irp, A.icol, A.val, x)
    tol = 1e-13 * s + 1e-300
    assert np.all(np.abs(y_dense - y_ref) <= tol)
    irow = oracle.crs_to_coo_row(A.n_rows, A.irp)
    ev, ec, W = oracle.crs_to_ell_row(A.n_rows, A.irp, A.icol, A.val)
    irp_t, icol_t, val_t, _ = oracle.crs_to_ccs(A.n_rows, A.n_cols, A.irp, A.icol, A.val)
    jcol = oracle.ccs_to_coo_col(A.n_cols, irp_t)
    ev2, er2, W2 = oracle.ccs_to_ell_col(A.n_cols, irp_t, icol_t, val_t)
    ys = {
        "crs": oracle.spmv_crs(A.n_rows, A.irp, A.icol, A.val, x),
        "coo_row": oracle.spmv_coo(A.n_rows, irow, A.icol, A.val, x),
        "coo_col": oracle.spmv_coo(A.n_rows, icol_t, jcol, val_t, x),
        "ell_row": oracle.spmv_ell_row(A.n_rows, W, ev, ec, x),
        "ell_col": oracle.spmv_ell_col(A.n_rows, A.n_cols, W2, ev2, er2, x),
        "ccs": oracle.spmv_ccs(A.n_rows, A.n_cols, irp_t, icol_t, val_t, x),
    }
    for name, y in ys.items():
        assert np.all(np.abs(y - y_ref) <= tol), name


def test_crs_spmv_sums_in_storage_order():
    # one row whose sum depends on order: 1e16 + 1 - 1e16 (storage order) = 0
    irp = np.array([0, 3], np.int32)
    icol = np.array([0, 1, 2], np.int32)
    val = np.array([1e16, 1.0, -1e16])
    x = np.ones(3)
    assert oracle.spmv_crs(1, irp, icol, val, x)[0] == 0.0
    y_ref, s = oracle.spmv_ref(1, irp, icol, val, x)
    assert y_ref[0] == 1.0


# ------------------------------------------------------- Eq. (4) closed forms


def test_laplacian_64x64_closed_form():
    A = synth.laplacian_2d_5pt(64)
    # grid counts: 4 corners (3 entries), 248 edge points (4), 3844 interior (5)
    counts = {3: 4, 4: 4 * 62, 5: 62 * 62}
    n = sum(counts.values())
    nnz = sum(k * v for k, v in counts.items())
    mu = Fraction(nnz, n)
    var = Fraction(sum(k * k * v for k, v in counts.items()), n) - mu * mu
    st = oracle.analyze(A.n_rows, A.irp)
    assert (n, nnz) == (4096, 20224) == (A.n_rows, A.nnz)
    assert st["mu"] == 4.9375 == float(mu)
    assert math.isclose(st["sigma"], math.sqrt(var), rel_tol=1e-14)
    assert math.isclose(st["sigma"], 0.246063, abs_tol=5e-7)
    assert math.isclose(st["dmat"], 0.0498355, abs_tol=5e-8)
    assert st["W"] == 5
    ev, ec, W = oracle.crs_to_ell_row(A.n_rows, A.irp, A.icol, A.val)
    assert W * A.n_rows - A.nnz == 256


def stencil27_irp(N):
    """Row pointers of the 27-point pattern from per-axis neighbour counts."""
    c = np.full(N, 3, np.int64)
    c[0] = c[-1] = 2
    lens = (c[:, None, None] * c[None, :, None] * c[None, None, :]).reshape(-1)
    irp = np.zeros(N ** 3 + 1, np.int64)
    np.cumsum(lens, out=irp[1:])
    return irp.astype(np.int32)


@pytest.mark.parametrize("N", [16, 128])
def test_27pt_closed_form(N):
    irp = stencil27_irp(N)
    n = N ** 3
    # per axis: count c = 2 at the two faces, 3 inside; row length = product
    e1 = Fraction(2 * 2 + 3 * (N - 2), N)
    e2 = Fraction(2 * 4 + 9 * (N - 2), N)
    mu, m2 = e1 ** 3, e2 ** 3
    st = oracle.analyze(n, irp)
    assert int(irp[-1]) == (3 * N - 2) ** 3
    assert math.isclose(st["mu"], float(mu), rel_tol=1e-15)
    # plain recursive summation of n non-negative terms: relative error <= n*u
    assert math.isclose(st["sigma"], math.sqrt(m2 - mu * mu), rel_tol=n * 2.0 ** -53)
    assert st["W"] == 27
    if N == 128:
        assert int(irp[-1]) == 55742968
        assert math.isclose(st["dmat"], 0.0720398, abs_tol=5e-8)
    if N == 16:
        A = synth.stencil_3d_27pt(16)
        assert np.array_equal(A.irp, irp)


def test_symmetric_laplacian_ccs_equals_crs():
    A = synth.laplacian_2d_5pt(64)
    irp_t, icol_t, val_t, nc = oracle.crs_to_ccs(A.n_rows, A.n_cols, A.irp, A.icol, A.val)
    assert np.array_equal(irp_t, A.irp)
    assert np.array_equal(icol_t, A.icol)
    assert np.array_equal(val_t.view(np.uint64), A.val.view(np.uint64))


def test_27pt_pattern_is_structurally_symmetric():
    A = synth.stencil_3d_27pt(12)
    irp_t, icol_t, val_t, nc = oracle.crs_to_ccs(A.n_rows, A.n_cols, A.irp, A.icol, A.val)
    assert np.array_equal(irp_t, A.irp)
    assert np.array_equal(icol_t, A.icol)


def test_laplacian_times_ones_gives_exact_row_sums():
    A = synth.laplacian_2d_5pt(64)
    y = oracle.spmv_crs(A.n_rows, A.irp, A.icol, A.val, np.ones(A.n_cols))
    i = np.arange(A.n_rows)
    gx, gy = i % 64, i // 64
    missing = (gx == 0).astype(int) + (gx == 63) + (gy == 0) + (gy == 63)
    assert np.array_equal(y, missing.astype(float))  # interior rows exactly 0.0


# ---------------------------------------------------------- Table 1 (Sec 4.2)


def table1():
    rows = []
    with open(os.path.join(GOLDEN, "table1_test_matrices.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            no, name, n, nnz, mu, sg, dm = line.split()
            rows.append((int(no), name, int(n), int(nnz), float(mu), float(sg), float(dm)))
    return rows


def lengths_with(n, nnz, sigma):
    """Integer row lengths with sum exactly nnz and deviation close to sigma.

    Two levels a <= mu <= b: m rows of length b, the rest a, one row absorbing
    the rounding of the total. The pair (a, b) is chosen by the deviation the
    integer lengths actually reach, near the continuous two-point solution
    (mu - a)(b - mu) = sigma^2.
    """
    mu = nnz / n

    def build(a, b):
        m = int(round((nnz - a * n) / (b - a)))
        if not 0 < m <= n:
            return None
        lens = np.full(n, a, np.int64)
        lens[:m] = b
        lens[0] += nnz - int(lens.sum())
        return lens if lens.min() >= 0 else None

    best = None
    for a in range(0, int(math.floor(mu)) + 1):
        if mu - a <= 0:
            continue
        bstar = mu + sigma * sigma / (mu - a)
        for b in {int(math.ceil(mu)), *range(max(a + 1, int(bstar) - 2), int(bstar) + 3)}:
            if b <= a:
                continue
            lens = build(a, b)
            if lens is None:
                continue
            err = abs(float(np.std(lens)) - sigma)
            if best is None or err < best[0]:
                best = (err, lens)
    # three levels c-1, c, c+1 around c = round(mu): fractions p-, p+ with
    # p+ - p- = mu - c and p+ + p- = sigma^2 + (mu - c)^2
    c = int(round(mu))
    d = mu - c
    pp, pm = (sigma ** 2 + d * d + d) / 2, (sigma ** 2 + d * d - d) / 2
    if c >= 1 and pp >= 0 and pm >= 0 and pp + pm <= 1:
        mp, mm = int(round(pp * n)), int(round(pm * n))
        lens = np.full(n, c, np.int64)
        lens[:mp] = c + 1
        lens[mp:mp + mm] = c - 1
        lens[-1] += nnz - int(lens.sum())
        err = abs(float(np.std(lens)) - sigma)
        if lens.min() >= 0 and err < best[0]:
            best = (err, lens)
    lens = best[1]
    assert int(lens.sum()) == nnz and lens.min() >= 0
    return lens


def test_table1_mean_is_nnz_over_n():
    bad = []
    for no, name, n, nnz, mu, sg, dm in table1():
        lens = lengths_with(n, nnz, sg)
        irp = np.concatenate(([0], np.cumsum(lens))).astype(np.int32)
        st = oracle.analyze(n, irp)
        assert math.isclose(st["mu"], nnz / n, rel_tol=1e-15)
        if math.floor(st["mu"] * 100 + 1e-9) / 100 != mu:
            bad.append(name)
    assert bad == ["torso2"]  # printed 8.91, 1033473 / 115067 = 8.98


def test_table1_dmat_is_sigma_over_mu():
    for no, name, n, nnz, mu, sg, dm in table1():
        # the printed columns agree with Eq. (4) to the printed precision
        assert abs(sg / mu - dm) <= 0.01 + 1e-12, name
        lens = lengths_with(n, nnz, sg)
        irp = np.concatenate(([0], np.cumsum(lens))).astype(np.int32)
        st = oracle.analyze(n, irp)
        assert abs(st["sigma"] - sg) <= 0.02 * sg + 0.006, name
        assert abs(st["dmat"] - dm) <= 0.011, name


# ------------------------------------------------------- Sec. 2.2 AT pieces


def test_worked_example_of_eq3():
    with open(os.path.join(GOLDEN, "rell_worked_example.txt")) as f:
        sp, tt, r = [float(v) for v in [l for l in f if not l.startswith("#")][0].split()]
    t_crs = 1.0
    t_ell = t_crs / sp
    t_trans = tt * t_crs  # TT = t_trans / t_crs, the reading the example fixes
    assert math.isclose(oracle.r_ell(t_crs, t_ell, t_trans), r, rel_tol=1e-15)
    # the reciprocal form printed as Eq. (2) would give 100, not 1.0
    assert math.isclose(sp / (t_crs / t_trans), 100.0)


def test_dstar_rules_on_hand_built_points():
    d = [0.02, 0.10, 0.50, 0.30, 3.10]
    r = [5.0, 2.0, 0.8, 1.5, 2.0]
    assert oracle.dstar_from_points(d, r, 1.0, 0) == 0.50
    assert oracle.dstar_from_points(d, r, 1.0, 1) == 3.10
    assert oracle.dstar_from_points(d, [2.0] * 5, 1.0, 0) == math.inf
    assert oracle.dstar_from_points(d, [0.5, 2, 2, 2, 2], 1.0, 0) == 0.0
    assert oracle.dstar_from_points(d, [0.5] * 5, 1.0, 1) == 0.0
    # c is the threshold: R exactly c passes (R_ell >= c is advantageous, Sec. 2.2), under both rules
    assert oracle.dstar_from_points([0.1, 0.2], [1.0, 0.999], 1.0, 0) == 0.2
    assert oracle.dstar_from_points([0.1, 0.2], [1.0, 0.999], 1.0, 1) == 0.1
    assert oracle.dstar_from_points([0.1, 0.2], [1.5, 1.0], 1.0, 1) == 0.2
    assert oracle.dstar_from_points([], [], 1.0, 0) == math.inf
