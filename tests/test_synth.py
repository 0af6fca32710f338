"""Checks of the seeded input generators (shape, determinism, distributions)."""

import math

import numpy as np

import spmv_synth as synth


def test_counter_rng_is_a_pure_function_of_its_counter():
    a = synth.counter_u64(5, 2, np.arange(10))
    b = synth.counter_u64(5, 2, np.arange(20))[:10]
    assert np.array_equal(a, b)
    assert not np.array_equal(a, synth.counter_u64(6, 2, np.arange(10)))
    assert not np.array_equal(a, synth.counter_u64(5, 3, np.arange(10)))


def test_uniform_and_normal_moments():
    u = synth.uniform_pm1(0, 0, np.arange(200000))
    assert u.min() >= -1.0 and u.max() < 1.0
    assert abs(u.mean()) < 0.01 and abs(u.var() - 1 / 3) < 0.01
    z = synth.normal(1, 0, np.arange(200000))
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01


def test_laplacian_and_stencil_shapes():
    A = synth.laplacian_2d_5pt(64)
    assert (A.n_rows, A.nnz) == (4096, 20224)
    B = synth.stencil_3d_27pt(20)
    assert B.nnz == (3 * 20 - 2) ** 3
    lens = np.diff(B.irp)
    rows = np.repeat(np.arange(B.n_rows), lens)
    for i in (0, 4321, B.n_rows - 1):
        seg = slice(B.irp[i], B.irp[i + 1])
        assert np.all(np.diff(B.icol[seg]) > 0)
        d = B.val[seg][B.icol[seg] == i][0]
        off = B.val[seg][B.icol[seg] != i]
        assert d == 27.0 + abs(off.sum())
    assert rows.size == B.nnz


def test_power_law_row_lengths():
    A = synth.power_law(200000)
    lens = np.diff(A.irp)
    assert lens.min() >= 1 and lens.max() <= 20000
    assert abs(lens.mean() - 16.0) < 1.0
    assert math.isclose(synth.power_law_xmin(16.0, 20000.0), 1.7077, abs_tol=1e-4)
    for i in range(0, A.n_rows, 7):
        seg = A.icol[A.irp[i]:A.irp[i + 1]]
        assert np.all(np.diff(seg) > 0) and seg.min() >= 0 and seg.max() < A.n_cols


def test_random_crs_options():
    A = synth.random_crs(300, 100, 5, seed=3, empty_frac=0.5)
    assert (np.diff(A.irp) == 0).sum() > 100
    B = synth.random_crs(300, 100, 5, seed=3, dup=True)
    r = np.repeat(np.arange(B.n_rows), np.diff(B.irp))
    key = r * B.n_cols + B.icol
    assert np.all(np.diff(key) >= 0) and np.any(np.diff(key) == 0)


def test_batch_matrix_recipe():
    # even members: the 5-point stencil of a square grid cut to n rows / cols
    ms = synth.batch_set(40, seed=5)
    ns = np.array([A.n_rows for A in ms])
    assert ns.min() >= 100 and ns.max() <= 20000
    for i, A in enumerate(ms):
        assert A.n_rows == A.n_cols and A.irp[-1] == A.nnz
        seg_ok = all(np.all(np.diff(A.icol[A.irp[r]:A.irp[r + 1]]) > 0) for r in range(0, A.n_rows, 17))
        assert seg_ok and A.icol.min() >= 0 and A.icol.max() < A.n_cols
        if i % 2 == 0:
            g = math.ceil(math.sqrt(A.n_rows))
            full = synth.laplacian_2d_5pt(g)
            # the cut keeps exactly the entries of the full stencil inside [0, n)^2
            n = A.n_rows
            rows = np.repeat(np.arange(full.n_rows), np.diff(full.irp))
            keep = (rows < n) & (full.icol < n)
            assert np.array_equal(A.icol, full.icol[keep]) and np.array_equal(A.val, full.val[keep])
        else:
            assert abs(np.diff(A.irp).mean() - 8.0) < 8.0 * 5 / math.sqrt(A.n_rows * 8.0) + 0.05
    B = synth.batch_matrix(7, seed=5)
    assert np.array_equal(B.icol, ms[7].icol) and np.array_equal(B.val, ms[7].val)
