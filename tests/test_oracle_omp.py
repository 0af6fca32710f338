"""The multi-core oracle build (timed by the benchmark on all host cores)
gives the serial oracle's results bit for bit: CRS and ELL-Row products per
row in the same order, and Phase I's CCS with the serial scatter."""

import numpy as np
import pytest

import oracle
import spmv_synth as synth

CASES = [
    lambda: synth.stencil_3d_27pt(20),
    lambda: synth.power_law(40000, kmax=5000, seed=7),
    lambda: synth.random_crs(3001, 2999, 8, seed=22, dup=True),
    lambda: synth.random_crs(5003, 4001, 6, seed=21, empty_frac=0.3),
    lambda: synth.random_crs(301, 5000, 20, seed=23),
    lambda: synth.CRS(1, 1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([2.5])),
    lambda: synth.CRS(7, 3, np.zeros(8, np.int32), np.zeros(0, np.int32), np.zeros(0)),
]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("nthreads", [0, 1, 3, 8])
def test_omp_build_equals_the_serial_oracle(case, nthreads):
    H = CASES[case]()
    xh = synth.vector_pm1(H.n_cols, seed=5)
    y = oracle.spmv_crs(H.n_rows, H.irp, H.icol, H.val, xh)
    yo = oracle.spmv_crs_omp(H.n_rows, H.irp, H.icol, H.val, xh, nthreads)
    assert np.array_equal(y.view(np.uint64), yo.view(np.uint64))
    ev, ec, W = oracle.crs_to_ell_row(H.n_rows, H.irp, H.icol, H.val)
    y = oracle.spmv_ell_row(H.n_rows, W, ev, ec, xh)
    yo = oracle.spmv_ell_row_omp(H.n_rows, W, ev, ec, xh, nthreads)
    assert np.array_equal(y.view(np.uint64), yo.view(np.uint64))
    irp_t, icol_t, val_t, _ = oracle.crs_to_ccs(H.n_rows, H.n_cols, H.irp, H.icol, H.val)
    p, r, v = oracle.crs_to_ccs_omp(H.n_rows, H.n_cols, H.irp, H.icol, H.val, nthreads)
    assert np.array_equal(p, irp_t) and np.array_equal(r, icol_t)
    assert np.array_equal(v.view(np.uint64), val_t.view(np.uint64))


def test_omp_uses_the_host_cores():
    assert oracle.omp_threads() >= 1
