"""Parity at the benchmark sizes, in the launch configuration the bench
times: the 27-point stencil on a 128^3 grid (n = 2,097,152, nnz = 55,742,968)
through the bench's own step (pipelines overlapped on several streams), and
the 4,000,000-row power law. Products are checked on sampled row ranges that
the oracle computes one by one; transformations are compared with the
oracle's in full, bit for bit."""

import numpy as np
import pytest

import oracle
import spmv_synth as synth
from gpu_helpers import assert_spmv_close, bits, lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib()


@pytest.fixture(scope="module")
def stencil128():
    H = synth.stencil_3d_27pt(128, seed=1)
    return H, synth.vector_pm1(H.n_cols, seed=2)


def _sample_starts(n, span, count, seed):
    rng = np.random.default_rng(seed)
    starts = sorted(set([0, n - span] + [int(v) for v in rng.integers(0, n - span, size=count)]))
    return starts


def test_bench_step_products_at_full_size(stencil128):
    import torch

    import bench
    L = lib()
    H, xh = stencil128
    A = L.Crs.from_host(H)
    x = torch.from_numpy(xh).cuda()
    fmts = ["crs", "coo_row", "ell_row", "coo_col", "ell_col"]
    ys = {f: torch.full((H.n_rows,), float("nan"), dtype=torch.float64, device="cuda") for f in fmts}
    step = bench.Step(L, A, x, ys, dstar=0.0, cap=0, concurrent=True)
    step.run()
    step.run()  # twice: the second pass reuses the pool and the streams as the timed steps do
    torch.cuda.synchronize()
    assert step.chosen == "CRS"
    yh = {f: ys[f].cpu().numpy() for f in fmts}
    span = 512
    for r0 in _sample_starts(H.n_rows, span, 12, seed=3):
        S = H.row_slice(r0, r0 + span)
        for f in fmts:
            assert_spmv_close(yh[f][r0:r0 + span], S, xh, what=f"{f} rows {r0}..{r0 + span}")


def test_transformations_bit_exact_at_full_size(stencil128):
    L = lib()
    H, _ = stencil128
    A = L.Crs.from_host(H)
    ccs = L.spmv_transform(A, L.SPMV_CRS, L.SPMV_COLWISE)
    arr = ccs.arrays()
    irp_t, icol_t, val_t, _ = oracle.crs_to_ccs(H.n_rows, H.n_cols, H.irp, H.icol, H.val)
    assert np.array_equal(arr["ptr"].cpu().numpy(), irp_t)
    assert np.array_equal(arr["idx"].cpu().numpy(), icol_t)
    assert np.array_equal(bits(arr["val"].cpu().numpy()), bits(val_t))
    ccs.close()
    ell = L.spmv_transform(A, L.SPMV_ELL, L.SPMV_ROWWISE)
    d = ell.describe()
    W, ld = d["width"], d["ld"]
    ea = ell.arrays()
    ev, ei, rW = oracle.crs_to_ell_row(H.n_rows, H.irp, H.icol, H.val)
    assert W == rW
    gv = ea["val"].cpu().numpy().reshape(W, ld)[:, :H.n_rows]
    gi = ea["idx"].cpu().numpy().reshape(W, ld)[:, :H.n_rows]
    assert np.array_equal(bits(gv), bits(ev.reshape(W, H.n_rows)))
    assert np.array_equal(gi, ei.reshape(W, H.n_rows))
    ell.close()
    coo = L.spmv_transform(A, L.SPMV_COO, L.SPMV_ROWWISE)
    assert np.array_equal(coo.arrays()["idx2"].cpu().numpy(), oracle.crs_to_coo_row(H.n_rows, H.irp))
    coo.close()


def test_power_law_4m_phase1_and_products():
    import torch
    L = lib()
    H = synth.power_law(4_000_000, seed=3)
    xh = synth.vector_pm1(H.n_cols, seed=4)
    A = L.Crs.from_host(H)
    x = torch.from_numpy(xh).cuda()
    # the on-line rule with the 40 GB cap: the ELL (n x W x 12 bytes) does not fit
    M, st = L.spmv_autotune(A, dstar=float("inf"), mem_cap_bytes=40 * 10 ** 9)
    assert M.describe()["format"] == L.SPMV_CRS and st["ell_bytes"] > 40 * 10 ** 9
    ccs = L.spmv_transform(A, L.SPMV_CRS, L.SPMV_COLWISE, 40 * 10 ** 9)
    arr = ccs.arrays()
    irp_t, icol_t, val_t, _ = oracle.crs_to_ccs(H.n_rows, H.n_cols, H.irp, H.icol, H.val)
    assert np.array_equal(arr["ptr"].cpu().numpy(), irp_t)
    assert np.array_equal(arr["idx"].cpu().numpy(), icol_t)
    assert np.array_equal(bits(arr["val"].cpu().numpy()), bits(val_t))
    assert np.diff(irp_t).max() > 32  # long columns: the overflow placement ran
    # every other product at full size: COO-Row (the entry-split product,
    # since 128-row tiles of this matrix exceed shared memory), COO-Column and
    # ELL-Column from the CCS
    coo_row = L.spmv_transform(A, L.SPMV_COO, L.SPMV_ROWWISE, 40 * 10 ** 9)
    coo_col = L.spmv_transform_from(ccs, L.SPMV_COO, 40 * 10 ** 9)
    ell_col = L.spmv_transform_from(ccs, L.SPMV_ELL, 40 * 10 ** 9)
    assert ell_col.describe()["width"] == int(np.diff(irp_t).max())
    ys = {}
    for name, h in (("crs", M), ("ccs", ccs), ("coo_row", coo_row), ("coo_col", coo_col), ("ell_col", ell_col)):
        y = torch.full((H.n_rows,), float("nan"), dtype=torch.float64, device="cuda")
        L.spmv_apply(h, x, y)
        ys[name] = y
    torch.cuda.synchronize()
    span = 1024
    for r0 in _sample_starts(H.n_rows, span, 8, seed=5):
        S = H.row_slice(r0, r0 + span)
        for name, y in ys.items():
            assert_spmv_close(y[r0:r0 + span].cpu().numpy(), S, xh, what=f"power law {name} rows {r0}")
    # the longest rows (thousands of entries, split over many threads) on their own
    lens = np.diff(H.irp)
    for r in np.argsort(lens)[-4:]:
        S = H.row_slice(int(r), int(r) + 1)
        for name, y in ys.items():
            assert_spmv_close(y[int(r):int(r) + 1].cpu().numpy(), S, xh, what=f"power law {name} long row {r}")
    for h in (M, ccs, coo_row, coo_col, ell_col):
        h.close()
