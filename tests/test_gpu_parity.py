"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Transformations must match bit for bit; SpMV within 1e-12 * sum_j |a_ij x_j|
per row. Sizes span several tiles of every kernel and leave ragged tails.
"""

import numpy as np
import pytest

import oracle
import spmv_synth as synth
from gpu_helpers import TOL, assert_spmv_close, bits, dev, ell_from_gpu, lib, run_apply, xvec

pytestmark = pytest.mark.gpu


def dense_col_matrix(n=9000, seed=5):
    """Random rows plus column 7 in every row (a 9000-long column) and
    column 11 in every 60th row (a 150-long column)."""
    base = synth.random_crs(n, n, 4, seed=seed)
    rows = []
    for i in range(n):
        c = set(base.icol[base.irp[i]:base.irp[i + 1]].tolist())
        c.add(7)
        if i % 60 == 0:
            c.add(11)
        rows.append(sorted(c))
    irp = np.zeros(n + 1, np.int64)
    irp[1:] = np.cumsum([len(r) for r in rows])
    icol = np.concatenate([np.array(r, np.int32) for r in rows])
    val = synth.normal(seed, 77, np.arange(icol.size))
    return synth.CRS(n, n, irp.astype(np.int32), icol, val)


CASES = {
    "laplace64": lambda: synth.laplacian_2d_5pt(64),
    "laplace37x23": lambda: synth.laplacian_2d_5pt(37, 23),
    "stencil27_24": lambda: synth.stencil_3d_27pt(24),
    "stencil27_37": lambda: synth.stencil_3d_27pt(37),
    "laplace300x221": lambda: synth.laplacian_2d_5pt(300, 221),
    "powerlaw_60k": lambda: synth.power_law(60000, kmax=20000),
    "random_empty_rows": lambda: synth.random_crs(5003, 4001, 6, seed=21, empty_frac=0.3),
    "random_duplicates": lambda: synth.random_crs(3001, 2999, 8, seed=22, dup=True),
    "wide": lambda: synth.random_crs(301, 5000, 20, seed=23),
    "tall": lambda: synth.random_crs(5000, 301, 3, seed=24),
    "one_by_one": lambda: synth.CRS(1, 1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([2.5])),
    "all_empty": lambda: synth.CRS(100, 100, np.zeros(101, np.int32), np.zeros(0, np.int32), np.zeros(0)),
    "long_row": lambda: synth.random_crs(4000, 6000, 3, seed=25, long_rows=3, long_len=5000),
    "dense_column": dense_col_matrix,
}

_cache = {}


def crs_uneven(H):
    """The CRS schedule takes the entry-split product: D_mat > 0.5 or a row of
    2048 entries or more (the plan's rule for uneven rows)."""
    st = oracle.analyze(H.n_rows, H.irp)
    return st["dmat"] > 0.5 or st["W"] >= 2048


def coo_tiles_overflow(H):
    """The COO-Row schedule takes the entry-split product: some 128-row tile
    holds more entries than the row-tile kernel stages (6144)."""
    edges = H.irp[np.minimum(np.arange(0, H.n_rows + 128, 128), H.n_rows)].astype(np.int64)
    return H.nnz > 0 and int(np.diff(edges).max()) * 16 > 96 * 1024


def case(name):
    if name not in _cache:
        _cache[name] = CASES[name]()
    return _cache[name]


@pytest.fixture(scope="module", autouse=True)
def _device():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib()


@pytest.mark.parametrize("name", list(CASES))
def test_analyze(name):
    H = case(name)
    st = lib().spmv_analyze(dev(H))
    ref = oracle.analyze(H.n_rows, H.irp)
    assert st["W"] == ref["W"]
    rel = H.n_rows * 2.0 ** -53 + 1e-15
    for k in ("mu", "sigma", "dmat"):
        assert abs(st[k] - ref[k]) <= rel * abs(ref[k]), k
    lens = np.diff(H.irp)
    assert st["n_empty"] == int((lens == 0).sum())
    assert st["min_len"] == int(lens.min())
    cls = np.where(lens == 0, 0, np.floor(np.log2(np.maximum(lens, 1))).astype(int) + 1)
    assert st["hist"] == np.bincount(cls, minlength=32).tolist()


@pytest.mark.parametrize("name", list(CASES))
def test_rowwise_transforms_bit_exact(name):
    H = case(name)
    L = lib()
    A = dev(H)
    # COO-Row: IROW, with VAL / ICOL borrowed from the CRS
    M = L.spmv_transform(A, L.SPMV_COO, L.SPMV_ROWWISE)
    arr = M.arrays()
    assert np.array_equal(arr["idx2"].cpu().numpy(), oracle.crs_to_coo_row(H.n_rows, H.irp))
    assert arr["idx"].data_ptr() == A.icol.data_ptr() or H.nnz == 0
    M.close()
    # ELL-Row
    M = L.spmv_transform(A, L.SPMV_ELL, L.SPMV_ROWWISE)
    W, ld, ev, ei = ell_from_gpu(M, H.n_rows)
    rv, ri, rW = oracle.crs_to_ell_row(H.n_rows, H.irp, H.icol, H.val)
    assert W == rW and ld >= H.n_rows and ld % 32 == 0
    if W:
        assert np.array_equal(bits(ev[:, :H.n_rows]), bits(rv.reshape(W, H.n_rows)))
        assert np.array_equal(ei[:, :H.n_rows], ri.reshape(W, H.n_rows))
        assert np.all(bits(ev[:, H.n_rows:]) == 0) and np.all(ei[:, H.n_rows:] == 0)
    M.close()


@pytest.mark.parametrize("name", list(CASES))
def test_colwise_transforms_bit_exact(name):
    H = case(name)
    L = lib()
    A = dev(H)
    irp_t, icol_t, val_t, nc = oracle.crs_to_ccs(H.n_rows, H.n_cols, H.irp, H.icol, H.val)
    ccs = L.spmv_transform(A, L.SPMV_CRS, L.SPMV_COLWISE)
    arr = ccs.arrays()
    assert np.array_equal(arr["ptr"].cpu().numpy(), irp_t)
    assert np.array_equal(arr["idx"].cpu().numpy(), icol_t)
    assert np.array_equal(bits(arr["val"].cpu().numpy()), bits(val_t))
    # Phase II from the CCS handle, and the direct Phase I + II call
    jcol = oracle.ccs_to_coo_col(H.n_cols, irp_t)
    coo = L.spmv_transform_from(ccs, L.SPMV_COO)
    assert np.array_equal(coo.arrays()["idx2"].cpu().numpy(), jcol)
    coo2 = L.spmv_transform(A, L.SPMV_COO, L.SPMV_COLWISE)
    a2 = coo2.arrays()
    assert np.array_equal(a2["idx2"].cpu().numpy(), jcol)
    assert np.array_equal(a2["idx"].cpu().numpy(), icol_t)
    assert np.array_equal(bits(a2["val"].cpu().numpy()), bits(val_t))
    # ELL-Column, from the CCS handle and directly
    rv, rr, rW = oracle.ccs_to_ell_col(H.n_cols, irp_t, icol_t, val_t)
    for M in (L.spmv_transform_from(ccs, L.SPMV_ELL), L.spmv_transform(A, L.SPMV_ELL, L.SPMV_COLWISE)):
        W, ld, ev, ei = ell_from_gpu(M, H.n_cols)
        assert W == rW
        if W:
            assert np.array_equal(bits(ev[:, :H.n_cols]), bits(rv.reshape(W, H.n_cols)))
            assert np.array_equal(ei[:, :H.n_cols], rr.reshape(W, H.n_cols))
        M.close()
    # the CCS arrays outlive the handle that built them
    ccs.close()
    assert np.array_equal(coo.arrays()["idx"].cpu().numpy(), icol_t)
    coo.close()
    coo2.close()


@pytest.mark.parametrize("name", list(CASES))
def test_spmv_every_format(name):
    import torch
    H = case(name)
    L = lib()
    A = dev(H)
    xh = xvec(H.n_cols, seed=3)
    x = torch.from_numpy(xh).cuda()
    mats = {
        "crs": L.spmv_transform(A, L.SPMV_CRS, L.SPMV_ROWWISE),
        "coo_row": L.spmv_transform(A, L.SPMV_COO, L.SPMV_ROWWISE),
        "ell_row": L.spmv_transform(A, L.SPMV_ELL, L.SPMV_ROWWISE),
        "ccs": L.spmv_transform(A, L.SPMV_CRS, L.SPMV_COLWISE),
    }
    mats["coo_col"] = L.spmv_transform_from(mats["ccs"], L.SPMV_COO)
    mats["ell_col"] = L.spmv_transform_from(mats["ccs"], L.SPMV_ELL)
    for fmt, M in mats.items():
        y = run_apply(M, x, H.n_rows)
        assert_spmv_close(y, H, xh, what=f"{name}/{fmt}")
        # row-wise products sum in a fixed order and repeat bit for bit, except
        # the entry-split product of uneven rows, which adds row pieces with atomics
        if fmt == "ell_row" or (fmt == "crs" and not crs_uneven(H)) or (fmt == "coo_row" and not coo_tiles_overflow(H)):
            assert np.array_equal(bits(run_apply(M, x, H.n_rows)), bits(y)), fmt
    for M in mats.values():
        M.close()


@pytest.mark.parametrize("name", ["laplace64", "stencil27_24", "powerlaw_60k", "random_empty_rows", "all_empty"])
def test_fused_transform_and_first_spmv(name):
    import torch
    H = case(name)
    L = lib()
    A = dev(H)
    xh = xvec(H.n_cols, seed=4)
    x = torch.from_numpy(xh).cuda()
    y = torch.full((H.n_rows,), float("nan"), dtype=torch.float64, device="cuda")
    M = L.spmv_transform_apply(A, x, y)
    torch.cuda.synchronize()
    assert_spmv_close(y.cpu().numpy(), H, xh, what=f"{name}/fused")
    W, ld, ev, ei = ell_from_gpu(M, H.n_rows)
    rv, ri, rW = oracle.crs_to_ell_row(H.n_rows, H.irp, H.icol, H.val)
    assert W == rW
    if W:
        assert np.array_equal(bits(ev[:, :H.n_rows]), bits(rv.reshape(W, H.n_rows)))
        assert np.array_equal(ei[:, :H.n_rows], ri.reshape(W, H.n_rows))
    M.close()


def test_crs_schedule_for_uneven_rows():
    """Uneven rows take the entry-split product: rows crossing thread and
    tile edges, rows of one entry, empty rows and rows thousands of entries
    long all land inside the tolerance."""
    import torch
    L = lib()
    mats = [synth.power_law(30000, kmax=8000, seed=9), case("powerlaw_60k"), case("long_row"),
            case("random_empty_rows"), case("dense_column"), case("random_duplicates")]
    for i, H in enumerate(mats):
        A = dev(H)
        xh = xvec(H.n_cols, seed=5 + i)
        M = L.spmv_transform(A, L.SPMV_CRS, L.SPMV_ROWWISE)
        for rep in range(2):
            assert_spmv_close(run_apply(M, torch.from_numpy(xh).cuda(), H.n_rows), H, xh, what=f"seg/{i}/{rep}")
        M.close()
    assert L.spmv_analyze(dev(mats[0]))["dmat"] > 0.5  # the first one is uneven


def test_unaligned_caller_arrays_take_the_global_path():
    """VAL / ICOL not 16-byte aligned: the TMA-staged kernels fall back to
    plain loads and give the same bits."""
    import torch
    L = lib()
    H = synth.stencil_3d_27pt(16)
    icol = torch.empty(H.nnz + 1, dtype=torch.int32, device="cuda")[1:]
    val = torch.empty(H.nnz + 1, dtype=torch.float64, device="cuda")[1:]
    icol.copy_(torch.from_numpy(H.icol))
    val.copy_(torch.from_numpy(H.val))
    assert icol.data_ptr() % 16 and val.data_ptr() % 16
    A = L.Crs(H.n_rows, H.n_cols, torch.from_numpy(H.irp).cuda(), icol, val)
    xh = xvec(H.n_cols, seed=6)
    x = torch.from_numpy(xh).cuda()
    M = L.spmv_transform(A, L.SPMV_ELL, L.SPMV_ROWWISE)
    W, ld, ev, ei = ell_from_gpu(M, H.n_rows)
    rv, ri, rW = oracle.crs_to_ell_row(H.n_rows, H.irp, H.icol, H.val)
    assert np.array_equal(bits(ev[:, :H.n_rows]), bits(rv.reshape(W, H.n_rows)))
    assert np.array_equal(ei[:, :H.n_rows], ri.reshape(W, H.n_rows))
    M.close()
    for fmt, lay in ((L.SPMV_CRS, L.SPMV_ROWWISE), (L.SPMV_COO, L.SPMV_COLWISE)):
        M = L.spmv_transform(A, fmt, lay)
        assert_spmv_close(run_apply(M, x, H.n_rows), H, xh, what=f"unaligned {fmt}/{lay}")
        M.close()


def test_outputs_at_any_8_byte_offset():
    """y (and x) need only 8-byte alignment: every row-wise format writes the
    same bits into y + 1 as into an aligned y."""
    import torch
    L = lib()
    H = synth.laplacian_2d_5pt(37, 23)  # odd row count
    A = dev(H)
    xh = xvec(H.n_cols, seed=8)
    xb = torch.empty(H.n_cols + 1, dtype=torch.float64, device="cuda")
    xb[1:].copy_(torch.from_numpy(xh))
    for fmt in (L.SPMV_CRS, L.SPMV_COO, L.SPMV_ELL):
        M = L.spmv_transform(A, fmt, L.SPMV_ROWWISE)
        ya = torch.empty(H.n_rows, dtype=torch.float64, device="cuda")
        yb = torch.full((H.n_rows + 1,), float("nan"), dtype=torch.float64, device="cuda")
        L.spmv_apply(M, xb[1:], ya)
        L.spmv_apply(M, xb[1:], yb[1:])
        torch.cuda.synchronize()
        assert np.array_equal(bits(ya.cpu().numpy()), bits(yb[1:].cpu().numpy()))
        assert_spmv_close(ya.cpu().numpy(), H, xh, what=f"offset y, format {fmt}")
        M.close()


@pytest.mark.parametrize("split", [1, 2, 4, 8, -1])
def test_crs_kernel_variants(split):
    """Every CRS schedule for regular rows (1, 2, 4 or 8 threads per row of a
    staged tile; -1: V lanes per row without staging) gives results inside
    the tolerance, on cases of one to several hundred row tiles with ragged
    last tiles."""
    import torch
    L = lib()
    for name in ("laplace37x23", "stencil27_24", "laplace300x221", "stencil27_37"):
        H = case(name)
        xh = xvec(H.n_cols, seed=7)
        with L.hint(L.SPMV_HINT_CRS_SPLIT, split):
            M = L.spmv_transform(dev(H), L.SPMV_CRS, L.SPMV_ROWWISE)
        y = run_apply(M, torch.from_numpy(xh).cuda(), H.n_rows)
        assert_spmv_close(y, H, xh, what=f"{name}/split={split}")
        assert np.array_equal(bits(run_apply(M, torch.from_numpy(xh).cuda(), H.n_rows)), bits(y))
        M.close()


def test_crs_vector_kernel_on_rows_too_long_for_a_staged_tile():
    """Regular rows longer than 64 entries (a 128-row tile would not fit
    shared memory) take the V-lanes-per-row kernel without any hint."""
    import torch
    L = lib()
    H = synth.banded_random_crs(3000, 300000, 10.0, seed=31)  # mean 100, D_mat 0.10, W 146
    st = oracle.analyze(H.n_rows, H.irp)
    assert st["dmat"] <= 0.5 and st["W"] > 64
    xh = xvec(H.n_cols, seed=32)
    M = L.spmv_transform(dev(H), L.SPMV_CRS, L.SPMV_ROWWISE)
    L.spmv_profile_enable(True)
    L.spmv_profile_read(reset=True)
    try:
        y = run_apply(M, torch.from_numpy(xh).cuda(), H.n_rows)
        prof = L.spmv_profile_read(reset=True)
    finally:
        L.spmv_profile_enable(False)
    assert any(k.startswith("spmv_crs_v") for k in prof), prof
    assert_spmv_close(y, H, xh, what="vector kernel")
    M.close()


@pytest.mark.parametrize("flat", [0, 1])
def test_coo_row_schedules(flat):
    """Row-aligned tiles and the entry-split product agree with the oracle."""
    import torch
    L = lib()
    for name in ("laplace37x23", "stencil27_24", "random_empty_rows", "long_row", "all_empty", "powerlaw_60k",
                 "dense_column", "one_by_one"):
        H = case(name)
        xh = xvec(H.n_cols, seed=8)
        with L.hint(L.SPMV_HINT_COO_FLAT, flat):
            M = L.spmv_transform(dev(H), L.SPMV_COO, L.SPMV_ROWWISE)
        assert_spmv_close(run_apply(M, torch.from_numpy(xh).cuda(), H.n_rows), H, xh,
                          what=f"{name}/flat={flat}")
        M.close()


@pytest.mark.parametrize("flat", [0, 1])
def test_coo_col_schedules(flat):
    """Column-aligned tiles (lanes on consecutive columns) and the flat entry
    kernel agree with the oracle; a 9000-entry column exceeds the tile
    capacity and takes the flat kernel either way."""
    import torch
    L = lib()
    for name in ("laplace37x23", "stencil27_24", "random_empty_rows", "wide", "tall", "dense_column", "all_empty",
                 "powerlaw_60k"):
        H = case(name)
        xh = xvec(H.n_cols, seed=9)
        C = L.spmv_transform(dev(H), L.SPMV_CRS, L.SPMV_COLWISE)
        with L.hint(L.SPMV_HINT_COO_FLAT, flat):
            M = L.spmv_transform_from(C, L.SPMV_COO)
        C.close()
        for rep in range(2):
            assert_spmv_close(run_apply(M, torch.from_numpy(xh).cuda(), H.n_rows), H, xh,
                              what=f"{name}/flat={flat}/{rep}")
        M.close()


def _ccs_matches_oracle(M, H):
    irp_t, icol_t, val_t, _ = oracle.crs_to_ccs(H.n_rows, H.n_cols, H.irp, H.icol, H.val)
    arr = M.arrays()
    assert np.array_equal(arr["ptr"].cpu().numpy(), irp_t)
    assert np.array_equal(arr["idx"].cpu().numpy(), icol_t)
    assert np.array_equal(bits(arr["val"].cpu().numpy()), bits(val_t))


def _claims(L, H):
    """Builds the CCS of H with the kernel profile on; returns the handle and
    how many claim passes ran (2 = the row-position or grouped path handed
    over to the (k, row) slot path)."""
    L.spmv_profile_enable(True)
    L.spmv_profile_read(reset=True)
    try:
        M = L.spmv_transform(dev(H), L.SPMV_CRS, L.SPMV_COLWISE)
        prof = L.spmv_profile_read(reset=True)
    finally:
        L.spmv_profile_enable(False)
    return M, sum(prof.get(k, (0, 0.0))[0] for k in ("col_claim_grp", "col_claim_rk", "col_claim"))


def shuffled_rows(H, seed=3):
    """The same matrix with each row's entries in a seeded random order (no
    repeated (i, j)): the serial scatter still lists every column's rows in
    ascending order."""
    icol, val = H.icol.copy(), H.val.copy()
    rng = np.random.default_rng(seed)
    for i in range(H.n_rows):
        a, b = int(H.irp[i]), int(H.irp[i + 1])
        p = rng.permutation(b - a) + a
        icol[a:b], val[a:b] = H.icol[p], H.val[p]
    return synth.CRS(H.n_rows, H.n_cols, H.irp.copy(), icol, val)


def with_extra_columns(n, mean_len, seed, every):
    """Random rows plus, for each (column, period) in `every`, that column in
    every period-th row."""
    base = synth.random_crs(n, n, mean_len, seed=seed)
    rows = []
    for i in range(n):
        c = set(base.icol[base.irp[i]:base.irp[i + 1]].tolist())
        for col, period in every:
            if i % period == 0:
                c.add(col)
        rows.append(sorted(c))
    irp = np.zeros(n + 1, np.int64)
    irp[1:] = np.cumsum([len(r) for r in rows])
    icol = np.concatenate([np.array(r, np.int32) for r in rows])
    return synth.CRS(n, n, irp.astype(np.int32), icol, synth.normal(seed, 5, np.arange(icol.size)))


PHASE1_MODES = {"scatter": 1, "kslot": 2, "rk": 3, "grp": 4, "sym": 5}  # SPMV_PHASE1_*


@pytest.mark.parametrize("mode", list(PHASE1_MODES))
@pytest.mark.parametrize("name", ["stencil27_24", "powerlaw_60k", "random_duplicates", "dense_column", "wide",
                                  "tall", "all_empty", "one_by_one", "laplace37x23"])
def test_phase1_paths_bit_exact(mode, name):
    """Every Phase I path (count + scatter; (k, row) slots with ranks;
    (k, row) slots sorted by row per column; (row, value) records in 64-column
    group regions; the last two hand over to the first slot path on repeated
    entries, full groups or columns over 4096) gives the oracle's CCS bit for
    bit."""
    L = lib()
    H = case(name)
    with L.hint(L.SPMV_HINT_PHASE1, PHASE1_MODES[mode]):
        M = L.spmv_transform(dev(H), L.SPMV_CRS, L.SPMV_COLWISE)
    _ccs_matches_oracle(M, H)
    M.close()


@pytest.mark.parametrize("mode", ["rk", "grp"])
def test_phase1_register_sort_paths_on_shuffled_rows(mode):
    """Columns in arbitrary order within rows: the row-position and grouped
    paths order every column by row (register networks, overflow records and
    the long-column sort all run)."""
    L = lib()
    H = shuffled_rows(with_extra_columns(3000, 12, 81, [(5, 3), (9, 40)]))
    with L.hint(L.SPMV_HINT_PHASE1, PHASE1_MODES[mode]):
        M, claims = _claims(L, H)
    assert claims == 1
    _ccs_matches_oracle(M, H)
    M.close()


def upper_stencil():
    """The 27-point stencil's upper triangle (columns >= row): neighbouring
    columns, but not a symmetric pattern."""
    H = case("stencil27_24")
    rows = np.repeat(np.arange(H.n_rows), np.diff(H.irp))
    keep = H.icol >= rows
    irp = np.zeros(H.n_rows + 1, np.int64)
    irp[1:] = np.cumsum(np.bincount(rows[keep], minlength=H.n_rows))
    return synth.CRS(H.n_rows, H.n_cols, irp.astype(np.int32), H.icol[keep], H.val[keep])


@pytest.mark.parametrize("name,path", [("upper_stencil", "col_claim_rk"), ("powerlaw_60k", "col_claim_grp"),
                                       ("random12", "col_claim_grp")])
def test_phase1_path_follows_column_locality(name, path):
    """Neighbouring columns (a stencil's upper triangle) keep the per-column
    slots; scattered columns (random columns, the power law) take the grouped
    path."""
    L = lib()
    H = {"random12": lambda: synth.random_crs(3000, 3000, 12, seed=85), "upper_stencil": upper_stencil}.get(
        name, lambda: case(name))()
    assert 32 * H.n_cols <= 4 * H.nnz  # a slot path is taken
    L.spmv_profile_enable(True)
    L.spmv_profile_read(reset=True)
    try:
        M = L.spmv_transform(dev(H), L.SPMV_CRS, L.SPMV_COLWISE)
        prof = L.spmv_profile_read(reset=True)
    finally:
        L.spmv_profile_enable(False)
    assert path in prof and prof["col_locality"][0] == 1
    _ccs_matches_oracle(M, H)
    M.close()


@pytest.mark.parametrize("kind", ["duplicates", "column_over_4096", "many_beyond_slots"])
def test_phase1_register_sort_paths_hand_over(kind):
    """Matrices the grouped and row-position paths do not cover are rebuilt on
    the (k, row) slot path, and the result is still the serial CCS."""
    L = lib()
    if kind == "duplicates":
        H = synth.random_crs(3001, 2999, 12, seed=82, dup=True)
    elif kind == "column_over_4096":
        H = with_extra_columns(6000, 10, 83, [(7, 1)])
    else:
        H = with_extra_columns(4000, 10, 84, [(c, 4) for c in range(200)])
    assert 32 * H.n_cols <= 4 * H.nnz  # a slot path is taken
    M, claims = _claims(L, H)
    assert claims == 2
    _ccs_matches_oracle(M, H)
    M.close()


def test_phase1_slot_path_with_long_columns():
    """Columns longer than the slot capacity (32) next to short ones, on a
    matrix dense enough per column for the slot path."""
    L = lib()
    n = 3000
    H = with_extra_columns(n, 12, 71, [(5, 3), (9, 40)])  # column 5: 1000 entries, column 9: 75
    assert 32 * n <= 4 * H.nnz  # the slot path is taken
    M, claims = _claims(L, H)
    assert claims == 1  # the register-sort paths cover columns of up to 4096 entries
    _ccs_matches_oracle(M, H)
    M.close()


def _drop_entry(H, r, c):
    """H without entry (r, c) (its mirror (c, r) stays): no longer symmetric."""
    a, b = int(H.irp[r]), int(H.irp[r + 1])
    k = a + int(np.nonzero(H.icol[a:b] == c)[0][0])
    keep = np.ones(H.nnz, bool)
    keep[k] = False
    irp = H.irp.copy()
    irp[r + 1:] -= 1
    return synth.CRS(H.n_rows, H.n_cols, irp, H.icol[keep], H.val[keep])


def _reverse_row(H, r):
    icol, val = H.icol.copy(), H.val.copy()
    a, b = int(H.irp[r]), int(H.irp[r + 1])
    icol[a:b], val[a:b] = H.icol[a:b][::-1], H.val[a:b][::-1]
    return synth.CRS(H.n_rows, H.n_cols, H.irp.copy(), icol, val)


def _phase1_kernels(L, H):
    L.spmv_profile_enable(True)
    L.spmv_profile_read(reset=True)
    try:
        M = L.spmv_transform(dev(H), L.SPMV_CRS, L.SPMV_COLWISE)
        prof = L.spmv_profile_read(reset=True)
    finally:
        L.spmv_profile_enable(False)
    return M, prof


@pytest.mark.parametrize("name", ["laplace64", "laplace37x23", "stencil27_24", "stencil27_37", "laplace300x221",
                                  "one_by_one"])
def test_symmetric_patterns_take_the_mirror_path(name):
    """Structurally symmetric matrices (stencils, Laplacians) build the CCS in
    one mirror-gather pass: IRP_T = IRP, rows = ICOL, values of the mirror
    entries, bit for bit the serial Phase I."""
    L = lib()
    H = case(name)
    M, prof = _phase1_kernels(L, H)
    assert "ccs_sym" in prof and not any(k.startswith("col_claim") or k == "col_count" for k in prof), prof
    _ccs_matches_oracle(M, H)
    arr = M.arrays()
    assert np.array_equal(arr["ptr"].cpu().numpy(), H.irp) and np.array_equal(arr["idx"].cpu().numpy(), H.icol)
    # the longest column feeds ELL-Column
    E = L.spmv_transform_from(M, L.SPMV_ELL)
    assert E.describe()["width"] == int(np.diff(H.irp).max())
    E.close()
    M.close()


@pytest.mark.parametrize("kind", ["one_mirror_missing", "one_row_reversed"])
def test_symmetric_path_hands_over_when_a_condition_fails(kind):
    """A matrix that passes the sample but breaks the conditions in one row
    (one entry without its mirror, or one row in descending order) is rebuilt
    on a general path, and the CCS is still the serial one."""
    L = lib()
    H = synth.stencil_3d_27pt(24)
    r = 7001
    H = _drop_entry(H, r, int(H.icol[H.irp[r] + 3])) if kind == "one_mirror_missing" else _reverse_row(H, r)
    M, prof = _phase1_kernels(L, H)
    assert "ccs_sym" in prof and any(k.startswith("col_claim") or k == "col_count" for k in prof), prof
    _ccs_matches_oracle(M, H)
    M.close()


def test_symmetric_path_not_taken_for_scattered_columns():
    L = lib()
    H = synth.random_crs(3000, 3000, 12, seed=85)
    M, prof = _phase1_kernels(L, H)
    assert "ccs_sym" not in prof and "sym_sample" in prof
    _ccs_matches_oracle(M, H)
    M.close()


@pytest.mark.parametrize("name", ["stencil27_24", "laplace37x23"])
def test_symmetric_path_with_unaligned_arrays(name):
    """ICOL and VAL at addresses that are not 16-byte aligned (views one
    element into larger buffers): the mirror pass takes its scalar loads and
    stores, and the CCS is still the serial one bit for bit."""
    import torch
    L = lib()
    H = case(name)
    icol = torch.empty(H.nnz + 1, dtype=torch.int32, device="cuda")[1:]
    val = torch.empty(H.nnz + 1, dtype=torch.float64, device="cuda")[1:]
    icol.copy_(torch.from_numpy(H.icol))
    val.copy_(torch.from_numpy(H.val))
    assert icol.data_ptr() % 16 and val.data_ptr() % 16
    A = L.Crs(H.n_rows, H.n_cols, torch.from_numpy(H.irp).cuda(), icol, val)
    L.spmv_profile_enable(True)
    L.spmv_profile_read(reset=True)
    try:
        M = L.spmv_transform(A, L.SPMV_CRS, L.SPMV_COLWISE)
        prof = L.spmv_profile_read(reset=True)
    finally:
        L.spmv_profile_enable(False)
    assert "ccs_sym" in prof, prof
    _ccs_matches_oracle(M, H)
    M.close()

