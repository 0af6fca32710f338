"""Transformations carry every value bit for bit, special values included.

Sec. 2.1's transformations only move VAL: ELL-Row, Phase I (every path),
Phase II, ELL-Column, the fused ELL-Row build and the batch ELL build must
keep -0.0, subnormals, infinities and NaNs with their payloads exactly. A
kernel that added 0.0 to a value or selected through arithmetic would turn
-0.0 into +0.0 or quiet a signalling NaN, and the comparisons of bits below
would fail. Products on matrices with such values: rows of finite values stay
inside the SpMV tolerance, rows holding an infinity or a NaN give a
non-finite result.
"""

import numpy as np
import pytest

import oracle
import spmv_synth as synth
from gpu_helpers import TOL, bits, dev, ell_from_gpu, lib, xvec

pytestmark = pytest.mark.gpu

# -0.0, the smallest subnormal, the largest negative subnormal, +inf, -inf,
# quiet NaNs with payloads (positive and negative), a signalling NaN
SPECIAL_BITS = np.array([0x8000000000000000, 0x0000000000000001, 0x800FFFFFFFFFFFFF, 0x7FF0000000000000,
                         0xFFF0000000000000, 0x7FF8000000000123, 0xFFF800000000BEEF, 0x7FF0000000000ABC],
                        dtype=np.uint64)


def with_special_values(H, seed, every=5):
    """H with a seeded share (one in `every`) of its values replaced by the
    special values above (cycled), the rest unchanged."""
    val = H.val.copy()
    u = synth.uniform01(seed, 31, np.arange(H.nnz, dtype=np.uint64))
    pos = np.nonzero(u < 1.0 / every)[0]
    vb = val.view(np.uint64)
    vb[pos] = SPECIAL_BITS[np.arange(pos.size) % SPECIAL_BITS.size]
    return synth.CRS(H.n_rows, H.n_cols, H.irp.copy(), H.icol.copy(), val)


CASES = {
    "stencil27_24": lambda: with_special_values(synth.stencil_3d_27pt(24), 1),
    "powerlaw_60k": lambda: with_special_values(synth.power_law(60000, kmax=20000), 2),
    "random_empty_rows": lambda: with_special_values(synth.random_crs(5003, 4001, 6, seed=21, empty_frac=0.3), 3),
    "laplace37x23": lambda: with_special_values(synth.laplacian_2d_5pt(37, 23), 4),
    "long_row": lambda: with_special_values(synth.random_crs(4000, 6000, 3, seed=25, long_rows=3, long_len=5000), 5),
}
_cache = {}


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


def test_the_cases_hold_every_special_value():
    H = case("stencil27_24")
    present = set(H.val.view(np.uint64).tolist())
    assert all(int(b) in present for b in SPECIAL_BITS)


def assert_products_with_specials(y, H, xh, what):
    """Finite rows within the tolerance of the compensated oracle sum;
    rows holding an infinity or a NaN give a non-finite result."""
    y_ref, s = oracle.spmv_ref(H.n_rows, H.irp, H.icol, H.val, xh)
    finite_entry = np.isfinite(H.val)
    row_of = np.repeat(np.arange(H.n_rows), np.diff(H.irp))
    bad_row = np.zeros(H.n_rows, bool)
    bad_row[row_of[~finite_entry]] = True
    ok = ~bad_row
    err = np.abs(y[ok] - y_ref[ok])
    assert np.all((err <= TOL * s[ok]) & ((s[ok] > 0) | (y[ok] == 0))), what
    assert not np.any(np.isfinite(y[bad_row])), what


def _ell_row_matches(M, H):
    W, ld, ev, ei = ell_from_gpu(M, H.n_rows)
    rv, ri, rW = oracle.crs_to_ell_row(H.n_rows, H.irp, H.icol, H.val)
    assert W == rW
    if W:
        assert np.array_equal(bits(ev[:, :H.n_rows]), bits(rv.reshape(W, H.n_rows)))
        assert np.array_equal(ei[:, :H.n_rows], ri.reshape(W, H.n_rows))


@pytest.mark.parametrize("name", list(CASES))
def test_ell_row_keeps_special_bits(name):
    L = lib()
    H = case(name)
    M = L.spmv_transform(dev(H), L.SPMV_ELL, L.SPMV_ROWWISE)
    _ell_row_matches(M, H)
    M.close()


@pytest.mark.parametrize("name", list(CASES))
def test_fused_build_keeps_special_bits(name):
    import torch
    L = lib()
    H = case(name)
    xh = xvec(H.n_cols, seed=6)
    x = torch.from_numpy(xh).cuda()
    y = torch.full((H.n_rows,), 7.0, dtype=torch.float64, device="cuda")
    M = L.spmv_transform_apply(dev(H), x, y)
    torch.cuda.synchronize()
    _ell_row_matches(M, H)
    assert_products_with_specials(y.cpu().numpy(), H, xh, f"{name}/fused")
    M.close()


@pytest.mark.parametrize("mode", [1, 2, 3, 4, 5])  # SPMV_PHASE1_COUNT, _KSLOT, _ROWPOS, _GROUPED, _SYMMETRIC
@pytest.mark.parametrize("name", list(CASES))
def test_column_wise_transforms_keep_special_bits(mode, name):
    L = lib()
    H = case(name)
    irp_t, icol_t, val_t, _ = oracle.crs_to_ccs(H.n_rows, H.n_cols, H.irp, H.icol, H.val)
    with L.hint(L.SPMV_HINT_PHASE1, mode):
        ccs = L.spmv_transform(dev(H), L.SPMV_CRS, L.SPMV_COLWISE)
    arr = ccs.arrays()
    assert np.array_equal(arr["ptr"].cpu().numpy(), irp_t)
    assert np.array_equal(arr["idx"].cpu().numpy(), icol_t)
    assert np.array_equal(bits(arr["val"].cpu().numpy()), bits(val_t))
    coo = L.spmv_transform_from(ccs, L.SPMV_COO)  # Phase II
    ca = coo.arrays()
    assert np.array_equal(ca["idx2"].cpu().numpy(), oracle.ccs_to_coo_col(H.n_cols, irp_t))
    assert np.array_equal(bits(ca["val"].cpu().numpy()), bits(val_t))
    ell = L.spmv_transform_from(ccs, L.SPMV_ELL)
    W, ld, ev, ei = ell_from_gpu(ell, H.n_cols)
    rv, rr, rW = oracle.ccs_to_ell_col(H.n_cols, irp_t, icol_t, val_t)
    assert W == rW
    if W:
        assert np.array_equal(bits(ev[:, :H.n_cols]), bits(rv.reshape(W, H.n_cols)))
        assert np.array_equal(ei[:, :H.n_cols], rr.reshape(W, H.n_cols))
    for M in (ell, coo, ccs):
        M.close()


@pytest.mark.parametrize("name", ["stencil27_24", "random_empty_rows"])
def test_products_on_special_values(name):
    """Every format's product: finite rows inside the tolerance, rows with a
    non-finite entry non-finite (special values on one entry in 40, so that
    most rows stay finite)."""
    import torch
    L = lib()
    base = {"stencil27_24": lambda: synth.stencil_3d_27pt(24),
            "random_empty_rows": lambda: synth.random_crs(5003, 4001, 6, seed=21, empty_frac=0.3)}[name]()
    H = with_special_values(base, 8, every=40)
    A = dev(H)
    xh = xvec(H.n_cols, seed=7)
    x = torch.from_numpy(xh).cuda()
    mats = {"crs": L.spmv_transform(A, L.SPMV_CRS, L.SPMV_ROWWISE),
            "coo_row": L.spmv_transform(A, L.SPMV_COO, L.SPMV_ROWWISE),
            "ell_row": L.spmv_transform(A, L.SPMV_ELL, L.SPMV_ROWWISE),
            "ccs": L.spmv_transform(A, L.SPMV_CRS, L.SPMV_COLWISE)}
    mats["coo_col"] = L.spmv_transform_from(mats["ccs"], L.SPMV_COO)
    mats["ell_col"] = L.spmv_transform_from(mats["ccs"], L.SPMV_ELL)
    for fmt, M in mats.items():
        y = torch.full((H.n_rows,), 7.0, dtype=torch.float64, device="cuda")
        L.spmv_apply(M, x, y)
        torch.cuda.synchronize()
        assert_products_with_specials(y.cpu().numpy(), H, xh, f"{name}/{fmt}")
    for M in mats.values():
        M.close()


@pytest.mark.parametrize("fused", [False, True])
def test_batch_ell_build_keeps_special_bits(fused):
    import torch
    L = lib()
    hs = [with_special_values(synth.batch_matrix(i, seed=5, n_lo=100, n_hi=3000), 40 + i, every=20)
          for i in range(12)]
    hs.append(synth.CRS(1, 1, np.array([0, 1], np.int32), np.array([0], np.int32),
                        np.array([SPECIAL_BITS[7]], np.uint64).view(np.float64)))
    devs = L.Crs.batch_from_host(hs)
    nc, nr = sum(H.n_cols for H in hs), sum(H.n_rows for H in hs)
    xh = synth.vector_pm1(nc, seed=9)
    x = torch.from_numpy(xh).cuda()
    y = torch.full((nr,), 7.0, dtype=torch.float64, device="cuda")
    B = L.spmv_batch_create(devs, x=x if fused else None, y=y if fused else None, dstar=float("inf"))
    plans = B.plans()
    torch.cuda.synchronize()
    for H, P in zip(hs, plans):
        assert P["format"] == L.SPMV_ELL
        ev, ei, W = oracle.crs_to_ell_row(H.n_rows, H.irp, H.icol, H.val)
        assert W == P["width"]
        W_, ld = P["width"], P["ld"]
        gv = L.device_view(P["ell_val"], W_ * ld, torch.float64).cpu().numpy().reshape(W_, ld)[:, :H.n_rows]
        gi = L.device_view(P["ell_idx"], W_ * ld, torch.int32).cpu().numpy().reshape(W_, ld)[:, :H.n_rows]
        assert np.array_equal(bits(gv), bits(ev.reshape(W, H.n_rows)))
        assert np.array_equal(gi, ei.reshape(W, H.n_rows))
    if not fused:
        B.apply(x, y)
        torch.cuda.synchronize()
    yh = y.cpu().numpy()
    for i, (H, P) in enumerate(zip(hs, plans)):
        xs = xh[P["x_offset"]:P["x_offset"] + H.n_cols]
        assert_products_with_specials(yh[P["y_offset"]:P["y_offset"] + H.n_rows], H, xs, f"batch {i}")
    B.close()


def test_ell_column_padding_with_non_finite_x():
    """ELL-Column pads short columns with zeros (Fig. 3). The product skips
    the adds of zero slots when x_j is finite (they leave y unchanged) and
    keeps them when x_j is infinite or NaN, so its result equals the padded
    product of the oracle: the same rows NaN, the same rows +-Inf with the
    same sign, the finite rows within the tolerance."""
    import torch
    L = lib()
    H = synth.random_crs(3000, 2500, 6, seed=27, empty_frac=0.2)
    irp_t, icol_t, val_t, _ = oracle.crs_to_ccs(H.n_rows, H.n_cols, H.irp, H.icol, H.val)
    ev, er, W = oracle.ccs_to_ell_col(H.n_cols, irp_t, icol_t, val_t)
    ccs = L.spmv_transform(dev(H), L.SPMV_CRS, L.SPMV_COLWISE)
    ell = L.spmv_transform_from(ccs, L.SPMV_ELL)
    for seed in (1, 2):
        xh = xvec(H.n_cols, seed=40 + seed)
        pick = np.nonzero(synth.uniform01(seed, 41, np.arange(H.n_cols, dtype=np.uint64)) < 0.01)[0]
        xh[pick[0::3]] = np.inf
        xh[pick[1::3]] = -np.inf
        xh[pick[2::3]] = np.nan
        y_ref = oracle.spmv_ell_col(H.n_rows, H.n_cols, W, ev, er, xh)
        assert np.isnan(y_ref).any() and np.isinf(y_ref).any()
        y = torch.full((H.n_rows,), 7.0, dtype=torch.float64, device="cuda")
        L.spmv_apply(ell, torch.from_numpy(xh).cuda(), y)
        torch.cuda.synchronize()
        yh = y.cpu().numpy()
        assert np.array_equal(np.isnan(yh), np.isnan(y_ref))
        inf = np.isinf(y_ref)
        assert np.array_equal(np.isinf(yh), inf) and np.array_equal(np.sign(yh[inf]), np.sign(y_ref[inf]))
        fin = np.isfinite(y_ref)
        _, s = oracle.spmv_ref(H.n_rows, H.irp, H.icol, H.val, np.where(np.isfinite(xh), xh, 0.0))
        assert np.all(np.abs(yh[fin] - y_ref[fin]) <= TOL * s[fin])
    ell.close()
    ccs.close()
