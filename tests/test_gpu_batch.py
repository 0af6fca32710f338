"""GPU parity of batches of independent matrices: statistics (Eq. (4)) per
matrix, the on-line rule per matrix, bit-exact ELL-Row arrays (Sec. 2.1) and
SpMV within the tolerance for every matrix, against the oracle."""

import math

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


def _special():
    long_rows = synth.random_crs(700, 650, 6.0, seed=41, long_rows=3, long_len=600)
    dense_rows = synth.random_crs(300, 300, 200.0, seed=42)  # tiles larger than the staging capacity
    empty = synth.CRS(5, 7, np.zeros(6, np.int32), np.zeros(0, np.int32), np.zeros(0, np.float64))
    one = synth.CRS(1, 1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([-0.0]))
    gaps = synth.random_crs(1000, 1200, 3.0, seed=43, empty_frac=0.4)
    return [long_rows, dense_rows, empty, one, gaps]


@pytest.fixture(scope="module")
def host_set():
    mats = synth.batch_set(60, seed=5, n_lo=50, n_hi=3000)
    sp = _special()
    return mats[:30] + sp + mats[30:]


def _xy(mats, seed=11):
    import torch
    nc = sum(A.n_cols for A in mats)
    nr = sum(A.n_rows for A in mats)
    xh = synth.vector_pm1(nc, seed=seed)
    x = torch.from_numpy(xh).cuda()
    y = torch.full((nr,), float("nan"), dtype=torch.float64, device="cuda")
    return xh, x, y


def _check_products(mats, plans, xh, yh, what):
    for i, (H, P) in enumerate(zip(mats, plans)):
        xs = xh[P["x_offset"]:P["x_offset"] + H.n_cols]
        ys = yh[P["y_offset"]:P["y_offset"] + H.n_rows]
        assert_spmv_close(ys, H, xs, what=f"{what} matrix {i}")


def _ell_arrays(P, n_rows):
    import torch
    L = lib()
    W, ld = P["width"], P["ld"]
    ev = L.device_view(P["ell_val"], W * ld, torch.float64).cpu().numpy().reshape(W, ld)[:, :n_rows]
    ei = L.device_view(P["ell_idx"], W * ld, torch.int32).cpu().numpy().reshape(W, ld)[:, :n_rows]
    return ev, ei


@pytest.mark.parametrize("dstar", [0.0, math.inf, 0.2])
def test_batch_matches_oracle(host_set, dstar):
    import torch
    L = lib()
    dev = L.Crs.batch_from_host(host_set)
    B = L.spmv_batch_create(dev, dstar=dstar)
    plans = B.plans()
    info = B.info()
    assert info["n_matrices"] == len(host_set)
    assert info["total_rows"] == sum(A.n_rows for A in host_set)
    assert info["total_nnz"] == sum(A.nnz for A in host_set)
    n_ell = 0
    for H, P in zip(host_set, plans):
        st = oracle.analyze(H.n_rows, H.irp)
        assert math.isclose(P["mu"], st["mu"], rel_tol=1e-15)
        assert math.isclose(P["dmat"], st["dmat"], rel_tol=1e-12, abs_tol=1e-15)
        assert P["max_row_len"] == st["W"]
        want_ell = P["dmat"] < dstar
        assert P["format"] == (L.SPMV_ELL if want_ell else L.SPMV_CRS)
        n_ell += want_ell
        if want_ell and P["width"] > 0:
            ev, ei, W = oracle.crs_to_ell_row(H.n_rows, H.irp, H.icol, H.val)
            assert W == P["width"]
            gv, gi = _ell_arrays(P, H.n_rows)
            torch.cuda.synchronize()
            assert np.array_equal(bits(gv), bits(ev.reshape(W, H.n_rows)))
            assert np.array_equal(gi, ei.reshape(W, H.n_rows))
    assert info["n_ell"] == n_ell
    xh, x, y = _xy(host_set)
    B.apply(x, y)
    torch.cuda.synchronize()
    _check_products(host_set, plans, xh, y.cpu().numpy(), f"D*={dstar}")
    B.close()


def test_fused_build_equals_apply_and_rerun_is_deterministic(host_set):
    import torch
    L = lib()
    dev = L.Crs.batch_from_host(host_set)
    xh, x, y0 = _xy(host_set, seed=12)
    B = L.spmv_batch_create(dev, x=x, y=y0, dstar=0.2)
    y1 = torch.full_like(y0, float("nan"))
    y2 = torch.full_like(y0, float("nan"))
    B.apply(x, y1)
    B.apply(x, y2)
    torch.cuda.synchronize()
    a, b, c = (bits(t.cpu().numpy()) for t in (y0, y1, y2))
    assert np.array_equal(a, b) and np.array_equal(b, c)
    _check_products(host_set, B.plans(), xh, y1.cpu().numpy(), "fused")


@pytest.mark.parametrize("tpr", ["1", "8", "32"])
def test_every_threads_per_row_schedule(host_set, tpr):
    import torch
    L = lib()
    dev = L.Crs.batch_from_host(host_set)
    with L.hint(L.SPMV_HINT_BATCH_TPR, int(tpr)):
        B = L.spmv_batch_create(dev, dstar=0.0)
    assert all(P["threads_per_row"] == int(tpr) for P in B.plans())
    xh, x, y = _xy(host_set, seed=13)
    B.apply(x, y)
    torch.cuda.synchronize()
    _check_products(host_set, B.plans(), xh, y.cpu().numpy(), f"tpr={tpr}")


@pytest.mark.parametrize("dstar", [0.0, 0.2])
def test_multi_vector_products_equal_single_products(host_set, dstar, monkeypatch):
    import torch
    L = lib()
    dev = L.Crs.batch_from_host(host_set)
    B = L.spmv_batch_create(dev, dstar=dstar)
    info = B.info()
    nvec, nc, nr = 5, info["total_cols"], info["total_rows"]
    ldx, ldy = nc + 3, nr + 1  # padded strides, y at odd offsets
    xs = [synth.vector_pm1(nc, seed=40 + j) for j in range(nvec)]
    X = torch.zeros(nvec * ldx, dtype=torch.float64, device="cuda")
    for j in range(nvec):
        X[j * ldx:j * ldx + nc] = torch.from_numpy(xs[j])
    Y = torch.full((nvec * ldy,), float("nan"), dtype=torch.float64, device="cuda")
    B.apply_multi(X, Y, nvec, ldx, ldy)
    for j in range(nvec):
        y1 = torch.empty(nr, dtype=torch.float64, device="cuda")
        B.apply(X[j * ldx:j * ldx + nc], y1)
        torch.cuda.synchronize()
        assert np.array_equal(bits(Y[j * ldy:j * ldy + nr].cpu().numpy()), bits(y1.cpu().numpy()))
        if j in (0, nvec - 1):
            _check_products(host_set, B.plans(), xs[j], y1.cpu().numpy(), f"multi {j}")
    assert torch.isnan(Y[nr:ldy]).all()  # padding between vectors untouched
    with pytest.raises(L.SpmvError):
        B.apply_multi(X, Y, 2, nc - 1, ldy)


def test_memory_cap_takes_matrices_in_order(host_set):
    L = lib()
    dev = L.Crs.batch_from_host(host_set)
    need = [((H.n_rows + 31) // 32 * 32) * int(np.diff(H.irp).max(initial=0)) * 12 for H in host_set]
    cap = sum(need[:10]) + 1
    B = L.spmv_batch_create(dev, dstar=math.inf, mem_cap_bytes=cap)
    used, fmt = 0, []
    for b in need:
        ok = used + b <= cap
        used += b if ok else 0
        fmt.append(L.SPMV_ELL if ok else L.SPMV_CRS)
    assert [P["format"] for P in B.plans()] == fmt
    assert B.info()["ell_bytes"] == used


def test_batch_equals_per_matrix_handles(host_set):
    import torch
    L = lib()
    dev = L.Crs.batch_from_host(host_set)
    B = L.spmv_batch_create(dev, dstar=0.0)
    xh, x, y = _xy(host_set, seed=14)
    B.apply(x, y)
    torch.cuda.synchronize()
    for A, P in list(zip(dev, B.plans()))[::7]:
        M = L.spmv_transform(A, L.SPMV_CRS, L.SPMV_ROWWISE)
        yi = torch.empty(A.n_rows, dtype=torch.float64, device="cuda")
        L.spmv_apply(M, x[P["x_offset"]:P["x_offset"] + A.n_cols], yi)
        torch.cuda.synchronize()
        ys = y[P["y_offset"]:P["y_offset"] + A.n_rows]
        _, s = oracle.spmv_ref(A.n_rows, A.irp.cpu().numpy(), A.icol.cpu().numpy(), A.val.cpu().numpy(),
                               xh[P["x_offset"]:P["x_offset"] + A.n_cols])
        assert np.all(np.abs(yi.cpu().numpy() - ys.cpu().numpy()) <= 2e-12 * s)


def test_apply_replays_in_a_cuda_graph(host_set):
    import torch
    L = lib()
    dev = L.Crs.batch_from_host(host_set)
    B = L.spmv_batch_create(dev, dstar=0.2)
    xh, x, y = _xy(host_set, seed=15)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        B.apply(x, y, stream=s)  # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        B.apply(x, y)
    x2h = synth.vector_pm1(x.numel(), seed=16)
    x.copy_(torch.from_numpy(x2h))
    y.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    _check_products(host_set, B.plans(), x2h, y.cpu().numpy(), "graph replay")


def test_malformed_members_are_rejected():
    import torch
    L = lib()
    good = synth.batch_set(3, seed=5, n_lo=50, n_hi=200)
    bad_col = synth.batch_matrix(1, seed=5, n_lo=50, n_hi=200)
    bad_col.icol[len(bad_col.icol) // 2] = bad_col.n_cols
    with pytest.raises(L.SpmvError) as e:
        L.spmv_batch_create(L.Crs.batch_from_host(good + [bad_col]), dstar=0.0)
    assert e.value.status == 2  # SPMV_ERR_INVALID_MATRIX
    bad_ptr = synth.batch_matrix(2, seed=5, n_lo=50, n_hi=200)
    bad_ptr.irp[5], bad_ptr.irp[6] = bad_ptr.irp[6], bad_ptr.irp[5] - 1
    with pytest.raises(L.SpmvError) as e:
        L.spmv_batch_create(L.Crs.batch_from_host([bad_ptr] + good), dstar=0.0)
    assert e.value.status == 2  # SPMV_ERR_INVALID_MATRIX
    dev = L.Crs.batch_from_host(good)
    x = torch.zeros(sum(A.n_cols for A in good), dtype=torch.float64, device="cuda")
    with pytest.raises(L.SpmvError) as e:
        L.spmv_batch_create(dev, x=x, dstar=0.0)
    assert e.value.status == 1  # SPMV_ERR_INVALID_ARG
    torch.cuda.synchronize()


def test_allocation_failure_is_reported_and_nothing_leaks(host_set):
    import torch
    L = lib()
    dev = L.Crs.batch_from_host(host_set[:8])
    live = {}

    def alloc(n, ctx, s):
        if n >= 4096:
            return 0  # the tile list and the ELL pool cannot be had
        p = torch.cuda.caching_allocator_alloc(n, stream=s)
        live[p] = n
        return p

    def free(p, n, ctx, s):
        live.pop(p)
        torch.cuda.caching_allocator_delete(p)

    L.spmv_set_allocator(alloc, free)
    try:
        with pytest.raises(L.SpmvError) as e:
            L.spmv_batch_create(dev, dstar=math.inf)
        assert e.value.status == 3  # SPMV_ERR_OOM
    finally:
        L.spmv_set_allocator(None, None)
    torch.cuda.synchronize()
    assert live == {}
    L.spmv_batch_create(dev, dstar=math.inf).close()


# ---- batches planned on the device (one CUDA graph for build and products) ----
def _cap_for(host_set, dstar):
    """A cap that fits every candidate of the host-planned batch."""
    L = lib()
    B = L.spmv_batch_create(L.Crs.batch_from_host(host_set), dstar=dstar)
    eb = B.info()["ell_bytes"]
    B.close()
    return max(eb, 1 << 20)


@pytest.mark.parametrize("dstar", [0.0, math.inf, 0.2])
def test_device_planned_batch_equals_the_host_planned_one(host_set, dstar):
    """prepare + build gives the host path's plan (format, lanes, widths,
    statistics) and its products bit for bit, and ELL arrays equal to the
    oracle's."""
    import torch
    L = lib()
    dev = L.Crs.batch_from_host(host_set)
    kw = dict(dstar=dstar, mem_cap_bytes=_cap_for(host_set, dstar) if dstar > 0 else 0)
    H = L.spmv_batch_create(dev, **kw)
    D = L.spmv_batch_prepare(dev, **kw)
    xh, x, y0 = _xy(host_set, seed=21)
    y1 = torch.full_like(y0, float("nan"))
    D.build(x, y1)  # the first product fused with the build
    D.status()
    ph, pd = H.plans(), D.plans()
    for i, (a, b) in enumerate(zip(ph, pd)):
        for k in ("format", "threads_per_row", "rows_per_tile", "width", "ld", "max_row_len", "x_offset",
                  "y_offset"):
            assert a[k] == b[k], (i, k, a[k], b[k])
        for k in ("mu", "sigma", "dmat"):
            assert a[k] == b[k] or math.isclose(a[k], b[k], rel_tol=2 ** -52), (i, k, a[k], b[k])
        if b["format"] == L.SPMV_ELL and b["width"] > 0:
            Hm = host_set[i]
            ev, ei, W = oracle.crs_to_ell_row(Hm.n_rows, Hm.irp, Hm.icol, Hm.val)
            gv, gi = _ell_arrays(b, Hm.n_rows)
            assert np.array_equal(bits(gv), bits(ev.reshape(W, Hm.n_rows)))
            assert np.array_equal(gi, ei.reshape(W, Hm.n_rows))
    hi, di = H.info(), D.info()
    assert hi["n_tiles"] == di["n_tiles"] and hi["n_ell"] == di["n_ell"] and hi["ell_bytes"] == di["ell_bytes"]
    H.apply(x, y0)
    y2 = torch.full_like(y0, float("nan"))
    D.apply(x, y2)
    torch.cuda.synchronize()
    assert np.array_equal(bits(y0.cpu().numpy()), bits(y2.cpu().numpy()))
    _check_products(host_set, pd, xh, y1.cpu().numpy(), f"device plan, fused, D*={dstar}")
    H.close()
    D.close()


def test_device_planned_build_and_products_in_one_cuda_graph(host_set):
    """The whole build (analysis, rule, tiles, ELL build, first product) and
    two more products captured in one CUDA graph and replayed: every product
    equals the oracle within the tolerance, and replays repeat their bits."""
    import torch
    L = lib()
    dev = L.Crs.batch_from_host(host_set)
    D = L.spmv_batch_prepare(dev, dstar=0.2, mem_cap_bytes=_cap_for(host_set, 0.2))
    xh, x, y0 = _xy(host_set, seed=22)
    y1 = torch.full_like(y0, float("nan"))
    xx = torch.cat([x, x])
    yy = torch.full((2 * y0.numel(),), float("nan"), dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s):
        D.build(x, y0)
        D.apply(x, y1)
        D.apply_multi(xx, yy, 2)
    launches0 = L.spmv_launch_count()
    for rep in range(3):
        y0.fill_(float("nan"))
        y1.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        a, b = y0.cpu().numpy(), y1.cpu().numpy()
        if rep == 0:
            first = bits(b).copy()
        assert np.array_equal(bits(b), first)
    assert L.spmv_launch_count() == launches0  # replays launch nothing through the host library
    D.status()
    plans = D.plans()
    assert sum(P["format"] == L.SPMV_ELL for P in plans) > 0
    _check_products(host_set, plans, xh, a, "graph build + first product")
    _check_products(host_set, plans, xh, b, "graph product")
    yyh = yy.cpu().numpy()
    assert np.array_equal(bits(yyh[:y0.numel()]), bits(b)) and np.array_equal(bits(yyh[y0.numel():]), bits(b))
    D.close()


def test_device_planned_batch_reports_a_malformed_member(host_set):
    L = lib()
    bad = synth.CRS(4, 4, np.array([0, 2, 1, 3, 4], np.int32), np.array([0, 1, 2, 3], np.int32), np.ones(4))
    D = L.spmv_batch_prepare(L.Crs.batch_from_host(host_set[:5] + [bad]), dstar=0.0)
    D.build()
    with pytest.raises(L.SpmvError) as e:
        D.status()
    assert e.value.status == 2  # SPMV_ERR_INVALID_MATRIX
    D.close()


def test_schedule_table_sets_lanes_per_row(host_set):
    L = lib()
    old = L.spmv_batch_schedule_get()
    try:
        L.spmv_batch_schedule_set([8] * L.SPMV_BATCH_SCHED_CLASSES)
        B = L.spmv_batch_create(L.Crs.batch_from_host(host_set), dstar=0.0)
        assert all(P["threads_per_row"] == 8 for P in B.plans())
        xh, x, y = _xy(host_set, seed=23)
        B.apply(x, y)
        _check_products(host_set, B.plans(), xh, y.cpu().numpy(), "table of 8 lanes")
        assert B.time(x, y, warm=1, reps=3) > 0
        B.close()
        with pytest.raises(L.SpmvError):
            L.spmv_batch_schedule_set([3])
    finally:
        L.spmv_batch_schedule_set(old)
