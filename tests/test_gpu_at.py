"""GPU tests of the AT rule (Sec. 2.2), the memory cap, and failure paths:
bounded waits, injected allocation failure and malformed input. None of
them faults or hangs the device: failures are made on the host or by a
bounded wait that runs out."""

import math

import numpy as np
import pytest

import oracle
import spmv_synth as synth
from gpu_helpers import assert_spmv_close, dev, lib, run_apply, xvec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib()


def test_lookback_wait_times_out_and_device_stays_usable():
    L = lib()
    assert L.spmv_debug_scan_timeout(1 << 16, 2000) == 5  # SPMV_ERR_TIMEOUT
    H = synth.laplacian_2d_5pt(16)
    import torch
    xh = xvec(H.n_cols)
    M = L.spmv_transform(dev(H), L.SPMV_CRS, L.SPMV_COLWISE)
    assert_spmv_close(run_apply(M, torch.from_numpy(xh).cuda(), H.n_rows), H, xh, what="after timeout")
    M.close()


def test_memory_cap_rejects_before_allocating():
    L = lib()
    H = synth.laplacian_2d_5pt(64)
    A = dev(H)
    need = L.spmv_ell_bytes(H.n_rows, 5)
    with pytest.raises(L.SpmvError) as e:
        L.spmv_transform(A, L.SPMV_ELL, L.SPMV_ROWWISE, need - 1)
    assert e.value.status == 4
    L.spmv_transform(A, L.SPMV_ELL, L.SPMV_ROWWISE, need).close()
    with pytest.raises(L.SpmvError) as e:
        L.spmv_transform(A, L.SPMV_COO, L.SPMV_ROWWISE, 4 * H.nnz - 1)
    assert e.value.status == 4
    with pytest.raises(L.SpmvError) as e:
        L.spmv_transform(A, L.SPMV_ELL, L.SPMV_COLWISE, 1000)
    assert e.value.status == 4


def test_injected_allocation_failure_is_oom():
    L = lib()
    H = synth.laplacian_2d_5pt(32)
    A = dev(H)
    calls = []
    L.spmv_set_allocator(lambda n, ctx, s: calls.append(n) or 0, lambda p, n, ctx, s: None)
    try:
        for fmt, lay in ((L.SPMV_COO, L.SPMV_ROWWISE), (L.SPMV_ELL, L.SPMV_ROWWISE), (L.SPMV_CRS, L.SPMV_COLWISE)):
            with pytest.raises(L.SpmvError) as e:
                L.spmv_transform(A, fmt, lay)
            assert e.value.status == 3
    finally:
        L.spmv_set_allocator(None, None)
    assert calls
    L.spmv_transform(A, L.SPMV_COO, L.SPMV_ROWWISE).close()


def test_allocator_hook_serves_every_allocation():
    import torch
    L = lib()
    H = synth.random_crs(3000, 3000, 9, seed=61)
    A = dev(H)
    live = {}

    def alloc(n, ctx, s):
        p = torch.cuda.caching_allocator_alloc(n, stream=s)
        live[p] = n
        return p

    def free(p, n, ctx, s):
        live.pop(p)
        torch.cuda.caching_allocator_delete(p)

    L.spmv_set_allocator(alloc, free)
    try:
        xh = xvec(H.n_cols)
        x = torch.from_numpy(xh).cuda()
        for fmt, lay in ((L.SPMV_COO, L.SPMV_ROWWISE), (L.SPMV_ELL, L.SPMV_ROWWISE), (L.SPMV_ELL, L.SPMV_COLWISE)):
            M = L.spmv_transform(A, fmt, lay)
            assert_spmv_close(run_apply(M, x, H.n_rows), H, xh, what=f"hooked {fmt}/{lay}")
            M.close()
        torch.cuda.synchronize()
        assert live == {}
    finally:
        L.spmv_set_allocator(None, None)


def test_malformed_input_is_reported_not_faulted():
    import torch
    L = lib()
    H = synth.random_crs(500, 400, 5, seed=62)
    bad = H.icol.copy()
    bad[bad.size // 2] = 400  # one column out of range
    A = L.Crs(H.n_rows, H.n_cols, torch.from_numpy(H.irp).cuda(), torch.from_numpy(bad).cuda(),
              torch.from_numpy(H.val).cuda())
    with pytest.raises(L.SpmvError) as e:
        L.spmv_validate(A)
    assert e.value.status == 2
    for fmt, lay in ((L.SPMV_CRS, L.SPMV_ROWWISE), (L.SPMV_ELL, L.SPMV_ROWWISE), (L.SPMV_CRS, L.SPMV_COLWISE),
                     (L.SPMV_ELL, L.SPMV_COLWISE)):
        with pytest.raises(L.SpmvError) as e:
            L.spmv_transform(A, fmt, lay)
        assert e.value.status == 2
    irp = H.irp.copy()
    irp[10], irp[11] = irp[11], irp[10] - 1  # not monotone
    B = L.Crs(H.n_rows, H.n_cols, torch.from_numpy(irp).cuda(), torch.from_numpy(H.icol).cuda(),
              torch.from_numpy(H.val).cuda())
    with pytest.raises(L.SpmvError) as e:
        L.spmv_analyze(B)
    assert e.value.status == 2
    for fmt, lay in ((L.SPMV_COO, L.SPMV_ROWWISE), (L.SPMV_ELL, L.SPMV_ROWWISE), (L.SPMV_CRS, L.SPMV_COLWISE)):
        with pytest.raises(L.SpmvError) as e:
            L.spmv_transform(B, fmt, lay)
        assert e.value.status == 2
    # the device still works
    L.spmv_validate(dev(H))


def test_online_rule_picks_ell_below_dstar_and_respects_cap():
    import torch
    L = lib()
    H = synth.stencil_3d_27pt(20)
    A = dev(H)
    xh = xvec(H.n_cols)
    x = torch.from_numpy(xh).cuda()
    st = L.spmv_analyze(A)
    cases = [(math.inf, 0, L.SPMV_ELL), (st["dmat"], 0, L.SPMV_CRS), (st["dmat"] * 1.01, 0, L.SPMV_ELL),
             (math.inf, st["ell_bytes"] - 1, L.SPMV_CRS), (0.0, 0, L.SPMV_CRS)]
    for dstar, cap, want in cases:
        M, s2 = L.spmv_autotune(A, dstar=dstar, mem_cap_bytes=cap)
        assert M.describe()["format"] == want, (dstar, cap)
        assert s2["dmat"] == st["dmat"]
        (f, lay), _ = L.spmv_autotune_choose(A, dstar=dstar, mem_cap_bytes=cap)
        assert f == want and lay == L.SPMV_ROWWISE
        assert_spmv_close(run_apply(M, x, H.n_rows), H, xh, what=f"autotune {dstar}")
        M.close()
    M, _ = L.spmv_autotune(A, dstar=0.0, flags=L.SPMV_AT_TRY_COO, timing_reps=3, warmup_reps=1)
    assert M.describe()["format"] in (L.SPMV_CRS, L.SPMV_COO)
    assert_spmv_close(run_apply(M, x, H.n_rows), H, xh, what="try coo")
    M.close()


def test_powerlaw_under_cap_rejects_ell():
    """The irregular workload shape: ELL padding explodes, the 40 GB cap
    forces CRS (or COO) whatever D* says."""
    L = lib()
    H = synth.power_law(400000, seed=3)
    A = dev(H)
    st = L.spmv_analyze(A)
    assert st["ell_bytes"] > 40 * 10 ** 9
    M, _ = L.spmv_autotune(A, dstar=math.inf, mem_cap_bytes=40 * 10 ** 9)
    assert M.describe()["format"] == L.SPMV_CRS
    M.close()
    with pytest.raises(L.SpmvError) as e:
        L.spmv_transform(A, L.SPMV_ELL, L.SPMV_ROWWISE, 40 * 10 ** 9)
    assert e.value.status == 4


def test_measure_and_calibrate_follow_eqs_1_to_3():
    L = lib()
    mats = [dev(synth.laplacian_2d_5pt(128)), dev(synth.stencil_3d_27pt(24)),
            dev(synth.power_law(50000, kmax=2000, seed=8))]
    for A in mats:
        t = L.spmv_measure(A, timing_reps=5, warmup_reps=1)
        assert t["t_crs_ms"] > 0 and t["t_ell_ms"] > 0 and t["t_trans_ms"] > 0
        assert math.isclose(t["sp"], t["t_crs_ms"] / t["t_ell_ms"], rel_tol=1e-12)
        assert math.isclose(t["tt"], t["t_trans_ms"] / t["t_crs_ms"], rel_tol=1e-12)
        assert math.isclose(t["r_ell"], oracle.r_ell(t["t_crs_ms"], t["t_ell_ms"], t["t_trans_ms"]), rel_tol=1e-12)
    for rule in (0, 1):
        dstar, d, r = L.spmv_calibrate(mats, c=1.0, dstar_rule=rule, timing_reps=5, warmup_reps=1)
        assert dstar == oracle.dstar_from_points(d, r, 1.0, rule)
        for A, dm in zip(mats, d):
            assert dm == L.spmv_analyze(A)["dmat"]


def test_offline_calibration_on_table1_shaped_set(tmp_path):
    # the off-line phase end to end at 2 % scale: D_mat of each point is the
    # oracle's sigma/mu, D* follows the rule, the result reloads
    import torch

    from paper_2407_00019_gb300 import calibrate as C
    mats = C.table1_shaped_set(scale=0.02)
    for rule in (0, 1):
        res = C.run_offline(mats, rule=rule, timing_reps=3, warmup_reps=1)
        d = [p[0] for p in res["points"]]
        r = [p[1] for p in res["points"]]
        assert len(d) == len(C.TABLE1_SHAPES)
        assert all(x > 0 and math.isfinite(x) for x in r)
        for H, dm in zip(mats, d):
            assert math.isclose(dm, oracle.analyze(H.n_rows, H.irp)["dmat"], rel_tol=1e-12)
        assert res["dstar"] == oracle.dstar_from_points(d, r, 1.0, rule)
        path = str(tmp_path / f"d{rule}.json")
        C.save_dstar(path, res)
        assert C.load_dstar(path, device=torch.cuda.get_device_name()) == res["dstar"]


def test_profile_counts_launches():
    import torch
    L = lib()
    H = synth.laplacian_2d_5pt(64)
    A = dev(H)
    M = L.spmv_transform(A, L.SPMV_ELL, L.SPMV_ROWWISE)
    x = torch.zeros(H.n_cols, dtype=torch.float64, device="cuda")
    y = torch.empty(H.n_rows, dtype=torch.float64, device="cuda")
    L.spmv_profile_read(reset=True)
    n0 = L.spmv_launch_count()
    L.spmv_profile_enable(True)
    for _ in range(7):
        L.spmv_apply(M, x, y)
    L.spmv_profile_enable(False)
    prof = L.spmv_profile_read(reset=True)
    assert L.spmv_launch_count() - n0 == 7
    assert prof["spmv_ell_row"][0] == 7 and prof["spmv_ell_row"][1] > 0
    M.close()


def test_reserve_grows_the_pool_and_respects_hooks():
    import torch
    L = lib()
    L.spmv_reserve(64 << 20)
    L.spmv_reserve(0)
    calls = []
    L.spmv_set_allocator(lambda n, ctx, s: calls.append(n) or 0, lambda p, n, ctx, s: None)
    try:
        L.spmv_reserve(64 << 20)  # the caller's allocator owns the memory: nothing to do
    finally:
        L.spmv_set_allocator(None, None)
    assert calls == []
    with pytest.raises(L.SpmvError) as e:
        L.spmv_reserve(1 << 60)
    assert e.value.status == 3  # SPMV_ERR_OOM
    torch.cuda.synchronize()


def test_column_check_finds_every_position_at_every_alignment():
    """The index check reads the body of ICOL in 16-byte loads and the entries
    before the first 16-byte boundary and after the last whole vector one by
    one: an out-of-range column must be found wherever it sits, with ICOL
    starting 0, 4, 8 or 12 bytes past a 16-byte boundary."""
    import torch
    L = lib()
    H = synth.random_crs(300, 200, 7, seed=63)
    nnz = H.icol.size
    irp = torch.from_numpy(H.irp).cuda()
    val = torch.from_numpy(H.val).cuda()
    for off in range(4):
        base = torch.zeros(nnz + 4, dtype=torch.int32, device="cuda")
        icol = base[off:off + nnz]
        icol.copy_(torch.from_numpy(H.icol))
        A = L.Crs(H.n_rows, H.n_cols, irp, icol, val)
        L.spmv_validate(A)  # every column in range
        for pos in (0, 1, 2, 3, 4, nnz // 2, nnz - 5, nnz - 4, nnz - 3, nnz - 2, nnz - 1):
            keep = int(icol[pos])
            icol[pos] = H.n_cols if pos % 2 else -1
            with pytest.raises(L.SpmvError) as e:
                L.spmv_validate(A)
            assert e.value.status == 2, (off, pos)
            icol[pos] = keep
        L.spmv_validate(A)
