"""GPU tests of the serving runtime: requests over a matrix pool give the same
y in a concurrent mix as alone (and the oracle's, within the tolerance); the
format cache builds a transformation only after the amortisation threshold,
stays within its budget by evicting idle entries, and requests wait for the
producer of their x."""

import math
import threading

import numpy as np
import pytest

import spmv_synth as synth
from gpu_helpers import assert_spmv_close, bits, lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib()


def _pool():
    return [synth.laplacian_2d_5pt(60), synth.stencil_3d_27pt(12, seed=4), synth.power_law(5000, kmax=400, seed=5),
            synth.random_crs(3000, 2500, 7.0, seed=6, empty_frac=0.2), synth.laplacian_2d_5pt(31, 17),
            synth.batch_matrix(3, seed=9, n_lo=200, n_hi=4000)]


def _requests(pool, n_req, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for r in range(n_req):
        i = int(rng.integers(len(pool)))
        k = int(rng.integers(1, 6))
        xs = np.concatenate([synth.vector_pm1(pool[i].n_cols, seed=1000 * r + j) for j in range(k)])
        out.append((i, k, xs))
    return out


def _run(server, dev, ids, reqs, concurrent):
    import torch
    ys, handles = [], []
    for i, k, xs in reqs:
        x = torch.from_numpy(xs).cuda()
        y = torch.full((k * dev[i].n_rows,), float("nan"), dtype=torch.float64, device="cuda")
        h = server.submit(ids[i], k, x, y)
        handles.append((h, x, y))
        if not concurrent:
            server.wait(h, 60000)
    fmts = []
    for h, x, y in handles:
        if concurrent:
            fmts.append(server.wait(h, 60000)[1])
        ys.append(y.cpu().numpy())
    return ys, fmts


def _check_oracle(pool, reqs, ys, what):
    for (i, k, xs), y in zip(reqs, ys):
        H = pool[i]
        for j in range(k):
            assert_spmv_close(y[j * H.n_rows:(j + 1) * H.n_rows], H, xs[j * H.n_cols:(j + 1) * H.n_cols],
                              what=f"{what} matrix {i}")


def test_alone_equals_mix():
    L = lib()
    pool = _pool()
    dev = [L.Crs.from_host(H) for H in pool]
    reqs = _requests(pool, 40)
    fixed = L.Server.FIXED_THRESHOLD
    alone = L.Server(dstar=math.inf, n_streams=1, amortize_products=1, flags=fixed)
    ids = [alone.add_matrix(A) for A in dev]
    y_alone, _ = _run(alone, dev, ids, reqs, concurrent=False)
    alone.close()
    mix = L.Server(dstar=math.inf, n_streams=6, amortize_products=1, flags=fixed)
    ids = [mix.add_matrix(A) for A in dev]
    y_mix, fmts = _run(mix, dev, ids, reqs, concurrent=True)
    st = mix.stats()
    mix.close()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["products"] == sum(k for _, k, _ in reqs)
    _check_oracle(pool, reqs, y_mix, "mix")
    # with the threshold at 1 every request of an ELL-target matrix runs in
    # the same format alone and in the mix, so y agrees bit for bit
    for a, b in zip(y_alone, y_mix):
        assert np.array_equal(bits(a), bits(b))
    assert L.SPMV_ELL in fmts


def test_amortisation_threshold_then_cache_hits():
    import torch
    L = lib()
    H = synth.laplacian_2d_5pt(64)
    A = L.Crs.from_host(H)
    S = L.Server(dstar=math.inf, n_streams=2, amortize_products=5, flags=L.Server.FIXED_THRESHOLD)
    mid = S.add_matrix(A)
    fmts = []
    for r in range(5):
        xs = synth.vector_pm1(H.n_cols, seed=r)
        x = torch.from_numpy(xs).cuda()
        y = torch.empty(H.n_rows, dtype=torch.float64, device="cuda")
        fmts.append(S.wait(S.submit(mid, 2, torch.cat([x, x]), torch.cat([y, y])), 60000)[1])
    # products seen: 2, 4 (CRS), 6 -> transformation built, then cached
    assert fmts == [L.SPMV_CRS, L.SPMV_CRS, L.SPMV_ELL, L.SPMV_ELL, L.SPMV_ELL]
    st = S.stats()
    assert st["transforms"] == 1 and st["cache_hits"] == 2 and st["cache_misses"] == 3
    S.close()


def _breakeven(H):
    # Eqs. (1)-(3) with bytes for times: k >= TT / (1 - 1 / SP)
    n, nnz = H.n_rows, H.nnz
    W = int(np.diff(H.irp).max())
    ell = 12.0 * ((n + 31) // 32 * 32) * W
    crs = 12.0 * nnz + 4.0 * (n + 1) + 16.0 * n
    sp = crs / (ell + 16.0 * n)
    tt = (12.0 * nnz + 4.0 * (n + 1) + ell) / crs
    return math.ceil(tt / (1.0 - 1.0 / sp)) if sp > 1 else None


def test_breakeven_model_decides_when_to_transform():
    import torch
    L = lib()
    H = synth.laplacian_2d_5pt(64)
    P = synth.power_law(5000, kmax=400, seed=5)
    k_star = _breakeven(H)
    assert k_star is not None and k_star > 2 and _breakeven(P) is None
    S = L.Server(dstar=math.inf, n_streams=2, amortize_products=2)
    ids = [S.add_matrix(L.Crs.from_host(M)) for M in (H, P)]
    seen, fmts = 0, []
    for r in range(6):
        k = (k_star + 2) // 3
        x = torch.from_numpy(np.tile(synth.vector_pm1(H.n_cols, seed=r), k)).cuda()
        y = torch.empty(k * H.n_rows, dtype=torch.float64, device="cuda")
        fmts.append(S.wait(S.submit(ids[0], k, x, y), 60000)[1])
        seen += k
        assert fmts[-1] == (L.SPMV_ELL if seen >= k_star else L.SPMV_CRS)
        xp = torch.from_numpy(synth.vector_pm1(P.n_cols, seed=r)).cuda()
        yp = torch.empty(P.n_rows, dtype=torch.float64, device="cuda")
        assert S.wait(S.submit(ids[1], 1, xp, yp), 60000)[1] == L.SPMV_CRS  # SP < 1: never
        assert_spmv_close(yp.cpu().numpy(), P, xp.cpu().numpy(), what="power law")
    assert L.SPMV_ELL in fmts and S.stats()["transforms"] == 1
    S.close()


def test_budget_evicts_idle_entries():
    import torch
    L = lib()
    pool = [synth.laplacian_2d_5pt(80), synth.laplacian_2d_5pt(81)]
    dev = [L.Crs.from_host(H) for H in pool]
    one = max(L.spmv_analyze(A)["ell_bytes"] for A in dev)
    S = L.Server(mem_budget_bytes=one + one // 2, dstar=math.inf, n_streams=1, amortize_products=1,
                 flags=L.Server.FIXED_THRESHOLD)
    ids = [S.add_matrix(A) for A in dev]
    reqs = [(r % 2, 1, synth.vector_pm1(pool[r % 2].n_cols, seed=r)) for r in range(6)]
    ys, fmts = _run(S, dev, ids, reqs, concurrent=False)
    st = S.stats()
    assert st["transforms"] == 6 and st["evictions"] == 5
    assert st["peak_cache_bytes"] <= one + one // 2
    _check_oracle(pool, reqs, ys, "evicting")
    S.close()


def test_request_waits_for_its_producer_stream():
    import torch
    L = lib()
    H = synth.stencil_3d_27pt(20, seed=2)
    A = L.Crs.from_host(H)
    S = L.Server(dstar=0.0, n_streams=2)
    mid = S.add_matrix(A)
    side = torch.cuda.Stream()
    xs = synth.vector_pm1(H.n_cols, seed=3)
    x = torch.zeros(H.n_cols, dtype=torch.float64, device="cuda")
    y = torch.empty(H.n_rows, dtype=torch.float64, device="cuda")
    big = torch.empty(1 << 26, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(side):
        for _ in range(20):
            big.mul_(1.0)  # keep the producer stream busy before x is written
        x.copy_(torch.from_numpy(xs).cuda(non_blocking=False))
    h = S.submit(mid, 1, x, y, after=side)
    S.wait(h, 60000)
    assert_spmv_close(y.cpu().numpy(), H, xs, what="after stream")
    S.close()


def test_two_client_threads():
    import torch
    L = lib()
    pool = _pool()[:3]
    dev = [L.Crs.from_host(H) for H in pool]
    S = L.Server(dstar=math.inf, n_streams=4, amortize_products=3, flags=L.Server.FIXED_THRESHOLD)
    ids = [S.add_matrix(A) for A in dev]
    reqs = _requests(pool, 30, seed=4)
    out = [None] * len(reqs)

    def client(part):
        torch.cuda.set_device(0)
        for n, (i, k, xs) in enumerate(reqs):
            if n % 2 != part:
                continue
            x = torch.from_numpy(xs).cuda()
            y = torch.empty(k * dev[i].n_rows, dtype=torch.float64, device="cuda")
            S.wait(S.submit(ids[i], k, x, y), 60000)
            out[n] = y.cpu().numpy()

    th = [threading.Thread(target=client, args=(p,)) for p in (0, 1)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    _check_oracle(pool, reqs, out, "threads")
    S.drain(60000)
    assert S.stats()["completed"] == len(reqs)
    S.close()


def test_bad_arguments():
    import torch
    L = lib()
    S = L.Server()
    A = L.Crs.from_host(synth.laplacian_2d_5pt(8))
    mid = S.add_matrix(A)
    x = torch.zeros(64, dtype=torch.float64, device="cuda")
    with pytest.raises(L.SpmvError):
        S.submit(mid + 5, 1, x, x)
    with pytest.raises(L.SpmvError):
        S.submit(mid, -1, x, x)
    with pytest.raises(L.SpmvError):
        S.wait(123456, 10)
    h = S.submit(mid, 0, None, None)
    S.wait(h, 60000)
    S.close()


def test_malformed_matrix_is_refused_at_registration():
    L = lib()
    H = synth.laplacian_2d_5pt(16)
    H.icol[7] = H.n_cols  # column out of range
    S = L.Server()
    with pytest.raises(L.SpmvError) as e:
        S.add_matrix(L.Crs.from_host(H))
    assert e.value.status == 2  # SPMV_ERR_INVALID_MATRIX
    S.close()


def test_failed_transformation_falls_back_to_crs():
    import torch
    L = lib()
    H = synth.laplacian_2d_5pt(64)
    S = L.Server(dstar=math.inf, n_streams=1, amortize_products=1, flags=L.Server.FIXED_THRESHOLD)
    mid = S.add_matrix(L.Crs.from_host(H))

    def alloc(n, ctx, s):
        return 0 if n >= 65536 else torch.cuda.caching_allocator_alloc(n, stream=s)

    def free(p, n, ctx, s):
        torch.cuda.caching_allocator_delete(p)

    xs = synth.vector_pm1(H.n_cols, seed=1)
    x = torch.from_numpy(xs).cuda()
    y = torch.full((H.n_rows,), float("nan"), dtype=torch.float64, device="cuda")
    L.spmv_set_allocator(alloc, free)
    try:
        _, fmt = S.wait(S.submit(mid, 1, x, y), 60000)  # the ELL-Row build cannot allocate
    finally:
        L.spmv_set_allocator(None, None)
    assert fmt == L.SPMV_CRS and S.stats()["transforms"] == 0
    assert_spmv_close(y.cpu().numpy(), H, xs, what="fallback")
    _, fmt = S.wait(S.submit(mid, 1, x, y), 60000)  # memory is back: built now
    assert fmt == L.SPMV_ELL
    assert_spmv_close(y.cpu().numpy(), H, xs, what="after fallback")
    S.close()


def test_plain_form_serves_every_request_on_crs():
    """The per-matrix form the serving benchmark compares against: one slot,
    one spmv_apply per product on CRS, no format cache; results within the
    tolerance and in CRS whatever D* says."""
    L = lib()
    pool = _pool()
    dev = [L.Crs.from_host(H) for H in pool]
    reqs = _requests(pool, 24, seed=3)
    S = L.Server(dstar=math.inf, n_streams=6, amortize_products=1, flags=L.Server.PLAIN)
    ids = [S.add_matrix(A) for A in dev]
    launches0 = L.spmv_launch_count()
    ys, fmts = _run(S, dev, ids, reqs, concurrent=True)
    st = S.stats()
    S.close()
    assert all(f == L.SPMV_CRS for f in fmts)
    assert st["transforms"] == 0 and st["cache_hits"] == 0 and st["completed"] == len(reqs)
    assert st["products"] == sum(k for _, k, _ in reqs)
    assert L.spmv_launch_count() - launches0 >= st["products"]  # at least one launch per product
    _check_oracle(pool, reqs, ys, "plain")


def test_uneven_rows_run_per_product_in_the_mix():
    """Matrices with uneven rows (D_mat > 0.5 or a row of 2048 entries) that
    stay in CRS run each product as spmv_apply's entry-split product: results
    alone and in the mix agree within the tolerance, and both with the
    oracle."""
    L = lib()
    pool = [synth.power_law(20000, kmax=5000, seed=15), synth.laplacian_2d_5pt(40)]
    assert L.spmv_analyze(L.Crs.from_host(pool[0]))["dmat"] > 0.5
    dev = [L.Crs.from_host(H) for H in pool]
    reqs = _requests(pool, 16, seed=5)
    outs = []
    for streams, conc in ((1, False), (4, True)):
        S = L.Server(dstar=0.0, n_streams=streams)
        ids = [S.add_matrix(A) for A in dev]
        launches0 = L.spmv_launch_count()
        ys, fmts = _run(S, dev, ids, reqs, concurrent=conc)
        S.close()
        outs.append(ys)
        _check_oracle(pool, reqs, ys, f"uneven, {streams} slots")
    # the power-law requests took one launch (or more) per product
    assert L.spmv_launch_count() - launches0 >= sum(k for i, k, _ in reqs if i == 0)
