"""The COO-Row SpMV entry point that allocates no device memory.

It serves callers that cannot allocate device memory while they multiply:
solvers that reserve all of their memory up front from a fixed arena and
must not grow it, and latency-critical loops where an allocation could block
or fail between iterations. Its temporaries live in one fixed device array
that every call shares, so these tests check each call against the CPU
oracle and against the allocating entry point, on calls in a row with
different matrices (a call that read a slot the previous call left behind
would give the wrong rows), and that a repeated call repeats its bits. This
file is collected last so that a failure here leaves the rest of the suite
run.
"""

import ctypes

import numpy as np
import pytest

import oracle
import spmv_synth as synth

TOL = 1e-12  # the suite's SpMV tolerance: |y - y_ref| <= TOL * sum_j |a_ij x_j|


def _lib():
    from paper_2407_00019_gb300 import _build
    _build.build()
    import paper_2407_00019_gb300 as L
    L.load_library()
    return L


def test_sizes_beyond_the_fixed_array_are_rejected_without_a_device():
    L = _lib()
    C = L.load_library()
    too_many = L.SPMV_NOALLOC_COO_MAX_NNZ + 1
    fake = ctypes.c_void_p(256)
    # rejected before any device access, so fake pointers are never touched
    assert C.spmv_apply_coo_row_noalloc(10, 10, too_many, fake, fake, fake, fake, fake, None) == 7
    assert C.spmv_apply_coo_row_noalloc(0, 10, 5, fake, fake, fake, fake, fake, None) == 1


def _within(y, H, xh, what):
    y_ref, s = oracle.spmv_ref(H.n_rows, H.irp, H.icol, H.val, xh)
    bad = ~(np.abs(y - y_ref) <= TOL * s) | ((s == 0) & (y != 0))
    assert not bad.any(), f"{what}: {int(bad.sum())} rows outside the tolerance"
    return s


@pytest.mark.gpu
def test_noalloc_matches_the_oracle_and_the_allocating_entry_point_on_calls_in_a_row():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L = _lib()
    # A: uneven rows that cross many 2048-entry tiles; B: short regular rows
    # with another tile-crossing pattern and another x
    cases = []
    for H, seed in ((synth.power_law(200000, kmax=20000, seed=11), 12), (synth.stencil_3d_27pt(30, seed=13), 14)):
        A = L.Crs.from_host(H)
        M = L.spmv_transform(A, L.SPMV_COO, L.SPMV_ROWWISE)
        xh = synth.vector_pm1(H.n_cols, seed=seed)
        x = torch.from_numpy(xh).cuda()
        y_apply = torch.full((H.n_rows,), float("nan"), dtype=torch.float64, device="cuda")
        L.spmv_apply(M, x, y_apply)
        torch.cuda.synchronize()
        cases.append((H, A, M, xh, x, y_apply.cpu().numpy()))
    # no library allocation may happen inside the no-alloc calls
    calls = []
    L.spmv_set_allocator(lambda n, ctx, st: calls.append(n) or 0, lambda p, n, ctx, st: None)
    got = []
    try:
        for i in (0, 1, 0):
            H, A, M, xh, x, _ = cases[i]
            y = torch.full((H.n_rows,), float("nan"), dtype=torch.float64, device="cuda")
            L.spmv_apply_coo_row_noalloc(H.n_rows, H.n_cols, M.arrays()["idx2"], A.icol, A.val, x, y)
            torch.cuda.synchronize()
            got.append(y.cpu().numpy())
    finally:
        L.spmv_set_allocator(None, None)
    assert calls == []
    for call, i in enumerate((0, 1, 0)):
        H, _, _, xh, _, y_apply = cases[i]
        s = _within(got[call], H, xh, f"call {call} vs the oracle")
        assert np.all(np.abs(got[call] - y_apply) <= TOL * s), f"call {call} vs spmv_apply"
    # the same matrix and x again, after a call on another matrix: same bits
    assert np.array_equal(got[0].view(np.uint64), got[2].view(np.uint64))
    for c in cases:
        c[2].close()


@pytest.mark.gpu
def test_noalloc_checks_its_tensors_before_the_call():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L = _lib()
    H = synth.laplacian_2d_5pt(16)
    A = L.Crs.from_host(H)
    M = L.spmv_transform(A, L.SPMV_COO, L.SPMV_ROWWISE)
    irow = M.arrays()["idx2"]
    x = torch.zeros(H.n_cols, dtype=torch.float64, device="cuda")
    y = torch.zeros(H.n_rows, dtype=torch.float64, device="cuda")
    with pytest.raises(TypeError):
        L.spmv_apply_coo_row_noalloc(H.n_rows, H.n_cols, irow.long(), A.icol, A.val, x, y)
    with pytest.raises(ValueError):
        L.spmv_apply_coo_row_noalloc(H.n_rows, H.n_cols, irow[:-1], A.icol, A.val, x, y)
    with pytest.raises(ValueError):
        L.spmv_apply_coo_row_noalloc(H.n_rows, H.n_cols, irow, A.icol, A.val, x[:-1], y)
    with pytest.raises(ValueError):
        L.spmv_apply_coo_row_noalloc(H.n_rows, H.n_cols, irow, A.icol, A.val, x.cpu(), y)
    with pytest.raises(ValueError):
        xs = torch.zeros(2 * H.n_cols, dtype=torch.float64, device="cuda")[::2]
        L.spmv_apply_coo_row_noalloc(H.n_rows, H.n_cols, irow, A.icol, A.val, xs, y)
    M.close()
