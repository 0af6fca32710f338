"""The COO-Row SpMV entry point that allocates no device memory.

It serves callers that cannot allocate device memory while they multiply
(solvers that reserve all memory up front, latency-critical loops). Its
temporaries live in one fixed device array shared by every call. This file
is collected last so that a failure here leaves the rest of the suite run.
"""

import ctypes

import numpy as np
import pytest

import spmv_synth as synth


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


@pytest.mark.gpu
def test_noalloc_matches_the_allocating_entry_point_on_two_calls():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L = _lib()
    H = synth.power_law(200000, kmax=20000, seed=11)  # rows crossing many tiles
    A = L.Crs.from_host(H)
    M = L.spmv_transform(A, L.SPMV_COO, L.SPMV_ROWWISE)
    irow = M.arrays()["idx2"]
    x = torch.from_numpy(synth.vector_pm1(H.n_cols, seed=12)).cuda()
    y_ref = torch.full((H.n_rows,), float("nan"), dtype=torch.float64, device="cuda")
    L.spmv_apply(M, x, y_ref)
    torch.cuda.synchronize()
    ref = y_ref.cpu().numpy()
    import oracle
    _, s = oracle.spmv_ref(H.n_rows, H.irp, H.icol, H.val, x.cpu().numpy())  # sum_j |a_ij x_j|
    # no library allocation may happen inside the no-alloc call
    calls = []
    L.spmv_set_allocator(lambda n, ctx, st: calls.append(n) or 0, lambda p, n, ctx, st: None)
    try:
        for rep in range(2):
            y = torch.full((H.n_rows,), float("nan"), dtype=torch.float64, device="cuda")
            L.spmv_apply_coo_row_noalloc(H.n_rows, H.n_cols, irow, A.icol, A.val, x, y)
            torch.cuda.synchronize()
            got = y.cpu().numpy()
            assert np.all(np.abs(got - ref) <= 1e-12 * s), f"call {rep}"  # the suite's SpMV tolerance
    finally:
        L.spmv_set_allocator(None, None)
    assert calls == []
    M.close()
