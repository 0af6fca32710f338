"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and compare with the CPU oracle on the same seeded inputs."""

import numpy as np

import oracle

# SpMV acceptance: |y_gpu - y_ref| <= TOL * sum_j |a_ij x_j| per row, y_ref
# the compensated oracle sum; rows with sum |a x| = 0 must give +-0.
TOL = 1e-12


def lib():
    import paper_2407_00019_gb300 as L
    L.load_library()
    return L


def dev(H):
    return lib().Crs.from_host(H)


def xvec(n, seed=0):
    import spmv_synth as synth
    return synth.vector_pm1(n, seed=seed)


def assert_spmv_close(y_gpu, H, xh, tol=TOL, what=""):
    y_ref, s = oracle.spmv_ref(H.n_rows, H.irp, H.icol, H.val, xh)
    err = np.abs(y_gpu - y_ref)
    bad = ~(err <= tol * s)
    zero_rows = s == 0
    bad |= zero_rows & (y_gpu != 0)
    if bad.any():
        i = int(np.nonzero(bad)[0][0])
        raise AssertionError(f"{what}: row {i}: gpu {y_gpu[i]!r} ref {y_ref[i]!r} s {s[i]!r} "
                             f"({int(bad.sum())} bad rows)")


def run_apply(M, x, n_rows):
    import torch
    L = lib()
    y = torch.full((n_rows,), float("nan"), dtype=torch.float64, device="cuda")
    L.spmv_apply(M, x, y)
    torch.cuda.synchronize()
    return y.cpu().numpy()


def bits(a):
    return np.ascontiguousarray(a).view(np.uint64)


def ell_from_gpu(M, n_lines):
    arr = M.arrays()
    d = M.describe()
    W, ld = d["width"], d["ld"]
    ev = arr["val"].cpu().numpy().reshape(W, ld) if W else np.zeros((0, ld))
    ei = arr["idx"].cpu().numpy().reshape(W, ld) if W else np.zeros((0, ld), np.int32)
    return W, ld, ev, ei
