"""One matrix over several GPUs: nnz-balanced row blocks, one rank per GPU.

SpMV (Sec. 3) needs no exchange beyond x: rank k owns rows [r_k, r_{k+1})
of A (its row block, columns global) and the same slice of x and y; a product
all-gathers x and multiplies the row block locally, y stays where it is.
Phase I (Sec. 2.1) splits the same way: each rank counts the columns of its
own rows; the column pointers of the whole CCS are the running sum over the
columns of the counts summed over ranks, and rank k's entries of column j
start after those of ranks 0..k-1 in that column (an exclusive scan over the
ranks, per column). Since the serial Phase I lists a column's rows in
ascending order, and rank k's rows all precede rank k+1's, every rank places
its own entries at their final CCS positions with no further exchange; the
local order inside a column is the local serial order, so the assembled CCS
is the serial one bit for bit.

Host-side logic only: the local steps are callables (on GPUs the library's
transforms and products, see `library_engine`), and the exchanges go through
torch.distributed (NCCL on GPUs; the tests use gloo ranks on the CPU with the
oracle as the local engine). No TMA multicast and no peer loads.
"""

from __future__ import annotations

import numpy as np


def nnz_balanced_rows(irp, parts: int) -> np.ndarray:
    """Row block boundaries b[0] = 0 < ... <= b[parts] = n: block k holds rows
    [b[k], b[k+1]), cut where the running entry count passes k * nnz / parts
    (every block gets about nnz / parts entries; rows are never split)."""
    irp = np.asarray(irp, dtype=np.int64)
    n = irp.size - 1
    if parts <= 0:
        raise ValueError("parts must be positive")
    nnz = int(irp[-1])
    targets = (np.arange(1, parts, dtype=np.float64) * nnz / parts)
    cuts = np.searchsorted(irp, targets, side="left") if nnz > 0 else (np.arange(1, parts) * n // parts)
    b = np.concatenate(([0], np.clip(cuts, 0, n), [n])).astype(np.int64)
    return np.maximum.accumulate(b)


def row_block(irp, icol, val, r0: int, r1: int):
    """Rows [r0, r1) of a CRS matrix as a local CRS (row pointers from 0,
    columns kept global): (irp_local, icol_local, val_local)."""
    irp = np.asarray(irp, dtype=np.int64)
    a, b = int(irp[r0]), int(irp[r1])
    return ((irp[r0:r1 + 1] - a).astype(np.int32), np.asarray(icol)[a:b].copy(), np.asarray(val)[a:b].copy())


def allgather_blocks(local, bounds, group=None):
    """The full vector from every rank's block (block k has bounds[k+1] -
    bounds[k] elements): one all-gather of blocks padded to the longest, then
    the padding is dropped. `local` is a 1-D torch tensor."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    sizes = [int(bounds[k + 1] - bounds[k]) for k in range(world)]
    m = max(sizes) if sizes else 0
    buf = torch.zeros(m, dtype=local.dtype, device=local.device)
    buf[:local.numel()] = local
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    return torch.cat([p[:s] for p, s in zip(parts, sizes)])


def sharded_spmv(local_apply, x_local, bounds, group=None):
    """y_local = (row block of A) x: all-gather x, then local_apply(x_full)."""
    return local_apply(allgather_blocks(x_local, bounds, group))


def ccs_offsets(nc_local, group=None):
    """Column pointers of the whole CCS and this rank's first position in
    every column, from the ranks' per-column counts (int64 torch tensors of
    n_cols): (cp [n_cols + 1], start [n_cols]). One all-gather of the counts;
    the scans are plain integer sums, the same on every rank."""
    import torch
    import torch.distributed as dist
    world, rank = dist.get_world_size(group), dist.get_rank(group)
    allc = [torch.empty_like(nc_local) for _ in range(world)]
    dist.all_gather(allc, nc_local, group=group)
    stack = torch.stack(allc)                      # [world, n_cols]
    total = stack.sum(dim=0)
    cp = torch.zeros(total.numel() + 1, dtype=torch.int64, device=nc_local.device)
    cp[1:] = torch.cumsum(total, dim=0)
    before = stack[:rank].sum(dim=0) if rank > 0 else torch.zeros_like(nc_local)
    return cp, cp[:-1] + before


def sharded_phase1(local_ccs, irp_local, icol_local, val_local, r0: int, n_cols: int, group=None):
    """Phase I of the whole matrix from this rank's row block. local_ccs(irp,
    icol, val, n_cols) must return the local CCS (irp_t, rows, vals) of the
    block, rows local. Returns (cp, pos, rows, vals): the global column
    pointers, and this rank's entries with their global CCS positions (pos),
    global row indices and values, in local CCS order."""
    import torch
    irp_t, rows, vals = local_ccs(irp_local, icol_local, val_local, n_cols)
    irp_t = torch.as_tensor(np.asarray(irp_t, dtype=np.int64))
    nc = irp_t[1:] - irp_t[:-1]
    cp, start = ccs_offsets(nc, group)
    col = torch.repeat_interleave(torch.arange(n_cols, dtype=torch.int64), nc)
    pos = start[col] + (torch.arange(col.numel(), dtype=torch.int64) - irp_t[:-1][col])
    rows_g = torch.as_tensor(np.asarray(rows, dtype=np.int64)) + int(r0)
    return cp, pos, rows_g, torch.as_tensor(np.asarray(vals))


def library_engine(L, device):
    """The local steps on this rank's GPU through the library: a product
    callable for sharded_spmv and a CCS callable for sharded_phase1 (both take
    and return torch tensors on `device`)."""
    import torch

    def make_apply(irp_local, icol_local, val_local, n_cols):
        A = L.Crs(len(irp_local) - 1, n_cols, torch.as_tensor(irp_local, device=device),
                  torch.as_tensor(icol_local, device=device), torch.as_tensor(val_local, device=device))
        M = L.spmv_transform(A, L.SPMV_CRS, L.SPMV_ROWWISE)

        def apply(x_full):
            y = torch.empty(A.n_rows, dtype=torch.float64, device=device)
            L.spmv_apply(M, x_full, y)
            return y
        apply.keep = (A, M)
        return apply

    def local_ccs(irp_local, icol_local, val_local, n_cols):
        A = L.Crs(len(irp_local) - 1, n_cols, torch.as_tensor(irp_local, device=device),
                  torch.as_tensor(icol_local, device=device), torch.as_tensor(val_local, device=device))
        C = L.spmv_transform(A, L.SPMV_CRS, L.SPMV_COLWISE)
        arr = C.arrays()
        out = (arr["ptr"].cpu().numpy(), arr["idx"].cpu().numpy(), arr["val"].cpu().numpy())
        C.close()
        return out

    return make_apply, local_ccs
