"""One matrix over several ranks (nnz-balanced row blocks, an all-gather of x
per product, Phase I with a cross-rank scan of the column counts), tested as
gloo ranks on the CPU with the oracle as each rank's local engine: the
gathered results equal the oracle's on the whole matrix bit for bit (the row
sums and the CCS order do not depend on the split)."""

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import spmv_synth as synth
from paper_2407_00019_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _matrices():
    return {"stencil": synth.stencil_3d_27pt(10, seed=3),
            "powerlaw": synth.power_law(3000, kmax=600, seed=4),
            "empty_rows": synth.random_crs(1500, 1500, 5, seed=6, empty_frac=0.4),
            "duplicates": synth.random_crs(900, 900, 6, seed=7, dup=True)}


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    res = {}
    for name, H in _matrices().items():
        b = shard.nnz_balanced_rows(H.irp, world)
        r0, r1 = int(b[rank]), int(b[rank + 1])
        irp_l, icol_l, val_l = shard.row_block(H.irp, H.icol, H.val, r0, r1)
        xh = synth.vector_pm1(H.n_cols, seed=11)
        x_local = torch.from_numpy(xh[r0:r1].copy())  # x split like the rows (square matrices)

        def local_apply(x_full):
            return torch.from_numpy(oracle.spmv_crs(r1 - r0, irp_l, icol_l, val_l, x_full.numpy()))
        y_local = shard.sharded_spmv(local_apply, x_local, b)

        def local_ccs(irp, icol, val, n_cols):
            irp_t, rows, vals, _ = oracle.crs_to_ccs(len(irp) - 1, n_cols, irp, icol, val)
            return irp_t, rows, vals
        cp, pos, rows, vals = shard.sharded_phase1(local_ccs, irp_l, icol_l, val_l, r0, H.n_cols)
        res[name] = (b.tolist(), y_local.numpy().tobytes(), cp.numpy(), pos.numpy(), rows.numpy(),
                     vals.numpy().view(np.uint64))
    out[rank] = res
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_spmv_and_phase1_equal_the_whole_matrix(world):
    import oracle
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for name, H in _matrices().items():
        parts = [out[r][name] for r in range(world)]
        b = parts[0][0]
        assert all(p[0] == b for p in parts) and b[0] == 0 and b[-1] == H.n_rows
        # SpMV: the concatenated local y equal the serial product bit for bit
        y = np.concatenate([np.frombuffer(p[1], dtype=np.float64) for p in parts])
        xh = synth.vector_pm1(H.n_cols, seed=11)
        y_ref = oracle.spmv_crs(H.n_rows, H.irp, H.icol, H.val, xh)
        assert np.array_equal(y.view(np.uint64), y_ref.view(np.uint64)), name
        # Phase I: every rank's entries at their global positions give the serial CCS
        irp_t, icol_t, val_t, _ = oracle.crs_to_ccs(H.n_rows, H.n_cols, H.irp, H.icol, H.val)
        rows = np.full(H.nnz, -1, np.int64)
        vals = np.zeros(H.nnz, np.uint64)
        for p in parts:
            assert np.array_equal(p[2], irp_t), name
            rows[p[3]] = p[4]
            vals[p[3]] = p[5]
        assert np.array_equal(rows, icol_t) and np.array_equal(vals, val_t.view(np.uint64)), name


def test_row_blocks_balance_the_entries():
    H = synth.power_law(20000, kmax=2000, seed=9)
    for parts in (1, 2, 4, 8):
        b = shard.nnz_balanced_rows(H.irp, parts)
        assert b[0] == 0 and b[-1] == H.n_rows and np.all(np.diff(b) >= 0)
        per = np.diff(H.irp[b].astype(np.int64))
        assert per.sum() == H.nnz
        # no block exceeds the fair share by more than the longest row
        assert per.max() <= H.nnz / parts + np.diff(H.irp).max()
    empty = synth.CRS(10, 10, np.zeros(11, np.int32), np.zeros(0, np.int32), np.zeros(0))
    assert shard.nnz_balanced_rows(empty.irp, 3).tolist()[-1] == 10
