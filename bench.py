#!/usr/bin/env python3
"""Benchmark of the run-time format transformation + SpMV + AT hot path.

One step = one pass of every row of the hot path over one synthetic matrix,
through the C ABI:
  on-line AT (analysis, D_mat, choice, build of the chosen format),
  CRS schedule, CRS -> COO-Row, CRS -> ELL-Row, Phase I (CRS -> CCS),
  Phase II (CCS -> COO-Column), CCS -> ELL-Column,
  SpMV in CRS, COO-Row, ELL-Row, COO-Column and ELL-Column.
`value` is the step's algorithmic bytes (the byte model below) over the
device time of the step, summed over ranks (each rank runs its own replica).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "SpMV GB/s (% HBM peak) per format; CRS->ELL cost in CRS-SpMV units; p99 ms"
L2_BYTES = 129 * 1024 * 1024
FALLBACK_HBM_GBS = 6800.0
PROFILE_STEPS = 3  # sequential steps timed per kernel after the timed region
PRODUCT_REPS = 20  # back-to-back products timed per format

WORKLOADS = {
    "stencil27_128": dict(kind="stencil27", N=128, seed_a=1, seed_x=2, cap=0,
                          desc="3-D 27-point stencil, 128^3 grid, N(0,1) off-diagonals, "
                               "diagonal 27 + |row sum|, x U[-1,1]"),
    "stencil27_80": dict(kind="stencil27", N=80, seed_a=1, seed_x=2, cap=0,
                         desc="3-D 27-point stencil, 80^3 grid (small case for profiling; CRS 162 MB > L2)"),
    "laplace2d_64": dict(kind="laplace", N=64, seed_x=0, cap=0,
                         desc="2-D 5-point Laplacian, 64x64 grid, x U[-1,1]"),
    "powerlaw_4m": dict(kind="powerlaw", n=4_000_000, seed_a=3, seed_x=4, cap=40 * 10 ** 9,
                        desc="n = 4e6, truncated power-law row lengths (exponent 2, mean 16, max 20000), "
                             "sorted unique random columns"),
    "powerlaw_1m": dict(kind="powerlaw", n=1_000_000, seed_a=3, seed_x=4, cap=40 * 10 ** 9,
                        desc="n = 1e6, the power law above at a quarter of the rows (CRS 196 MB > L2; "
                             "profiling size)"),
    "batch_10k": dict(kind="batch", count=10000, seed=5, n_lo=100, n_hi=20000, cap=60 * 10 ** 9,
                      desc="10,000 matrices, n log-uniform in [100, 20000]; even: 2-D 5-point stencil on a "
                           "ceil(sqrt(n)) grid cut to n, odd: Poisson(8) row lengths, unique random columns"),
    "batch_1k": dict(kind="batch", count=1000, seed=5, n_lo=100, n_hi=20000, cap=60 * 10 ** 9,
                     desc="first 1,000 matrices of batch_10k (374 MB per product, > L2; profiling size)"),
    "serve_300": dict(kind="serve", count=300, seed=6, n_lo=1000, n_hi=2000000, rate=2000.0, kmax=64,
                      requests=1500, warm_requests=200, budget=60 * 10 ** 9, streams=8, amortize=2,
                      rates=(250.0, 500.0, 750.0, 1000.0, 1500.0, 2000.0), p99_bound_ms=50.0,
                      desc="serving: pool of 300 matrices, n log-uniform in [1e3, 2e6], half cut 2-D 5-point "
                           "stencils, half power law (mean 16); Poisson arrivals (2000/s nominal, swept), 1-64 "
                           "products per request with fresh seeded x; 60 GB format-cache budget; the same "
                           "request stream through the serving runtime and through the per-matrix form"),
}
DEFAULT_WORKLOAD = "stencil27_128"


# ----------------------------------------------------------------- inputs
def make_matrix(w: dict, rank: int = 0):
    import spmv_synth as synth
    off = 1000 * rank  # each rank its own replica
    if w["kind"] == "stencil27":
        H = synth.stencil_3d_27pt(w["N"], seed=w["seed_a"] + off)
    elif w["kind"] == "laplace":
        H = synth.laplacian_2d_5pt(w["N"])
    else:
        H = synth.power_law(w["n"], seed=w["seed_a"] + off)
    x = synth.vector_pm1(H.n_cols, seed=w["seed_x"] + off)
    return H, x


def steady_products(L, torch, A, x, n_rows: int, cap: int, with_ell_row: bool) -> dict:
    """{format: {kernel: (launches, total ms)}} over PRODUCT_REPS back-to-back
    products of each format's handle (built once, 3 warm-up products)."""
    hs = {"crs": L.spmv_transform(A, L.SPMV_CRS, L.SPMV_ROWWISE),
          "coo_row": L.spmv_transform(A, L.SPMV_COO, L.SPMV_ROWWISE)}
    if with_ell_row:
        hs["ell_row"] = L.spmv_transform(A, L.SPMV_ELL, L.SPMV_ROWWISE, cap)
    ccs = L.spmv_transform(A, L.SPMV_CRS, L.SPMV_COLWISE, cap)
    hs["coo_col"] = L.spmv_transform_from(ccs, L.SPMV_COO, cap)
    hs["ell_col"] = L.spmv_transform_from(ccs, L.SPMV_ELL, cap)
    y = torch.empty(n_rows, dtype=torch.float64, device=x.device)
    out = {}
    for name, M in hs.items():
        for _ in range(3):
            L.spmv_apply(M, x, y)
        torch.cuda.synchronize()
        L.spmv_profile_read(reset=True)
        L.spmv_profile_enable(True)
        for _ in range(PRODUCT_REPS):
            L.spmv_apply(M, x, y)
        torch.cuda.synchronize()
        L.spmv_profile_enable(False)
        out[name] = L.spmv_profile_read(reset=True)
    for M in list(hs.values()) + [ccs]:
        M.close()
    return out


# -------------------------------------------------------------- byte model
def round32(n: int) -> int:
    return (n + 31) // 32 * 32


def byte_model(n_rows: int, n_cols: int, nnz: int, W: int, Wc: int) -> dict:
    """Algorithmic bytes of each hot-path row (x and y counted once)."""
    ld, ldc = round32(n_rows), round32(n_cols)
    xy = 8 * n_cols + 8 * n_rows
    return {
        "analyze": 4 * (n_rows + 1),
        "crs_schedule": 4 * (n_rows + 1) + 4 * nnz,  # row statistics + index check
        "crs_to_coo_row": 4 * (n_rows + 1) + 4 * nnz,
        "crs_to_ell_row": 12 * nnz + 4 * (n_rows + 1) + 12 * ld * W,
        "phase1_ccs": (4 * nnz + 4 * n_cols) + 8 * n_cols + (12 * nnz + 4 * (n_rows + 1) + 12 * nnz),
        "ccs_to_coo_col": 4 * (n_cols + 1) + 4 * nnz,
        "ccs_to_ell_col": 12 * nnz + 4 * (n_cols + 1) + 12 * ldc * Wc,
        "spmv_crs": 12 * nnz + 4 * (n_rows + 1) + xy,
        "spmv_coo_row": 16 * nnz + xy,
        "spmv_ell_row": 12 * ld * W + xy,
        "spmv_coo_col": 16 * nnz + xy,
        "spmv_ell_col": 12 * ldc * Wc + xy,
    }


def kernel_bytes(name: str, bm: dict, n_rows: int, n_cols: int, nnz: int):
    """Bytes one launch of a library kernel moves by design (None: not modelled)."""
    table = {
        "spmv_ell_row": bm.get("spmv_ell_row"),
        "spmv_coo_row": bm.get("spmv_coo_row"),
        "spmv_coo_col": bm.get("spmv_coo_col"),
        "spmv_ell_col": bm.get("spmv_ell_col"),
        "crs_to_ell_row": bm.get("crs_to_ell_row"),
        "ccs_to_ell_col": bm.get("ccs_to_ell_col"),
        "crs_to_coo_row": bm.get("crs_to_coo_row"),
        "ccs_to_coo_col": bm.get("ccs_to_coo_col"),
        "analyze": bm.get("analyze"),
        "row_width": 4 * (n_rows + 1),  # the ELL-Row builds' pointer pass
        "validate_idx": 4 * nnz,
        "spmv_ccs": 12 * nnz + 4 * (n_cols + 1) + 8 * n_cols + 8 * n_rows,
        # Phase I as built here: ICOL in, rank out; rank + ICOL in, (k, row)
        # pairs out; pairs + VAL gather in, ICOL_T + VAL_T out
        "col_count": 8 * nnz + 4 * n_cols,
        "scan_lookback": 8 * n_cols,
        "col_scatter": 16 * nnz + 4 * (n_rows + 1) + 4 * n_cols,
        "col_fixup_tiles": 28 * nnz + 4 * n_cols,
        # slot path: ICOL in, rank out, (k, row) into the slot array; slots in,
        # VAL gathered, ICOL_T + VAL_T out
        "col_claim": 16 * nnz + 4 * (n_rows + 1) + 4 * n_cols,
        "col_fixup_slots": 28 * nnz + 4 * n_cols,
        "col_overflow": 0,
        "tile_lines": 4 * (nnz // 2048 + 1),
        "spmv_coo_row_carry": 16 * (nnz // 2048 + 1),
        "col_fixup_block": 0,
        # row-position slot path (neighbouring columns): ICOL in, one 8-byte
        # {k, row} slot out; slots in, VAL gathered by k, ICOL_T + VAL_T out
        "col_claim_rk": 12 * nnz + 4 * (n_rows + 1) + 4 * n_cols,
        "coo_col_tile_bounds": 8 * (n_cols // 128 + 1),
        "col_fixup_rk": 28 * nnz + 4 * (n_cols + 1),
        "col_overflow_rk": 0,
        # grouped row-value path (the default): the same bytes, records in
        # 64-column group regions; the fix-up also writes IRP_T
        "col_claim_grp": 28 * nnz + 4 * (n_rows + 1),
        "col_locality": 8 * 4096,
        "col_fixup_grp": 28 * nnz + 4 * (n_cols + 1),
        "col_fixup_long_rv": 0,
        # structurally symmetric path: ICOL and IRP in, VAL gathered from the
        # mirror entries, ICOL_T (= ICOL) and VAL_T out (IRP_T is a copy of IRP)
        "ccs_sym": 24 * nnz + 8 * (n_rows + 1),
        "sym_sample": 16 * 4096,
        # the measuring stick of the column-wise products: atomics into y only
        "atomic_ceiling": 8 * n_rows,
        "crs_to_ell_row_fused_spmv": (bm["crs_to_ell_row"] + 8 * n_cols + 8 * n_rows) if "crs_to_ell_row" in bm else None,
    }
    if name.startswith("spmv_crs_"):
        return bm["spmv_crs"]
    if name.startswith("spmv_coo_row_rows") or name == "spmv_coo_row_seg":
        return bm["spmv_coo_row"]
    if name.startswith("spmv_coo_col_cols"):
        return bm["spmv_coo_col"]
    if name == "coo_row_tile_bounds":
        return 8 * (n_rows // 128 + 1)
    return table.get(name)


# --------------------------------------------------------------- the step
class Step:
    """All hot-path rows through the C ABI on one device-resident matrix.

    Three pipelines share nothing but the input: the on-line AT with the CRS
    schedule and ELL-Row (and their products), COO-Row (and its product), and
    the column-wise path (Phase I, then Phase II and CCS->ELL-Column, which
    both only read the CCS, and their products). With `concurrent` they run
    at the same time on CUDA streams (four: the column-wise path forks after
    Phase I), each driven by its own host thread (the library's calls
    synchronise per call, so one host thread would serialise them). Without
    it, they run one after the other on the current stream."""

    def __init__(self, L, A, x, ys, dstar: float, cap: int, concurrent: bool = False):
        self.L, self.A, self.x, self.ys = L, A, x, ys
        self.dstar, self.cap = dstar, cap
        self.chosen = None
        self.concurrent = concurrent
        if concurrent:
            import concurrent.futures as cf
            import torch
            self.torch = torch
            self.device = torch.cuda.current_device()
            self.streams = [torch.cuda.Stream() for _ in range(4)]
            # three workers: the column-wise task, the COO-Row task and the
            # column-wise task's second branch (which it waits for, so fewer
            # workers could deadlock)
            self.pool = cf.ThreadPoolExecutor(3)

    def _at(self, s):
        L, A = self.L, self.A
        chosen, stats = L.spmv_autotune(A, stream=s, dstar=self.dstar, mem_cap_bytes=self.cap)
        fmt = chosen.describe()["format"]
        self.chosen = {0: "CRS", 1: "COO-Row", 2: "ELL-Row"}[fmt]
        mats = {}
        # each product runs right after its own handle is built: the CRS
        # product does not follow the ELL build, whose 680 MB of writes would
        # still be draining from L2 during it
        mats["crs"] = chosen if fmt == L.SPMV_CRS else L.spmv_transform(A, L.SPMV_CRS, L.SPMV_ROWWISE, stream=s)
        L.spmv_apply(mats["crs"], self.x, self.ys["crs"], stream=s)
        if fmt == L.SPMV_ELL:
            mats["ell_row"] = chosen
        elif not self.cap or stats["ell_bytes"] <= self.cap:
            mats["ell_row"] = L.spmv_transform(A, L.SPMV_ELL, L.SPMV_ROWWISE, self.cap, stream=s)
        if "ell_row" in mats:
            L.spmv_apply(mats["ell_row"], self.x, self.ys["ell_row"], stream=s)
        self.stats = stats
        return list(mats.values())

    def _coo(self, s):
        L = self.L
        if self.concurrent:
            self.torch.cuda.set_device(self.device)
        M = L.spmv_transform(self.A, L.SPMV_COO, L.SPMV_ROWWISE, stream=s)
        L.spmv_apply(M, self.x, self.ys["coo_row"], stream=s)
        return [M]

    def _col_branch(self, ccs, fmt, name, s):
        L = self.L
        if self.concurrent:
            self.torch.cuda.set_device(self.device)
        M = L.spmv_transform_from(ccs, fmt, self.cap, stream=s)
        L.spmv_apply(M, self.x, self.ys[name], stream=s)
        return [M]

    def _col(self, s, s2=None):
        L, A = self.L, self.A
        if self.concurrent:
            self.torch.cuda.set_device(self.device)
        ccs = L.spmv_transform(A, L.SPMV_CRS, L.SPMV_COLWISE, self.cap, stream=s)
        if s2 is None:
            hs = self._col_branch(ccs, L.SPMV_COO, "coo_col", s) + self._col_branch(ccs, L.SPMV_ELL, "ell_col", s)
            return hs + [ccs]
        # Phase II and CCS -> ELL-Column both only read the CCS: one branch per stream
        built = self.torch.cuda.Event()
        built.record(s)
        s2.wait_event(built)
        f = self.pool.submit(self._col_branch, ccs, L.SPMV_ELL, "ell_col", s2)
        hs = self._col_branch(ccs, L.SPMV_COO, "coo_col", s)
        return hs + f.result() + [ccs]

    def run(self):
        if not self.concurrent:
            hs = self._at(None) + self._coo(None) + self._col(None)
            for M in hs:
                M.close()
            return self.stats
        torch = self.torch
        main = torch.cuda.current_stream()
        start = torch.cuda.Event()
        start.record(main)
        for st in self.streams:
            st.wait_event(start)
        f_col = self.pool.submit(self._col, self.streams[2], self.streams[3])
        f_coo = self.pool.submit(self._coo, self.streams[1])
        hs = self._at(self.streams[0]) + f_coo.result() + f_col.result()
        for st in self.streams:
            e = torch.cuda.Event()
            e.record(st)
            main.wait_event(e)
        for M in hs:  # freed in stream order on the streams that made them
            M.close()
        return self.stats


def calibrate_dstar(L, torch, quick: bool = True):
    """Off-line phase (Sec. 2.2) on a small synthetic set on this device."""
    import spmv_synth as synth
    mats = [synth.laplacian_2d_5pt(1024), synth.stencil_3d_27pt(64),
            synth.random_crs(1000000, 1000000, 12, seed=41),
            synth.power_law(1000000, kmax=2000, seed=42), synth.power_law(1000000, kmax=20000, seed=43)]
    dev = [L.Crs.from_host(H) for H in mats]
    dstar, d, r = L.spmv_calibrate(dev, c=1.0, timing_reps=5 if quick else 20, warmup_reps=2)
    return dstar, d, r


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.out = []  # (host time of arrival, line)
        self.window = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.out.append((time.perf_counter(), line.strip()))

    def mark(self, t0: float, t1: float):
        """Host-time window of the timed region."""
        self.window = (t0, t1)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.05)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = self.out
        if self.window:
            t0, t1 = self.window
            inside = [(t, l) for t, l in self.out if t0 <= t <= t1 + 0.03]
            if not inside and self.out:  # the region was shorter than one period: nearest sample
                mid = 0.5 * (t0 + t1)
                inside = [min(self.out, key=lambda tl: abs(tl[0] - mid))]
            lines = inside
        for _, line in lines:
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ distributed
def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def reduce_max_sum(torch, ms: float, nbytes: float, device, group=None):
    """(max of ms, sum of bytes) over ranks; identity when not distributed."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return ms, nbytes
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    b = torch.tensor([nbytes], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(b, op=dist.ReduceOp.SUM, group=group)
    return float(t.item()), float(b.item())


def barrier_sync(torch):
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()
    if torch.cuda.is_available():
        torch.cuda.synchronize()


# ------------------------------------------------------------ CPU oracle
def oracle_step(H, xh, cap: int = 0, omp: bool = False) -> dict:
    """The same rows on the CPU oracle; returns {row: seconds}. ELL-Row is
    left out, as in the GPU step, when its bytes exceed the workload's cap.
    omp: the CRS and ELL-Row products and Phase I's count and pointers run on
    all host cores (the multi-core oracle build, same bits), the rest serial."""
    import oracle
    spmv_crs = oracle.spmv_crs_omp if omp else oracle.spmv_crs
    spmv_ell_row = oracle.spmv_ell_row_omp if omp else oracle.spmv_ell_row
    t = {}
    c = time.perf_counter
    t0 = c(); st = oracle.analyze(H.n_rows, H.irp); t["analyze"] = c() - t0
    ell = not cap or 12 * H.n_rows * int(st["W"]) + 4 * (H.n_rows + 1) <= cap
    t0 = c(); irow = oracle.crs_to_coo_row(H.n_rows, H.irp); t["crs_to_coo_row"] = c() - t0
    W = int(st["W"])
    if ell:
        t0 = c(); ev, ec, W = oracle.crs_to_ell_row(H.n_rows, H.irp, H.icol, H.val); t["crs_to_ell_row"] = c() - t0
    t0 = c()
    if omp:
        irp_t, icol_t, val_t = oracle.crs_to_ccs_omp(H.n_rows, H.n_cols, H.irp, H.icol, H.val)
    else:
        irp_t, icol_t, val_t, nc = oracle.crs_to_ccs(H.n_rows, H.n_cols, H.irp, H.icol, H.val)
    t["phase1_ccs"] = c() - t0
    t0 = c(); jcol = oracle.ccs_to_coo_col(H.n_cols, irp_t); t["ccs_to_coo_col"] = c() - t0
    t0 = c(); ev2, er2, W2 = oracle.ccs_to_ell_col(H.n_cols, irp_t, icol_t, val_t); t["ccs_to_ell_col"] = c() - t0
    t0 = c(); spmv_crs(H.n_rows, H.irp, H.icol, H.val, xh); t["spmv_crs"] = c() - t0
    t0 = c(); oracle.spmv_coo(H.n_rows, irow, H.icol, H.val, xh); t["spmv_coo_row"] = c() - t0
    if ell:
        t0 = c(); spmv_ell_row(H.n_rows, W, ev, ec, xh); t["spmv_ell_row"] = c() - t0
    t0 = c(); oracle.spmv_coo(H.n_rows, icol_t, jcol, val_t, xh); t["spmv_coo_col"] = c() - t0
    t0 = c(); oracle.spmv_ell_col(H.n_rows, H.n_cols, W2, ev2, er2, xh); t["spmv_ell_col"] = c() - t0
    t["_W"], t["_Wc"], t["_ell"] = W, W2, ell
    return t


def host_cpu() -> dict:
    """The host's logical CPUs (nproc) and CPU model (lscpu, else /proc/cpuinfo)."""
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as fh:
                for line in fh:
                    if line.lower().startswith(("model name", "cpu model")):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return {"nproc": os.cpu_count() or 1, "model": model or "unknown"}


def oracle_bytes(H, W, Wc, ell: bool = True) -> float:
    bm = byte_model(H.n_rows, H.n_cols, H.nnz, W, Wc)
    # the oracle's ELL has ld = n; the row set matches the GPU step minus the
    # CRS schedule (the oracle needs none)
    keys = ["analyze", "crs_to_coo_row", "crs_to_ell_row", "phase1_ccs", "ccs_to_coo_col", "ccs_to_ell_col",
            "spmv_crs", "spmv_coo_row", "spmv_ell_row", "spmv_coo_col", "spmv_ell_col"]
    if not ell:
        keys = [k for k in keys if k not in ("crs_to_ell_row", "spmv_ell_row")]
    return float(sum(bm[k] for k in keys))


def workload_config(name: str, w: dict, H, W: int, Wc: int, dmat: float, world: int) -> dict:
    """The workload keys of the JSON line, the same for the native and the
    reference arm: the matrix, its ELL widths, D_mat and the step's
    algorithmic bytes (ELL-Row left out when its bytes exceed the cap, as the
    step does)."""
    bm = byte_model(H.n_rows, H.n_cols, H.nnz, W, Wc)
    if w["cap"] and 12 * round32(H.n_rows) * W > w["cap"]:
        bm.pop("crs_to_ell_row")
        bm.pop("spmv_ell_row")
    return {"workload": name, "desc": w["desc"], "n": H.n_rows, "nnz": H.nnz, "W": W, "W_col": Wc,
            "D_mat": dmat, "step_bytes": float(sum(bm.values())), "parallelism": f"replicas x{world}"}


CPU_SAMPLE_FRAC = 4  # the CPU legs run rows 0 .. n/4 of the workload


def _oracle_leg(S, xs, cap: int, omp: bool, budget_s: float):
    tot_t, tot_b, runs = 0.0, 0.0, 0
    while tot_t < budget_s and runs < 20:
        t = oracle_step(S, xs, cap, omp=omp)
        tot_t += sum(v for k, v in t.items() if not k.startswith("_"))
        tot_b += oracle_bytes(S, t["_W"], t["_Wc"], t["_ell"])
        runs += 1
    return tot_b / tot_t / 1e9, runs, tot_t


def cpu_baseline(H, xh, budget_s: float = 10.0, cap: int = 0) -> dict:
    """Times the oracle on a bounded row sample of the workload, on one thread
    and with the multi-core build on every host core. `value` and `cores` are
    the multi-core figures; the single-thread figure sits beside them."""
    import oracle
    rows = max(1, H.n_rows // CPU_SAMPLE_FRAC)
    S = H.row_slice(0, rows)
    xs = xh  # the slice keeps all columns
    host = host_cpu()
    v1, r1, t1 = _oracle_leg(S, xs, cap, False, budget_s)
    try:
        threads = oracle.omp_threads()
        vm, rm, tm = _oracle_leg(S, xs, cap, True, budget_s)
    except Exception as e:  # no OpenMP toolchain on the host: single thread only
        return {"value": v1, "unit": "GB/s", "cores": 1, "kind": "oracle", "cpu_model": host["model"],
                "nproc": host["nproc"],
                "sample": f"rows 0..{rows} of {H.n_rows} ({S.nnz} nnz), {r1} oracle step(s), {t1:.1f} s, single "
                          f"thread (multi-core build unavailable: {type(e).__name__})"}
    return {"value": vm, "unit": "GB/s", "cores": threads, "kind": "oracle", "cpu_model": host["model"],
            "nproc": host["nproc"],
            "single_thread": {"value": v1, "unit": "GB/s", "cores": 1, "steps": r1, "seconds": round(t1, 2)},
            "sample": f"rows 0..{rows} of {H.n_rows} ({S.nnz} nnz), {rm} oracle step(s), {tm:.1f} s on {threads} "
                      f"threads: CRS and ELL-Row products and the Phase I count and pointers in parallel, every "
                      f"other row and the Phase I scatter serial, FP64"}


# -------------------------------------------------------------- reference
def run_reference(args, w: dict) -> None:
    """The reference arm: the oracle as it stands (multi-core build where it
    has one, on every host core), on a row sample of the same workload."""
    import numpy as np
    import oracle
    rank, world, _ = dist_env()
    if rank != 0:
        return
    H, xh = make_matrix(w)
    rows = max(1, H.n_rows // 16)
    S = H.row_slice(0, rows)
    try:
        threads, omp = oracle.omp_threads(), True
    except Exception:
        threads, omp = 1, False
    for _ in range(args.warmup):
        oracle_step(S, xh, w.get("cap", 0), omp=omp)
    ts, bs = [], []
    for _ in range(args.steps):
        t = oracle_step(S, xh, w.get("cap", 0), omp=omp)
        ts.append(sum(v for k, v in t.items() if not k.startswith("_")))
        bs.append(oracle_bytes(S, t["_W"], t["_Wc"], t["_ell"]))
    total = sum(ts)
    value = sum(bs) / total / 1e9
    host = host_cpu()
    what = (f"{threads} threads (CRS, ELL-Row and the Phase I count in parallel, the rest serial)" if omp
            else "single thread")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {**workload_config(args.workload, w, H, int(np.diff(H.irp).max(initial=0)),
                                     int(np.bincount(H.icol, minlength=H.n_cols).max(initial=0)),
                                     oracle.analyze(H.n_rows, H.irp)["dmat"], world),
                   "sample_rows": rows, "sample_nnz": S.nnz,
                   "l2": "CPU oracle on the host cores (no GPU, no L2 flush)"},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": threads, "kind": "oracle",
                         "cpu_model": host["model"], "nproc": host["nproc"],
                         "sample": f"rows 0..{rows} of {H.n_rows} per step, FP64 oracle on {what}"},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------- batches
def _batch_part(args):
    import spmv_synth as synth
    lo, hi, seed, n_lo, n_hi = args
    return [synth.batch_matrix(i, seed, n_lo, n_hi) for i in range(lo, hi)]


def make_batch(w: dict, rank: int = 0):
    """The batch's host matrices, generated by a spawned process pool."""
    import concurrent.futures as cf
    import multiprocessing as mp
    seed = w["seed"] + 100000 * rank
    n, step = w["count"], 250
    parts = [(lo, min(n, lo + step), seed, w["n_lo"], w["n_hi"]) for lo in range(0, n, step)]
    workers = max(1, min(16, (os.cpu_count() or 2) - 1))
    with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        out = []
        for part in ex.map(_batch_part, parts):
            out.extend(part)
    return out


def batch_bytes(mats, plans) -> float:
    """Algorithmic bytes of one product over the batch: CRS 12 nnz + 4 (n+1),
    ELL 12 ld W, plus x and y once each."""
    b = 0.0
    for H, P in zip(mats, plans):
        if P["format"] == 2:
            b += 12.0 * P["ld"] * P["width"]
        else:
            b += 12.0 * H.nnz + 4.0 * (H.n_rows + 1)
        b += 8.0 * H.n_cols + 8.0 * H.n_rows
    return b


def per_matrix_loop(L, torch, dev, mats, plans, x, y, stream):
    """The same products as a loop of one spmv_apply per matrix (one CRS
    handle each), plain and captured in one CUDA graph; ms per loop."""
    handles = [L.spmv_transform(A, L.SPMV_CRS, L.SPMV_ROWWISE) for A in dev]
    views = [(x[P["x_offset"]:P["x_offset"] + H.n_cols], y[P["y_offset"]:P["y_offset"] + H.n_rows])
             for H, P in zip(mats, plans)]
    reps = 3

    def loop():
        for M, (xv, yv) in zip(handles, views):
            L.spmv_apply(M, xv, yv)

    loop()
    barrier_sync(torch)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        loop()
    e1.record(stream)
    barrier_sync(torch)
    loop_ms = e0.elapsed_time(e1) / reps
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="relaxed"):
        loop()
    g.replay()
    barrier_sync(torch)
    e0.record(stream)
    for _ in range(reps):
        g.replay()
    e1.record(stream)
    barrier_sync(torch)
    graph_ms = e0.elapsed_time(e1) / reps
    del g
    for M in handles:
        M.close()
    return loop_ms, graph_ms


def run_batch(args, w: dict) -> None:
    """One step = one product y = A x over every matrix of the batch (one
    launch). Also timed: the batch build (analysis, on-line rule, ELL
    build fused with a first product) and the same products as a loop of
    one spmv_apply per matrix, plain and captured in a CUDA graph."""
    rank, world, local = dist_env()
    if args.impl == "reference":
        if rank != 0:
            return
        import oracle
        import spmv_synth as synth
        mats = [synth.batch_matrix(i, w["seed"], w["n_lo"], w["n_hi"]) for i in range(400)]
        xs = [synth.vector_pm1(H.n_cols, seed=7 + i) for i, H in enumerate(mats)]
        for H, x in list(zip(mats, xs))[:args.warmup]:
            oracle.spmv_crs(H.n_rows, H.irp, H.icol, H.val, x)
        t0 = time.perf_counter()
        nb = 0.0
        for _ in range(args.steps):
            for H, x in zip(mats, xs):
                oracle.spmv_crs(H.n_rows, H.irp, H.icol, H.val, x)
                nb += 12.0 * H.nnz + 4.0 * (H.n_rows + 1) + 8.0 * (H.n_cols + H.n_rows)
        tot = time.perf_counter() - t0
        v = nb / tot / 1e9
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": "GB/s", "n_gpus": world,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic", "config": {"workload": args.workload, "sample_matrices": 400},
                          "cpu_baseline": {"value": v, "unit": "GB/s", "cores": 1, "kind": "oracle",
                                           "sample": "matrices 0..399 of the batch per step, CRS SpMV, single "
                                                     "thread"},
                          "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                          "gpu_launches": 0}), flush=True)
        return
    mats = make_batch(w, rank)  # before the first GPU call (spawned pool)
    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    import paper_2407_00019_gb300 as L
    import spmv_synth as synth
    L.load_library()
    dev = L.Crs.batch_from_host(mats, device=device)
    nc = sum(H.n_cols for H in mats)
    nr = sum(H.n_rows for H in mats)
    xh = synth.vector_pm1(nc, seed=7 + 1000 * rank)
    x = torch.from_numpy(xh).to(device)
    y = torch.empty(nr, dtype=torch.float64, device=device)
    if args.dstar is None:
        # the max-pass rule of the committed calibration: members with small
        # D_mat (the stencils) take ELL-Row, the rest CRS
        dstar, dstar_src = committed_dstar(L, torch, "maxpass")
    else:
        dstar, dstar_src = args.dstar, "--dstar"
    stream = torch.cuda.current_stream()
    # the committed off-line schedule table of this device (lanes per row by
    # mean row length), else the library's default
    from paper_2407_00019_gb300 import calibrate as cal
    try:
        L.spmv_batch_schedule_set(cal.load_schedule(cal.committed_schedule_path(), torch.cuda.get_device_name()))
        sched_src = "committed schedule calibration"
    except (OSError, ValueError, KeyError):
        sched_src = "library default (no committed schedule for this device)"
    # build: analysis + on-line rule + ELL build fused with the first product
    create_ms = []
    for _ in range(3):
        barrier_sync(torch)
        t0 = time.perf_counter()
        B = L.spmv_batch_create(dev, x=x, y=y, dstar=dstar, mem_cap_bytes=w["cap"])
        torch.cuda.synchronize()
        create_ms.append(1e3 * (time.perf_counter() - t0))
        B.close()
    B = L.spmv_batch_create(dev, dstar=dstar, mem_cap_bytes=w["cap"])
    info, plans = B.info(), B.plans()
    step_bytes = batch_bytes(mats, plans)
    # the same build planned on the device and captured, with its first
    # product, in one CUDA graph (pool sized to the host plan's ELL bytes)
    D = L.spmv_batch_prepare(dev, dstar=dstar, mem_cap_bytes=max(info["ell_bytes"], 1 << 20))
    gs = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(graph, stream=gs):
        D.build(x, y)
    gms = []
    for _ in range(4):
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        graph.replay()
        g1.record(stream)
        g1.synchronize()
        gms.append(g0.elapsed_time(g1))
    D.status()
    dinfo = D.info()
    graph_build = {"ms": statistics.median(gms[1:]), "n_ell": dinfo["n_ell"], "n_tiles": dinfo["n_tiles"],
                   "same_plan_as_host": dinfo["n_ell"] == info["n_ell"] and dinfo["n_tiles"] == info["n_tiles"],
                   "what": "analysis, on-line rule, tile records, ELL build and first product: one CUDA graph "
                           "replayed (device time)"}
    del graph
    D.close()

    clocks = ClockSampler(local)
    clocks.start()
    for _ in range(args.warmup):
        B.apply(x, y)
    barrier_sync(torch)
    L.spmv_profile_read(reset=True)
    L.spmv_profile_enable(True)
    launches0 = L.spmv_launch_count()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    barrier_sync(torch)
    h0 = time.perf_counter()
    ev[0].record(stream)
    for i in range(args.steps):
        B.apply(x, y)
        ev[i + 1].record(stream)
    barrier_sync(torch)
    clocks.mark(h0, time.perf_counter())
    launches = L.spmv_launch_count() - launches0
    clk = clocks.stop()
    L.spmv_profile_enable(False)
    prof = L.spmv_profile_read(reset=True)
    per_step = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    t_max, bytes_all = reduce_max_sum(torch, ev[0].elapsed_time(ev[-1]), step_bytes * args.steps, device)
    value = bytes_all / (t_max * 1e-3) / 1e9
    peak, peak_kind = measured_hbm_peak()
    n_k, ms_k = prof["batch_apply"]
    achieved = step_bytes / (ms_k / n_k * 1e-3) / 1e9

    loop_ms = graph_ms = None
    if not args.no_loop:
        loop_ms, graph_ms = per_matrix_loop(L, torch, dev, mats, plans, x, y, stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    e2e = None
    if not args.no_e2e:
        xpin = torch.from_numpy(xh).pin_memory()
        ypin = torch.empty(nr, dtype=torch.float64).pin_memory()
        barrier_sync(torch)
        e0.record(stream)
        for _ in range(args.steps):
            x.copy_(xpin, non_blocking=True)
            B.apply(x, y)
            ypin.copy_(y, non_blocking=True)
        e1.record(stream)
        barrier_sync(torch)
        et, eb = reduce_max_sum(torch, e0.elapsed_time(e1), step_bytes * args.steps, device)
        e2e = {"value": eb / (et * 1e-3) / 1e9, "unit": "GB/s", "h2d_bytes_per_step": 8 * nc,
               "d2h_bytes_per_step": 8 * nr, "ms_per_step": et / args.steps}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        t0 = time.perf_counter()
        nb, k = 0.0, 0
        while time.perf_counter() - t0 < 10.0 and k < len(mats):
            H, P = mats[k], plans[k]
            oracle.spmv_crs(H.n_rows, H.irp, H.icol, H.val, xh[P["x_offset"]:P["x_offset"] + H.n_cols])
            nb += 12.0 * H.nnz + 4.0 * (H.n_rows + 1) + 8.0 * (H.n_cols + H.n_rows)
            k += 1
        tc = time.perf_counter() - t0
        cpu = {"value": nb / tc / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": f"CRS SpMV of matrices 0..{k - 1} of {len(mats)}, {tc:.1f} s, single thread"}

    if rank == 0:
        srt = sorted(per_step)
        p99 = srt[min(len(srt) - 1, int(math.ceil(0.99 * len(srt))) - 1)]
        fmt_count = {"ELL-Row": info["n_ell"], "CRS": info["n_matrices"] - info["n_ell"]}
        tpr = {}
        for P in plans:
            if P["format"] == 0:
                tpr[str(P["threads_per_row"])] = tpr.get(str(P["threads_per_row"]), 0) + 1
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "desc": w["desc"], "matrices": len(mats), "rows": nr,
                       "nnz": info["total_nnz"], "step_bytes": step_bytes, "tiles": info["n_tiles"],
                       "grid": info["grid"], "l2": "inputs larger than L2 (%.0f MB); no flush" % (step_bytes / 1e6),
                       "parallelism": f"replicas x{world}"},
            "roofline": {"kernel": "batch_apply", "bound": "hbm", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_kind,
                         "traffic": stored_traffic("batch_apply", args.workload),
                         "algorithmic_bytes_per_launch": step_bytes},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
            "p50_ms": statistics.median(per_step), "p99_ms": p99,
            "batch": {"create_ms": statistics.median(create_ms), "per_matrix_loop_ms": loop_ms,
                      "per_matrix_graph_ms": graph_ms,
                      "speedup_vs_loop": loop_ms / (t_max / args.steps) if loop_ms else None,
                      "speedup_vs_graph": graph_ms / (t_max / args.steps) if graph_ms else None,
                      "dstar": dstar if math.isfinite(dstar) else "inf", "dstar_source": dstar_src,
                      "formats": fmt_count,
                      "crs_threads_per_row": tpr, "schedule_table": L.spmv_batch_schedule_get(),
                      "schedule_source": sched_src, "graph_build": graph_build},
        }
        print(json.dumps(line), flush=True)
    B.close()
    if world > 1:
        dist.destroy_process_group()


# --------------------------------------------------------------- serving
def _serve_part(args):
    import spmv_synth as synth
    lo, hi, seed, n_lo, n_hi = args
    return [synth.serve_matrix(i, seed, n_lo, n_hi) for i in range(lo, hi)]


def committed_dstar(L, torch, rule: str):
    """D* of the committed off-line calibration of this device (the
    Table-1-shaped set, Sec. 2.2, 30 timed repetitions) under `rule`, else a
    quick calibration here; returns (D*, source)."""
    from paper_2407_00019_gb300 import calibrate as cal
    try:
        return cal.load_dstar(cal.committed_path(rule), torch.cuda.get_device_name()), f"committed {rule} calibration"
    except (OSError, ValueError, KeyError):
        return calibrate_dstar(L, torch)[0], "quick calibration (no committed file for this device)"


def serve_dstar(L, torch):
    """D* for serving: the max-pass rule, under which matrices with small D_mat
    target ELL-Row and the break-even rule decides when to build it."""
    return committed_dstar(L, torch, "maxpass")


def serve_arm(L, torch, S, ids, dev, reqs, rate, seed, device, warm, cap_bytes=16 * 10 ** 9):
    """Offers the request list `reqs` [(matrix, k)] at `rate` per second
    (Poisson gaps) to server S; the first `warm` requests are not measured.
    Each request's x is drawn on the device from its own seed just before
    submission; latency runs from its planned arrival to its completion, so
    time a request spends waiting behind the client (which keeps at most
    cap_bytes of x and y outstanding) counts too."""
    import numpy as np
    rng = np.random.default_rng(seed + int(rate))
    gaps = rng.exponential(1.0 / rate, size=len(reqs))
    pending, lat = [], []  # pending: [handle, planned arrival, submit time, bytes, x, y]
    held = 0

    def finish_oldest():
        nonlocal held
        h, t_arr, t_sub, nb, _, _ = pending.pop(0)
        ms, _ = S.wait(h, 600000)
        lat.append((t_sub - t_arr) * 1e3 + ms)
        held -= nb

    t_next = t0 = time.perf_counter()
    launches0 = L.spmv_launch_count()
    for r, (i, k) in enumerate(reqs):
        if r == warm:
            while pending:
                finish_oldest()
            lat.clear()
            S.stats(reset=True)
            t_next = t0 = time.perf_counter()
            launches0 = L.spmv_launch_count()
        t_next += gaps[r]
        while time.perf_counter() < t_next:
            pass
        A = dev[i]
        nb = 8 * k * (A.n_cols + A.n_rows)
        while pending and held + nb > cap_bytes:
            finish_oldest()
        g = torch.Generator(device=device)
        g.manual_seed(seed * 1000003 + r)
        x = torch.rand(k * A.n_cols, generator=g, dtype=torch.float64, device=device)
        y = torch.empty(k * A.n_rows, dtype=torch.float64, device=device)
        t_sub = time.perf_counter()
        pending.append([S.submit(ids[i], k, x, y), t_next, t_sub, nb, x, y])
        held += nb
    while pending:
        finish_oldest()
    t1 = time.perf_counter()
    st = S.stats()
    lat = np.array(lat)
    return {"offered_req_per_s": rate, "served_req_per_s": len(lat) / (t1 - t0),
            "GB/s": st["bytes"] / (t1 - t0) / 1e9, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "max_ms": float(lat.max()), "requests": int(len(lat)),
            "products": int(st["products"]), "launches": int(L.spmv_launch_count() - launches0),
            "cache": {k: st[k] for k in ("cache_hits", "cache_misses", "transforms", "evictions", "cache_bytes",
                                         "peak_cache_bytes")}, "seconds": t1 - t0}


def run_serve(args, w: dict) -> None:
    """One request stream (Poisson arrivals, each request k products with one
    matrix of the pool) served twice: by the serving runtime (continuous
    batching over stream slots, resident formats chosen by the on-line rule
    and built at their break-even point, a request's k products in one
    launch) and by the per-matrix form (requests one after the other, one
    spmv_apply per product on CRS). Each arm is swept over offered rates;
    reported: GB/s and latency percentiles per rate, and each arm's highest
    served rate with p99 latency within the stated bound."""
    import concurrent.futures as cf
    import multiprocessing as mp
    rank, world, local = dist_env()
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps({"impl": "reference", "unavailable": "serving has no CPU counterpart: the oracle "
                              "computes products, it does not schedule requests"}), flush=True)
        return
    seed = w["seed"] + 100000 * rank
    parts = [(lo, min(w["count"], lo + 4), seed, w["n_lo"], w["n_hi"]) for lo in range(0, w["count"], 4)]
    workers = max(1, min(16, (os.cpu_count() or 2) - 1))
    t_gen = time.perf_counter()
    with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        pool = [H for part in ex.map(_serve_part, parts) for H in part]
    t_gen = time.perf_counter() - t_gen
    import numpy as np
    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    import paper_2407_00019_gb300 as L
    L.load_library()
    dev = L.Crs.batch_from_host(pool, device=device)
    if args.dstar is not None:
        dstar, dsrc = args.dstar, "--dstar"
    else:
        dstar, dsrc = serve_dstar(L, torch)
    if args.requests:
        w = dict(w, requests=int(args.requests), warm_requests=max(50, int(args.requests) // 6))
    rng = np.random.default_rng(seed)
    n_req = w["warm_requests"] + w["requests"]
    reqs = list(zip(rng.integers(0, len(pool), size=n_req).tolist(), rng.integers(1, w["kmax"] + 1, size=n_req).tolist()))
    rates = [args.rate] if args.rate else list(w["rates"])
    if not args.rate and w["rate"] not in rates:
        rates.append(w["rate"])
    rates = sorted(rates)
    clocks = ClockSampler(local)
    clocks.start()
    h0 = time.perf_counter()
    arms = {}
    for arm, flags, streams in (("serve", 0, w["streams"]), ("plain", L.Server.PLAIN, 1)):
        S = L.Server(mem_budget_bytes=w["budget"], dstar=dstar, n_streams=streams, amortize_products=w["amortize"],
                     flags=flags)
        ids = [S.add_matrix(A) for A in dev]
        arms[arm] = []
        for rate in rates:
            res = serve_arm(L, torch, S, ids, dev, reqs, rate, seed, device, w["warm_requests"])
            arms[arm].append(res)
            if res["p99_ms"] > 20 * w["p99_bound_ms"]:
                break  # far past saturation: higher rates only queue longer
        S.close()
        torch.cuda.empty_cache()
    h1 = time.perf_counter()
    clocks.mark(h0, h1)
    clk = clocks.stop()
    peak, peak_kind = measured_hbm_peak()
    bound = w["p99_bound_ms"]

    def best(rows):
        ok = [r for r in rows if r["p99_ms"] <= bound]
        if not ok:
            return None
        r = max(ok, key=lambda r: r["served_req_per_s"])
        return {"offered_req_per_s": r["offered_req_per_s"], "served_req_per_s": r["served_req_per_s"],
                "GB/s": r["GB/s"], "p99_ms": r["p99_ms"]}
    nominal = {a: next(r for r in rows if r["offered_req_per_s"] == w["rate"]) if any(
        r["offered_req_per_s"] == w["rate"] for r in rows) else None for a, rows in arms.items()}
    nom = nominal["serve"] or arms["serve"][0]
    t_max, b_all = reduce_max_sum(torch, nom["seconds"] * 1e3, nom["GB/s"] * nom["seconds"] * 1e9, device)
    at_bound = {a: best(rows) for a, rows in arms.items()}
    if rank == 0:
        line = {
            "metric": METRIC, "value": b_all / (t_max * 1e-3) / 1e9, "unit": "GB/s", "n_gpus": world,
            "steps": w["requests"], "warmup": w["warm_requests"], "ms_per_step": nom["seconds"] * 1e3 / w["requests"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "desc": w["desc"], "pool_nnz": int(sum(H.nnz for H in pool)),
                       "pool_rows": int(sum(H.n_rows for H in pool)), "pool_max_n": int(max(H.n_rows for H in pool)),
                       "pool_generation_s": round(t_gen, 1), "streams": w["streams"],
                       "amortize_products": w["amortize"], "dstar": dstar if math.isfinite(dstar) else "inf",
                       "dstar_source": dsrc, "nominal_req_per_s": w["rate"], "p99_bound_ms": bound,
                       "parallelism": f"replicas x{world}",
                       "value": "serving runtime at the nominal rate: algorithmic bytes of the products served "
                                "(each format's byte model) over the measured interval"},
            "p50_ms": nom["p50_ms"], "p99_ms": nom["p99_ms"], "served_req_per_s": nom["served_req_per_s"],
            "frac_of_hbm_peak": nom["GB/s"] / peak, "peak": peak, "peak_source": peak_kind,
            "cache": nom["cache"], "arms": arms, "at_p99_bound": at_bound,
            "serving_beats_plain_at_p99_bound": (at_bound["serve"] is not None and (
                at_bound["plain"] is None or at_bound["serve"]["served_req_per_s"] >
                at_bound["plain"]["served_req_per_s"])),
            "gpu_launches": nom["launches"], "clocks": clk, "e2e": None, "cpu_baseline": None,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ------------------------------------------------------------------- main
def measured_hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


# Source files whose device code decides each kernel's DRAM traffic (the
# shared device header counts for all of them).
KERNEL_FILES = {
    "col_claim_rk": "kernels_colwise.cu", "col_fixup_rk": "kernels_colwise.cu", "ccs_sym": "kernels_colwise.cu",
    "col_claim_grp": "kernels_colwise.cu", "col_fixup_grp": "kernels_colwise.cu",
    "col_claim": "kernels_colwise.cu", "col_fixup_slots": "kernels_colwise.cu",
    "crs_to_ell_row": "kernels_rowwise.cu", "ccs_to_ell_col": "kernels_rowwise.cu",
    "crs_to_coo_row": "kernels_rowwise.cu", "ccs_to_coo_col": "kernels_rowwise.cu",
    "batch_apply": "kernels_batch.cu",
}


def csrc_digest(kernel: str = None) -> str:
    """Hash of the device code a kernel's DRAM traffic depends on: its own
    kernel file (spmv_* kernels: kernels_spmv.cu) and the device headers;
    every kernel file when the kernel is not listed."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2407_00019_gb300", "csrc")
    own = KERNEL_FILES.get(kernel, "kernels_spmv.cu" if (kernel or "").startswith("spmv_") else None)
    for f in sorted(os.listdir(d)):
        if f.endswith(".cuh") or (f.startswith("kernels_") and (own is None or f == own)):
            with open(os.path.join(d, f), "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


def stored_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from a committed ncu summary, if it matches the
    current device code of that kernel."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(p) as f:
            rows = json.load(f)
    except (OSError, ValueError):
        return None
    for r in rows:
        if r.get("kernel") == kernel and r.get("workload") == workload and r.get("csrc") == csrc_digest(kernel):
            return r.get("bytes_per_launch")
    return None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-other-configs", action="store_true",
                    help="default workload: skip the child runs of the other configurations")
    ap.add_argument("--requests", type=int, default=None, help="serving: measured requests per rate")
    ap.add_argument("--rate", type=float, default=None, help="serving: offered requests per second")
    ap.add_argument("--no-loop", action="store_true", help="batches: skip the per-matrix loop comparison")
    ap.add_argument("--sequential", action="store_true",
                    help="run the row-wise and column-wise pipelines of a step one after the other on one stream")
    ap.add_argument("--phase1", choices=["auto", "scatter", "kslot", "rk", "grp", "sym"], default="auto",
                    help="force one Phase I path through the library's schedule hint (profiling)")
    ap.add_argument("--dstar", type=float, default=None,
                    help="use this D* instead of the off-line calibration (profiling runs)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    w = dict(WORKLOADS[args.workload])
    if args.rate is not None:
        w["rate"] = args.rate
    if w["kind"] == "batch":
        run_batch(args, w)
        return
    if w["kind"] == "serve":
        run_serve(args, w)
        return
    if args.impl == "reference":
        run_reference(args, w)
        return

    import torch
    import torch.distributed as dist
    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    import paper_2407_00019_gb300 as L
    L.load_library()
    if args.phase1 != "auto":
        L.spmv_set_hint(L.SPMV_HINT_PHASE1, {"scatter": L.SPMV_PHASE1_COUNT, "kslot": L.SPMV_PHASE1_KSLOT,
                                             "rk": L.SPMV_PHASE1_ROWPOS, "grp": L.SPMV_PHASE1_GROUPED,
                                             "sym": L.SPMV_PHASE1_SYMMETRIC}[args.phase1])

    H, xh = make_matrix(w, rank)
    A = L.Crs.from_host(H)
    x = torch.from_numpy(xh).to(device)
    fmts = ["crs", "coo_row", "ell_row", "coo_col", "ell_col"]
    ys = {f: torch.empty(H.n_rows, dtype=torch.float64, device=device) for f in fmts}
    if args.dstar is None:
        dstar, dstar_src = committed_dstar(L, torch, "prefix")
    else:
        dstar, dstar_src = args.dstar, "--dstar"
    step = Step(L, A, x, ys, dstar, w["cap"], concurrent=not args.sequential)
    seq_step = Step(L, A, x, ys, dstar, w["cap"])
    stats = L.spmv_analyze(A)
    W = stats["W"]
    ccs = L.spmv_transform(A, L.SPMV_CRS, L.SPMV_COLWISE)
    ell_c = L.spmv_transform_from(ccs, L.SPMV_ELL)
    Wc = ell_c.describe()["width"]
    ell_c.close(); ccs.close()
    bm = byte_model(H.n_rows, H.n_cols, H.nnz, W, Wc)
    if w["cap"] and stats["ell_bytes"] > w["cap"]:
        bm.pop("crs_to_ell_row"); bm.pop("spmv_ell_row")
    step_bytes = float(sum(bm.values()))

    # reserve the step's working memory in the library's pool up front (a
    # step owns ~6x the CRS bytes while its pipelines overlap)
    free_b, _ = torch.cuda.mem_get_info()
    L.spmv_reserve(min(free_b // 4, 8 * (12 * H.nnz + 4 * H.n_rows)))
    clocks = ClockSampler(local)
    clocks.start()
    for _ in range(args.warmup):
        step.run()
    stream = torch.cuda.current_stream()
    # inputs smaller than L2 (the 64x64 Laplacian): a write of twice the L2
    # size before each timed step (outside its events) makes every step cold;
    # warm steps are timed separately
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device=device) if step_bytes < L2_BYTES else None
    barrier_sync(torch)
    launches0 = L.spmv_launch_count()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev_in = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier_sync(torch)
    h0 = time.perf_counter()
    ev[0].record(stream)
    for i in range(args.steps):
        if flush is not None:
            flush.fill_(i)
            ev_in[i].record(stream)
        step.run()
        ev[i + 1].record(stream)
    barrier_sync(torch)
    clocks.mark(h0, time.perf_counter())
    launches = L.spmv_launch_count() - launches0
    warm = None
    if flush is not None:
        ew = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ew[0].record(stream)
        for _ in range(args.steps):
            step.run()
        ew[1].record(stream)
        barrier_sync(torch)
        warm_ms = ew[0].elapsed_time(ew[1]) / args.steps
        warm = {"ms_per_step": warm_ms, "latency_us": 1e3 * warm_ms, "GB/s": step_bytes / (warm_ms * 1e-3) / 1e9,
                "note": "steps back to back, inputs resident in L2"}
    clk = clocks.stop()
    # per-kernel device times from steps run one kernel at a time (in the
    # timed steps the two pipelines overlap, which stretches each launch)
    L.spmv_profile_read(reset=True)
    L.spmv_profile_enable(True)
    for _ in range(PROFILE_STEPS):
        seq_step.run()
    torch.cuda.synchronize()
    L.spmv_profile_enable(False)
    prof = L.spmv_profile_read(reset=True)
    if flush is None:
        per_step = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
        total_ms = ev[0].elapsed_time(ev[-1])
    else:
        per_step = [ev_in[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
        total_ms = sum(per_step)
    t_max, bytes_all = reduce_max_sum(torch, total_ms, step_bytes * args.steps, device)
    value = bytes_all / (t_max * 1e-3) / 1e9

    peak, peak_kind = measured_hbm_peak()
    per_kernel = {}
    for name, (n, ms) in prof.items():
        kb = kernel_bytes(name, bm, H.n_rows, H.n_cols, H.nnz)
        avg = ms / n
        per_kernel[name] = {"launches": n, "ms_per_launch": avg, "share": None,
                            "GB/s": (kb / (avg * 1e-3) / 1e9) if kb else None}
    ksum = sum(ms for _, ms in prof.values()) or 1.0
    for name, (n, ms) in prof.items():
        per_kernel[name]["share"] = ms / ksum
    top = max(prof.items(), key=lambda kv: kv[1][1])[0]
    top_b = kernel_bytes(top, bm, H.n_rows, H.n_cols, H.nnz)
    top_ms = prof[top][1] / prof[top][0]
    achieved = top_b / (top_ms * 1e-3) / 1e9 if top_b else None
    roofline = {"kernel": top, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None, "peak_source": peak_kind,
                "traffic": stored_traffic(top, args.workload),
                "algorithmic_bytes_per_launch": top_b}

    # Per-format product rates in the steady state of an iterative solver: each
    # format's handle built once, its product run back to back (3 warm-up
    # runs, PRODUCT_REPS timed), the device time of the product's kernels from
    # the library's events (a product on uneven rows may be several launches).
    # These are the t_crs and t_ell of Eqs. 1-2; the per-kernel table above
    # times single launches inside the sequential steps instead.
    prods = steady_products(L, torch, A, x, H.n_rows, w["cap"], "spmv_ell_row" in bm)

    def fmt_rate(name, model):
        if name not in prods or model not in bm:
            return None
        ms = sum(t for _, t in prods[name].values()) / PRODUCT_REPS
        g = bm[model] / (ms * 1e-3) / 1e9
        return {"GB/s": g, "pct_hbm": 100.0 * g / peak, "ms": ms, "kernels": sorted(prods[name]),
                "runs": f"mean of {PRODUCT_REPS} back-to-back products after 3 warm-up runs"}
    per_format = {"crs": fmt_rate("crs", "spmv_crs"), "coo_row": fmt_rate("coo_row", "spmv_coo_row"),
                  "ell_row": fmt_rate("ell_row", "spmv_ell_row"), "coo_col": fmt_rate("coo_col", "spmv_coo_col"),
                  "ell_col": fmt_rate("ell_col", "spmv_ell_col")}
    # the ceiling of the column-wise products: their FP64 atomic adds alone
    # (coalesced, the best case on banded matrices), one per entry (COO-Column)
    # or per slot (ELL-Column)
    for fmt, adds in (("coo_col", H.nnz), ("ell_col", round32(H.n_cols) * Wc)):
        if per_format.get(fmt) and adds > 0:
            t_at = L.spmv_measure_atomics(H.n_rows, adds, reps=10)
            per_format[fmt]["atomics_ceiling_ms"] = t_at
            per_format[fmt]["frac_of_atomics_ceiling"] = t_at / per_format[fmt]["ms"]
    # CRS -> ELL cost in CRS-SpMV units: standalone build, and the fused
    # build + first SpMV counted beyond the SpMV it replaces
    t_crs = per_format["crs"]["ms"] if per_format["crs"] else None
    cost = None
    if t_crs and "crs_to_ell_row" in per_kernel:
        # the ELL-Row build's own pointer pass (the longest row), not the AT analysis
        t_an = per_kernel.get("row_width", per_kernel["analyze"])["ms_per_launch"]
        t_tr = per_kernel["crs_to_ell_row"]["ms_per_launch"]
        L.spmv_profile_enable(True)
        yf = torch.empty(H.n_rows, dtype=torch.float64, device=device)
        for _ in range(5):
            L.spmv_transform_apply(A, x, yf).close()
        torch.cuda.synchronize()
        L.spmv_profile_enable(False)
        pf = L.spmv_profile_read(reset=True)
        t_f = pf["crs_to_ell_row_fused_spmv"][1] / pf["crs_to_ell_row_fused_spmv"][0]
        cost = {"standalone": (t_an + t_tr) / t_crs, "fused_marginal": (t_an + t_f - t_crs) / t_crs,
                "t_crs_ms": t_crs, "t_trans_ms": t_an + t_tr, "t_fused_ms": t_an + t_f,
                "byte_floor_standalone": bm["crs_to_ell_row"] / bm["spmv_crs"]}

    e2e = None
    if not args.no_e2e:
        # Each step copies its own CRS arrays and x from pinned host memory and
        # reads its y back; step i+1's upload runs on a copy stream while step i
        # computes (two device buffers, ordered by events).
        pin = [torch.from_numpy(a).pin_memory() for a in (H.irp, H.icol, H.val)]
        xpin = torch.from_numpy(xh).pin_memory()
        yhost = torch.empty(H.n_rows, dtype=torch.float64).pin_memory()
        h2d = sum(t.numel() * t.element_size() for t in pin) + xpin.numel() * 8
        d2h = yhost.numel() * 8
        bufs = []
        for _ in range(2):
            irp_d, icol_d, val_d = (torch.empty_like(t, device=device) for t in pin)
            x_d = torch.empty_like(xpin, device=device)
            bufs.append((L.Crs(H.n_rows, H.n_cols, irp_d, icol_d, val_d), x_d))
        copy_stream = torch.cuda.Stream(device=device)
        estep = Step(L, A, x, ys, dstar, w["cap"], concurrent=not args.sequential)
        loaded = [torch.cuda.Event() for _ in range(2)]
        consumed = [torch.cuda.Event() for _ in range(2)]

        def upload(b):
            A_b, x_b = bufs[b]
            with torch.cuda.stream(copy_stream):
                copy_stream.wait_event(consumed[b])
                for dst, src in zip((A_b.irp, A_b.icol, A_b.val), pin):
                    dst.copy_(src, non_blocking=True)
                x_b.copy_(xpin, non_blocking=True)
                loaded[b].record(copy_stream)

        for b in range(2):
            consumed[b].record(stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier_sync(torch)
        e0.record(stream)
        upload(0)
        for i in range(args.steps):
            b = i % 2
            if i + 1 < args.steps:
                upload(1 - b)
            stream.wait_event(loaded[b])
            A_b, x_b = bufs[b]
            estep.A, estep.x = A_b, x_b
            estep.run()
            yhost.copy_(ys["ell_row" if estep.chosen == "ELL-Row" else "crs"], non_blocking=True)
            consumed[b].record(stream)
        e1.record(stream)
        barrier_sync(torch)
        et_max, eb_all = reduce_max_sum(torch, e0.elapsed_time(e1), step_bytes * args.steps, device)
        e2e = {"value": eb_all / (et_max * 1e-3) / 1e9, "unit": "GB/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": et_max / args.steps,
               "overlap": "upload of step i+1 on a copy stream during step i"}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(H, xh, cap=w["cap"])

    if rank == 0:
        srt = sorted(per_step)
        p99 = srt[min(len(srt) - 1, int(math.ceil(0.99 * len(srt))) - 1)]
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {**workload_config(args.workload, w, H, W, Wc, stats["dmat"], world),
                       "step_bytes": step_bytes,
                       "l2": ("inputs larger than L2 (CRS %.0f MB vs 129 MB L2); no flush" % (
                           (12 * H.nnz + 4 * H.n_rows) / 1e6)) if flush is None else
                             ("inputs smaller than L2 (step %.2f MB): L2 flushed by a %d MB write before each "
                              "timed step, outside its events; 'warm' has back-to-back steps" % (
                                  step_bytes / 1e6, 2 * L2_BYTES // 2 ** 20)),
                       "launches_before_timed": int(launches0),
                       "step_schedule": "sequential" if args.sequential else
                       "independent pipelines (AT+CRS+ELL-Row, COO-Row, Phase I then Phase II | CCS->ELL-Col) on four streams",
                       "per_kernel": f"{PROFILE_STEPS} sequential steps after the timed region",
                       "per_format": f"each product {PRODUCT_REPS} times back to back after 3 warm-up runs"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clk,
            "p50_ms": statistics.median(per_step), "p99_ms": p99, "per_step_ms": per_step,
            "latency_us": {"cold": 1e3 * t_max / args.steps, "warm": warm["latency_us"] if warm else None},
            "warm": warm,
            "per_format": per_format,
            "crs_to_ell_cost": cost,
            "at": {"dstar": dstar if math.isfinite(dstar) else "inf", "chosen": step.chosen,
                   "dstar_source": dstar_src},
            "per_kernel": per_kernel,
        }
        if world == 1 and args.workload == DEFAULT_WORKLOAD and not args.no_other_configs:
            line["other_configs"] = other_configs()
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# The other configurations of the benchmark, each as a child run of this
# script after the headline measurement (bounded in time), so that one default
# run also carries their figures: the 64x64 Laplacian (latency), the 4e6-row
# power law (the AT under the 40 GB cap), the 10,000-matrix batch and a short
# two-arm serving run.
OTHER_CONFIGS = [
    ("laplace2d_64", ["--steps", "20", "--warmup", "5"], 240),
    ("powerlaw_4m", ["--steps", "5", "--warmup", "3"], 420),
    ("batch_10k", ["--steps", "10", "--warmup", "3", "--no-loop"], 420),
    ("serve_300", ["--rate", "750", "--requests", "600"], 420),
]


def _summary(name: str, d: dict) -> dict:
    out = {"value": d.get("value"), "unit": d.get("unit"), "ms_per_step": d.get("ms_per_step")}
    if d.get("roofline"):
        r = d["roofline"]
        out["roofline"] = {k: r.get(k) for k in ("kernel", "frac", "achieved", "peak")}
    if name == "laplace2d_64":
        out["latency_us"] = d.get("latency_us")
    if name == "powerlaw_4m":
        out["at"] = d.get("at")
        out["per_format"] = {k: (v and {"GB/s": v["GB/s"], "pct_hbm": v["pct_hbm"]}) for k, v in
                             (d.get("per_format") or {}).items()}
    if name == "batch_10k":
        b = d.get("batch") or {}
        out["batch"] = {k: b.get(k) for k in ("create_ms", "formats", "schedule_table", "graph_build")}
    if name == "serve_300":
        out["arms"] = {a: [{k: r[k] for k in ("offered_req_per_s", "served_req_per_s", "GB/s", "p50_ms", "p99_ms")}
                           for r in rows] for a, rows in (d.get("arms") or {}).items()}
        out["cache"] = d.get("cache")
    return out


def other_configs() -> dict:
    res = {}
    for name, extra, limit in OTHER_CONFIGS:
        cmd = [sys.executable, os.path.abspath(__file__), "--workload", name, "--no-e2e", "--no-cpu-baseline"] + extra
        t0 = time.perf_counter()
        try:
            r = subprocess.run(cmd, capture_output=True, text=True, timeout=limit)
            lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
            if r.returncode != 0 or not lines:
                res[name] = {"error": f"exit {r.returncode}: {r.stderr.strip().splitlines()[-1:] or ''}"}
            else:
                res[name] = _summary(name, json.loads(lines[-1]))
        except subprocess.TimeoutExpired:
            res[name] = {"error": f"did not finish within {limit} s"}
        res[name]["wall_s"] = round(time.perf_counter() - t0, 1)
    return res


if __name__ == "__main__":
    main()
