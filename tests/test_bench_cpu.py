"""Host-side checks of the benchmark's accounting (no GPU): the byte models
behind every reported rate, the per-kernel byte table against the kernels the
library times, and the CPU oracle leg under a memory cap."""

import importlib.util
import os
import re

import numpy as np
import pytest

import spmv_synth as synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_byte_model_of_the_stencil_workload(bench):
    """The 27-point stencil on 128^3: n = 2,097,152, nnz = (3*128 - 2)^3,
    W = 27. The models count x and y once: CRS SpMV 12 nnz + 4(n+1) + 16n,
    ELL-Row SpMV 12 n W + 16n (n is a multiple of 32, so ld = n),
    CRS->ELL 12 nnz + 4(n+1) + 12 n W."""
    n, nnz, W = 128 ** 3, (3 * 128 - 2) ** 3, 27
    bm = bench.byte_model(n, n, nnz, W, W)
    assert nnz == 55_742_968
    assert bm["spmv_crs"] == 12 * nnz + 4 * (n + 1) + 16 * n == 710_858_660  # 710.9 MB
    assert bm["spmv_ell_row"] == 12 * n * W + 16 * n == 713_031_680  # 713.0 MB
    assert bm["crs_to_ell_row"] == 12 * nnz + 4 * (n + 1) + 12 * n * W == 1_356_781_476  # 1356.8 MB
    assert abs(bm["crs_to_ell_row"] / bm["spmv_crs"] - 1.9087) < 1e-4


def test_ell_width_rounds_the_leading_dimension(bench):
    """ELL keeps each slot column 32-line aligned: ld = round-up(n, 32)."""
    bm = bench.byte_model(33, 40, 100, 5, 7)
    assert bm["spmv_ell_row"] == 12 * 64 * 5 + 8 * 40 + 8 * 33
    assert bm["spmv_ell_col"] == 12 * 64 * 7 + 8 * 40 + 8 * 33


def _timed_kernel_names():
    names = set()
    d = os.path.join(ROOT, "paper_2407_00019_gb300", "csrc")
    for f in os.listdir(d):
        if not f.endswith(".cu"):
            continue
        src = open(os.path.join(d, f)).read()
        names |= set(re.findall(r'KernelScope ks\("([a-z0-9_]+)"', src))
        names |= set(re.findall(r'"((?:crs|ccs)_to_(?:coo|ell)_(?:row|col))"', src))
        names |= set(re.findall(r'"(coo_(?:row|col)_tile_bounds)"', src))
    return names


def test_every_step_kernel_has_a_byte_model(bench):
    """Each kernel the library times in the single-matrix steps has its
    algorithmic or design bytes in the bench's table, or is one of the few
    whose traffic depends on the data (long-column sorts, overflow placement)
    or that belong to other workloads (batches)."""
    names = _timed_kernel_names()
    assert {"col_claim_rk", "col_fixup_rk", "spmv_crs_rows_p", "crs_to_coo_row"} <= names
    bm = bench.byte_model(1000, 1000, 20000, 30, 40)
    unmodelled = {"col_fixup_block", "col_fixup_long_rv", "col_overflow_rk", "spmv_coo_row_carry"}
    for name in sorted(names):
        if name.startswith("batch_") or name in unmodelled:
            continue
        probe = name + "4" if name.endswith("_p") or name.endswith("_s") or name.endswith("_v") else name
        assert bench.kernel_bytes(probe, bm, 1000, 1000, 20000) is not None, name


def test_oracle_leg_leaves_out_ell_beyond_the_cap(bench):
    """As the GPU step does under the workload's cap, the oracle leg leaves out
    ELL-Row (and its bytes) when the sample's ELL would not fit the cap."""
    H = synth.power_law(3000, kmax=2000, seed=3)
    xh = synth.vector_pm1(H.n_cols, seed=4)
    t_all = bench.oracle_step(H, xh, 0)
    assert t_all["_ell"] and "spmv_ell_row" in t_all
    cap = 12 * H.n_rows * 10  # far below 12 n W for rows up to 2000 entries
    t_cap = bench.oracle_step(H, xh, cap)
    assert not t_cap["_ell"] and "spmv_ell_row" not in t_cap and "crs_to_ell_row" not in t_cap
    b_all = bench.oracle_bytes(H, t_all["_W"], t_all["_Wc"], True)
    b_cap = bench.oracle_bytes(H, t_cap["_W"], t_cap["_Wc"], False)
    bm = bench.byte_model(H.n_rows, H.n_cols, H.nnz, t_all["_W"], t_all["_Wc"])
    assert np.isclose(b_all - b_cap, bm["crs_to_ell_row"] + bm["spmv_ell_row"])


def test_reference_arm_runs_the_oracle_on_the_native_workload_keys():
    """`bench.py --impl reference` (the oracle on the host cores) prints one
    line whose workload keys are those of the native arm, here with the 64x64
    Laplacian's closed forms (n 4096, nnz 20224, W 5, D_mat 0.0498355)."""
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "laplace2d_64", "--steps", "2", "--warmup", "3"], capture_output=True, text=True,
                       timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    c = d["config"]
    assert d["impl"] == "reference" and d["value"] > 0 and d["gpu_launches"] == 0
    assert (c["workload"], c["n"], c["nnz"], c["W"], c["W_col"]) == ("laplace2d_64", 4096, 20224, 5, 5)
    assert abs(c["D_mat"] - 0.0498355) < 1e-7
    assert c["step_bytes"] == 3675168.0
    assert d["cpu_baseline"]["value"] == d["value"] and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_workload_config_leaves_out_ell_beyond_the_cap(bench):
    """Under a cap the step builds no ELL-Row, and its step bytes say so."""
    H = synth.power_law(3000, kmax=2000, seed=3)
    W = int(np.diff(H.irp).max())
    Wc = int(np.bincount(H.icol, minlength=H.n_cols).max())
    bm = bench.byte_model(H.n_rows, H.n_cols, H.nnz, W, Wc)
    free = bench.workload_config("t", {"cap": 0, "desc": ""}, H, W, Wc, 1.0, 1)
    capped = bench.workload_config("t", {"cap": 12 * H.n_rows * 10, "desc": ""}, H, W, Wc, 1.0, 1)
    assert free["step_bytes"] == float(sum(bm.values()))
    assert free["step_bytes"] - capped["step_bytes"] == bm["crs_to_ell_row"] + bm["spmv_ell_row"]


def test_stored_traffic_entries_cite_committed_profiles(bench):
    """Every stored DRAM figure names the ncu summary it comes from, that
    summary is committed, and the figure is within a factor of two of the
    kernel's byte model at the workload's size (far above would mean re-reads,
    far below a capture of the wrong launch)."""
    import json
    with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as f:
        entries = json.load(f)
    sizes = {"stencil27_128": (128 ** 3, 128 ** 3, (3 * 128 - 2) ** 3, 27, 27)}
    assert entries
    for e in entries:
        assert os.path.exists(os.path.join(ROOT, "profiles", e["source"])), e
        assert len(e["csrc"]) == 16 and e["bytes_per_launch"] > 0
        if e["workload"] in sizes:
            n, m, nnz, W, Wc = sizes[e["workload"]]
            model = bench.kernel_bytes(e["kernel"], bench.byte_model(n, m, nnz, W, Wc), n, m, nnz)
            assert model and 0.5 < e["bytes_per_launch"] / model < 2.0, (e["kernel"], e["bytes_per_launch"], model)


def test_cpu_baseline_times_one_thread_and_every_host_core():
    """The CPU baseline reports the multi-core oracle (cores = its threads)
    with the single-thread figure beside it, and names the host CPU."""
    import bench
    import oracle
    import spmv_synth as synth
    H = synth.laplacian_2d_5pt(64)
    xh = synth.vector_pm1(H.n_cols, seed=0)
    cb = bench.cpu_baseline(H, xh, budget_s=0.2)
    assert cb["kind"] == "oracle" and cb["unit"] == "GB/s" and cb["value"] > 0
    assert cb["cores"] == oracle.omp_threads() and cb["nproc"] >= 1 and cb["cpu_model"]
    assert cb["single_thread"]["cores"] == 1 and cb["single_thread"]["value"] > 0
    assert "rows 0..1024 of 4096" in cb["sample"]
