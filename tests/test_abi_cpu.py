"""The C-ABI library builds for sm_103a, loads without a GPU, exports every
function include/spmvat.h declares, and its host-only entry points agree
with the oracle and the paper's worked example."""

import math
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2407_00019_gb300 import _build
    _build.build()
    import paper_2407_00019_gb300 as L
    L.load_library()
    return L


def declared_functions():
    with open(os.path.join(ROOT, "include", "spmvat.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w\s\*]*?\b(spmv_\w+)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if not n.endswith("_fn")))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("spmv_analyze", "spmv_transform", "spmv_apply", "spmv_autotune"):
        assert must in names
    assert len(names) >= 20


def test_library_exports_every_declared_symbol(lib):
    L = lib.load_library()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert missing == []


def test_host_only_entry_points(lib):
    assert lib.spmv_version() == 1
    assert lib.spmv_status_string(5) == "SPMV_ERR_TIMEOUT"
    assert lib.spmv_status_string(0) == "SPMV_OK"
    # ELL bytes: leading dimension rounded up to 32 lines, 8 + 4 bytes per slot
    assert lib.spmv_ell_bytes(4096, 5) == 4096 * 5 * 12
    assert lib.spmv_ell_bytes(33, 2) == 64 * 2 * 12


def test_r_ell_matches_oracle_and_worked_example(lib):
    # Sec. 2.2: 10x speedup and a transformation of 10 CRS SpMVs -> R_ell = 1
    assert math.isclose(lib.spmv_r_ell(1.0, 0.1, 10.0), 1.0, rel_tol=1e-15)
    rng = np.random.default_rng(0)
    for t in rng.uniform(0.01, 10.0, size=(50, 3)):
        assert lib.spmv_r_ell(*t) == oracle.r_ell(*t)


def test_dstar_rule_matches_oracle(lib):
    rng = np.random.default_rng(1)
    for _ in range(200):
        m = int(rng.integers(0, 12))
        d = np.round(rng.uniform(0, 3, m), 2)  # ties happen
        r = rng.uniform(0.3, 3.0, m)
        for rule in (0, 1):
            assert lib.spmv_dstar_from_points(d, r, 1.0, rule) == oracle.dstar_from_points(d, r, 1.0, rule)
    assert lib.spmv_dstar_from_points([0.02, 0.1, 0.5, 0.3, 3.1], [5, 2, 0.8, 1.5, 2], 1.0, 0) == 0.5


def test_argument_errors_need_no_device(lib):
    import ctypes
    L = lib.load_library()
    h = ctypes.c_void_p()
    assert L.spmv_transform(None, 0, 0, 0, ctypes.byref(h), None) == 1
    assert L.spmv_analyze(None, None, None) == 1
    crs = lib._CrsT(0, 5, 0, 1, 0, 0)  # n_rows = 0
    assert L.spmv_transform(ctypes.byref(crs), 0, 0, 0, ctypes.byref(h), None) == 1
    crs = lib._CrsT(5, 5, 3, 16, 0, 0)  # nnz > 0 without ICOL/VAL
    assert L.spmv_transform(ctypes.byref(crs), 0, 0, 0, ctypes.byref(h), None) == 1
    crs = lib._CrsT(5, 5, 3, 16, 16, 16)
    assert L.spmv_transform(ctypes.byref(crs), 7, 0, 0, ctypes.byref(h), None) == 1  # bad format
    assert L.spmv_apply(None, None, None, None) == 1
    assert L.spmv_set_allocator(ctypes.c_void_p(1), None, None) == 1
    assert L.spmv_dstar_from_points(-1, None, None, 1.0, 0, None) == 1
    assert L.spmv_debug_scan_timeout(0, 1, None, None) == 1


def test_binding_fails_loudly_without_the_library(tmp_path):
    """A copy of the Python binding without libspmvat.so raises at load: the
    product has no CPU path to fall back on."""
    import shutil
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    pkg = tmp_path / "paper_2407_00019_gb300"
    pkg.mkdir()
    shutil.copy(os.path.join(root, "paper_2407_00019_gb300", "__init__.py"), pkg / "__init__.py")
    code = ("import paper_2407_00019_gb300 as L\n"
            "try:\n    L.load_library()\nexcept ImportError as e:\n    print('raised', e)\n"
            "else:\n    print('loaded')\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=str(tmp_path), capture_output=True, text=True,
                       timeout=300, env=dict(os.environ, PYTHONPATH=str(tmp_path)))
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.startswith("raised") and "libspmvat.so is missing" in r.stdout
