"""CPU oracle (FP64, plain serial loops) for the sparse-format method.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg use this package; the CUDA library and its Python binding
never import it. The arithmetic lives in ``spmv_oracle.c`` (plain C, built
with ``-O2 -ffp-contract=off``); this file only builds that shared object and
passes numpy arrays to it. ``spmv_oracle_omp.c`` is a multi-core build of the
CRS and ELL-Row products and the Phase I count and pointers, for timing the
oracle on all host cores; the tests check it bit for bit against the serial
functions.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spmv_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_SRC_OMP = os.path.join(_HERE, "spmv_oracle_omp.c")
_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_dptr = ctypes.POINTER(ctypes.c_double)
_iptr = ctypes.POINTER(ctypes.c_int32)


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source if missing or stale."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def build_omp(force: bool = False) -> str:
    """Compile liboracle_omp.so (gcc -fopenmp) if missing or stale."""
    if force or not os.path.exists(_LIB_OMP) or os.path.getmtime(_LIB_OMP) < os.path.getmtime(_SRC_OMP):
        tmp = _LIB_OMP + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC_OMP])
        os.replace(tmp, _LIB_OMP)
    return _LIB_OMP


def _load_omp():
    global _lib_omp
    with _lock:
        if _lib_omp is None:
            L = ctypes.CDLL(build_omp())
            L.orc_omp_threads.restype = ctypes.c_int32
            L.orc_omp_spmv_crs.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _f64p, _f64p, ctypes.c_int32]
            L.orc_omp_spmv_ell_row.argtypes = [ctypes.c_int32, ctypes.c_int32, _f64p, _i32p, _f64p, _f64p,
                                               ctypes.c_int32]
            L.orc_omp_crs_to_ccs.argtypes = [ctypes.c_int32, ctypes.c_int32, _i32p, _i32p, _f64p, _i32p, _i32p,
                                             _f64p, ctypes.c_int32]
            L.orc_omp_crs_to_ccs.restype = ctypes.c_int32
            _lib_omp = L
    return _lib_omp


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # SPMVAT_ORACLE_LIB: another build of this file's C source (the
            # planted-mistake tests point it at a mutated copy)
            path = os.environ.get("SPMVAT_ORACLE_LIB") or build()
            L = ctypes.CDLL(path)
            L.orc_analyze.argtypes = [ctypes.c_int32, _i32p, _dptr, _dptr, _dptr, _iptr]
            L.orc_crs_to_coo_row.argtypes = [ctypes.c_int32, _i32p, _i32p]
            L.orc_lines_to_ell.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, ctypes.c_int32, _f64p, _i32p]
            L.orc_crs_to_ccs.argtypes = [ctypes.c_int32, ctypes.c_int32, _i32p, _i32p, _f64p,
                                         _i32p, _i32p, _f64p, _i32p]
            L.orc_ccs_to_coo_col.argtypes = [ctypes.c_int32, _i32p, _i32p]
            L.orc_spmv_crs.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _f64p, _f64p]
            L.orc_spmv_coo.argtypes = [ctypes.c_int32, ctypes.c_int64, _i32p, _i32p, _f64p, _f64p, _f64p]
            L.orc_spmv_ell_row.argtypes = [ctypes.c_int32, ctypes.c_int32, _f64p, _i32p, _f64p, _f64p]
            L.orc_spmv_ell_col.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _f64p, _i32p,
                                           _f64p, _f64p]
            L.orc_spmv_ccs.argtypes = [ctypes.c_int32, ctypes.c_int32, _i32p, _i32p, _f64p, _f64p, _f64p]
            L.orc_spmv_ref.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p]
            L.orc_r_ell.argtypes = [ctypes.c_double] * 3
            L.orc_r_ell.restype = ctypes.c_double
            L.orc_dstar_from_points.argtypes = [ctypes.c_int32, _f64p, _f64p, ctypes.c_double, ctypes.c_int32]
            L.orc_dstar_from_points.restype = ctypes.c_double
            _lib = L
    return _lib


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def analyze(n_rows, irp):
    """Eq. (4): returns dict(mu, sigma, dmat, W)."""
    L = _load()
    mu, sg, dm = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    w = ctypes.c_int32()
    L.orc_analyze(int(n_rows), _i32(irp), ctypes.byref(mu), ctypes.byref(sg), ctypes.byref(dm), ctypes.byref(w))
    return {"mu": mu.value, "sigma": sg.value, "dmat": dm.value, "W": w.value}


def crs_to_coo_row(n_rows, irp):
    """Sec. 2.1: IROW for each CRS entry."""
    irp = _i32(irp)
    out = np.empty(int(irp[-1]), dtype=np.int32)
    _load().orc_crs_to_coo_row(int(n_rows), irp, out)
    return out


def lines_to_ell(n_lines, ptr, idx, val, width=None):
    """Sec. 2.1 / Fig. 3: (eval, eidx, width), slot k of line i at k*n_lines+i."""
    ptr = _i32(ptr)
    if width is None:
        width = int(np.diff(ptr).max()) if n_lines > 0 else 0
    ev = np.empty(int(width) * int(n_lines), dtype=np.float64)
    ei = np.empty(int(width) * int(n_lines), dtype=np.int32)
    _load().orc_lines_to_ell(int(n_lines), ptr, _i32(idx), _f64(val), int(width), ev, ei)
    return ev, ei, int(width)


def crs_to_ell_row(n_rows, irp, icol, val, width=None):
    return lines_to_ell(n_rows, irp, icol, val, width)


def crs_to_ccs(n_rows, n_cols, irp, icol, val):
    """Sec. 2.1 Phase I: (irp_t, icol_t = rows, val_t, nc)."""
    irp = _i32(irp)
    nnz = int(irp[-1])
    irp_t = np.empty(int(n_cols) + 1, dtype=np.int32)
    icol_t = np.empty(nnz, dtype=np.int32)
    val_t = np.empty(nnz, dtype=np.float64)
    nc = np.empty(max(int(n_cols), 1), dtype=np.int32)
    _load().orc_crs_to_ccs(int(n_rows), int(n_cols), irp, _i32(icol), _f64(val), irp_t, icol_t, val_t, nc)
    return irp_t, icol_t, val_t, nc[:int(n_cols)]


def ccs_to_coo_col(n_cols, irp_t):
    """Sec. 2.1 Phase II: column of each CCS entry."""
    irp_t = _i32(irp_t)
    out = np.empty(int(irp_t[-1]), dtype=np.int32)
    _load().orc_ccs_to_coo_col(int(n_cols), irp_t, out)
    return out


def ccs_to_ell_col(n_cols, irp_t, icol_t, val_t, width=None):
    return lines_to_ell(n_cols, irp_t, icol_t, val_t, width)


def spmv_crs(n_rows, irp, icol, val, x):
    y = np.empty(int(n_rows), dtype=np.float64)
    _load().orc_spmv_crs(int(n_rows), _i32(irp), _i32(icol), _f64(val), _f64(x), y)
    return y


def spmv_coo(n_rows, row, col, val, x):
    y = np.empty(int(n_rows), dtype=np.float64)
    row = _i32(row)
    _load().orc_spmv_coo(int(n_rows), int(row.size), row, _i32(col), _f64(val), _f64(x), y)
    return y


def spmv_ell_row(n_rows, width, eval_, ecol, x):
    y = np.empty(int(n_rows), dtype=np.float64)
    _load().orc_spmv_ell_row(int(n_rows), int(width), _f64(eval_), _i32(ecol), _f64(x), y)
    return y


def spmv_ell_col(n_rows, n_cols, width, eval_, erow, x):
    y = np.empty(int(n_rows), dtype=np.float64)
    _load().orc_spmv_ell_col(int(n_rows), int(n_cols), int(width), _f64(eval_), _i32(erow), _f64(x), y)
    return y


def spmv_ccs(n_rows, n_cols, irp_t, icol_t, val_t, x):
    y = np.empty(int(n_rows), dtype=np.float64)
    _load().orc_spmv_ccs(int(n_rows), int(n_cols), _i32(irp_t), _i32(icol_t), _f64(val_t), _f64(x), y)
    return y


def spmv_ref(n_rows, irp, icol, val, x):
    """Compensated reference: (y_ref, s_ref) with s_ref = sum |a_ij x_j|."""
    y = np.empty(int(n_rows), dtype=np.float64)
    s = np.empty(int(n_rows), dtype=np.float64)
    _load().orc_spmv_ref(int(n_rows), _i32(irp), _i32(icol), _f64(val), _f64(x), y, s)
    return y, s


def r_ell(t_crs, t_ell, t_trans):
    """Eqs. (1)-(3) with Eq. (2) read as t_trans / t_crs."""
    return _load().orc_r_ell(float(t_crs), float(t_ell), float(t_trans))


def dstar_from_points(dmat, rell, c=1.0, rule=0):
    """Off-line step (4) of Sec. 2.2; rule 0 = prefix, 1 = max-pass."""
    d, r = _f64(dmat), _f64(rell)
    return _load().orc_dstar_from_points(int(d.size), d, r, float(c), int(rule))


# ---- multi-core builds (same bits as the serial functions above) ----------
def omp_threads() -> int:
    """Threads the multi-core oracle uses by default (OpenMP's maximum)."""
    return int(_load_omp().orc_omp_threads())


def spmv_crs_omp(n_rows, irp, icol, val, x, nthreads=0):
    y = np.empty(int(n_rows), dtype=np.float64)
    _load_omp().orc_omp_spmv_crs(int(n_rows), _i32(irp), _i32(icol), _f64(val), _f64(x), y, int(nthreads))
    return y


def spmv_ell_row_omp(n_rows, width, eval_, ecol, x, nthreads=0):
    y = np.empty(int(n_rows), dtype=np.float64)
    _load_omp().orc_omp_spmv_ell_row(int(n_rows), int(width), _f64(eval_), _i32(ecol), _f64(x), y, int(nthreads))
    return y


def crs_to_ccs_omp(n_rows, n_cols, irp, icol, val, nthreads=0):
    """Phase I with the count and pointers on all cores: (irp_t, icol_t, val_t)."""
    irp = _i32(irp)
    nnz = int(irp[-1])
    irp_t = np.empty(int(n_cols) + 1, dtype=np.int32)
    icol_t = np.empty(nnz, dtype=np.int32)
    val_t = np.empty(nnz, dtype=np.float64)
    if _load_omp().orc_omp_crs_to_ccs(int(n_rows), int(n_cols), irp, _i32(icol), _f64(val), irp_t, icol_t, val_t,
                                      int(nthreads)) != 0:
        raise MemoryError("per-thread column counts")
    return irp_t, icol_t, val_t
