"""Python binding of libspmvat, the GB300 (sm_103a) library for run-time
sparse-format transformation, SpMV and D_mat / R_ell auto-tuning (Katagiri &
Sato, Sec. 2-3).

Argument marshalling only: every step runs in the CUDA library. Functions
carry the C names of ``include/spmvat.h``. Device arrays are torch CUDA
tensors (int32 indices, float64 values); the stream defaults to torch's
current stream. Importing this package never falls back to a CPU path: if
the shared library is missing it raises.
"""

from __future__ import annotations

import ctypes
import math
import os

__all__ = [
    "SpmvError", "Crs", "Matrix", "load_library", "library_path", "device_view",
    "SPMV_CRS", "SPMV_COO", "SPMV_ELL", "SPMV_ROWWISE", "SPMV_COLWISE",
    "SPMV_DSTAR_PREFIX", "SPMV_DSTAR_MAXPASS", "SPMV_AT_TRY_COO",
    "spmv_version", "spmv_status_string", "spmv_set_allocator", "spmv_reserve", "spmv_analyze", "spmv_validate",
    "spmv_ell_bytes", "spmv_transform", "spmv_transform_from", "spmv_apply", "spmv_transform_apply",
    "spmv_describe", "spmv_matrix_status", "spmv_destroy", "spmv_r_ell", "spmv_dstar_from_points", "spmv_measure",
    "spmv_calibrate", "spmv_autotune", "spmv_autotune_choose", "spmv_apply_coo_row_noalloc", "spmv_launch_count", "spmv_profile_enable", "spmv_profile_read",
    "spmv_debug_scan_timeout", "spmv_batch_create", "spmv_batch_apply", "spmv_batch_info_get",
    "spmv_batch_plan_get", "spmv_batch_destroy", "Batch", "spmv_batch_apply_multi", "Server", "spmv_server_create",
    "spmv_set_hint", "spmv_get_hint", "hint",
    "spmv_batch_prepare", "spmv_batch_build", "spmv_batch_status", "spmv_batch_schedule_set",
    "spmv_batch_schedule_get", "spmv_batch_time", "SPMV_BATCH_SCHED_CLASSES", "spmv_measure_atomics",
    "SPMV_HINT_PHASE1", "SPMV_HINT_CRS_SPLIT", "SPMV_HINT_COO_FLAT", "SPMV_HINT_BATCH_TPR",
    "SPMV_PHASE1_COUNT", "SPMV_PHASE1_KSLOT", "SPMV_PHASE1_ROWPOS", "SPMV_PHASE1_GROUPED", "SPMV_PHASE1_SYMMETRIC",
]

_HERE = os.path.dirname(os.path.abspath(__file__))

SPMV_OK = 0
SPMV_CRS, SPMV_COO, SPMV_ELL = 0, 1, 2
SPMV_ROWWISE, SPMV_COLWISE = 0, 1
SPMV_DSTAR_PREFIX, SPMV_DSTAR_MAXPASS = 0, 1
SPMV_AT_TRY_COO = 1
SPMV_HINT_PHASE1, SPMV_HINT_CRS_SPLIT, SPMV_HINT_COO_FLAT, SPMV_HINT_BATCH_TPR = 0, 1, 2, 3
SPMV_PHASE1_COUNT, SPMV_PHASE1_KSLOT, SPMV_PHASE1_ROWPOS, SPMV_PHASE1_GROUPED, SPMV_PHASE1_SYMMETRIC = 1, 2, 3, 4, 5
STATUS_NAMES = {0: "SPMV_OK", 1: "SPMV_ERR_INVALID_ARG", 2: "SPMV_ERR_INVALID_MATRIX", 3: "SPMV_ERR_OOM",
                4: "SPMV_ERR_MEMORY_CAP", 5: "SPMV_ERR_TIMEOUT", 6: "SPMV_ERR_CUDA", 7: "SPMV_ERR_UNSUPPORTED"}


class SpmvError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = int(status)
        super().__init__(f"{where}: {STATUS_NAMES.get(self.status, self.status)}")


class _CrsT(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int32), ("n_cols", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("irp", ctypes.c_void_p), ("icol", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class _StatsT(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_double), ("sigma", ctypes.c_double), ("dmat", ctypes.c_double),
                ("max_row_len", ctypes.c_int32), ("min_row_len", ctypes.c_int32),
                ("n_empty_rows", ctypes.c_int64), ("ell_bytes", ctypes.c_uint64),
                ("row_len_hist", ctypes.c_int64 * 32)]


class _AtParamsT(ctypes.Structure):
    _fields_ = [("c", ctypes.c_double), ("dstar", ctypes.c_double), ("mem_cap_bytes", ctypes.c_uint64),
                ("timing_reps", ctypes.c_int32), ("warmup_reps", ctypes.c_int32),
                ("dstar_rule", ctypes.c_int32), ("flags", ctypes.c_int32)]


class _TimingT(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("t_crs_ms", "t_ell_ms", "t_trans_ms", "t_coo_ms", "sp", "tt", "r_ell", "dmat")]


class _DescT(ctypes.Structure):
    _fields_ = [("format", ctypes.c_int32), ("layout", ctypes.c_int32), ("n_rows", ctypes.c_int32),
                ("n_cols", ctypes.c_int32), ("nnz", ctypes.c_int64), ("width", ctypes.c_int32),
                ("ld", ctypes.c_int32), ("ptr", ctypes.c_void_p), ("idx", ctypes.c_void_p),
                ("idx2", ctypes.c_void_p), ("val", ctypes.c_void_p), ("owned_bytes", ctypes.c_uint64)]


class _BatchInfoT(ctypes.Structure):
    _fields_ = [("n_matrices", ctypes.c_int32), ("n_ell", ctypes.c_int32), ("total_rows", ctypes.c_int64),
                ("total_cols", ctypes.c_int64), ("total_nnz", ctypes.c_int64), ("n_tiles", ctypes.c_int64),
                ("grid", ctypes.c_int32), ("pad", ctypes.c_int32), ("ell_bytes", ctypes.c_uint64),
                ("owned_bytes", ctypes.c_uint64)]


class _BatchPlanT(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_double), ("sigma", ctypes.c_double), ("dmat", ctypes.c_double),
                ("max_row_len", ctypes.c_int32), ("format", ctypes.c_int32), ("threads_per_row", ctypes.c_int32),
                ("rows_per_tile", ctypes.c_int32), ("width", ctypes.c_int32), ("ld", ctypes.c_int32),
                ("x_offset", ctypes.c_int64), ("y_offset", ctypes.c_int64), ("ell_val", ctypes.c_void_p),
                ("ell_idx", ctypes.c_void_p)]


class _ServerParamsT(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_uint64), ("dstar", ctypes.c_double), ("n_streams", ctypes.c_int32),
                ("amortize_products", ctypes.c_int32), ("flags", ctypes.c_int32), ("pad", ctypes.c_int32)]


class _ServerStatsT(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("submitted", "completed", "failed", "products")] + \
               [(n, ctypes.c_double) for n in ("bytes", "p50_ms", "p99_ms", "mean_ms", "max_ms", "busy_s")] + \
               [(n, ctypes.c_uint64) for n in ("cache_hits", "cache_misses", "transforms", "evictions",
                                                "cache_bytes", "peak_cache_bytes")]


class _KernelTimeT(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_uint64), ("total_ms", ctypes.c_double)]


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)

_lib = None


def library_path() -> str:
    return os.path.join(_HERE, "libspmvat.so")


def load_library():
    """Load libspmvat.so (built by ``__graft_entry__.build()``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build the CUDA library first "
                          "(python -c 'import __graft_entry__ as g; g.build()')")
    L = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp, i32, i64, u64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    sig = {
        "spmv_version": (i32, []),
        "spmv_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "spmv_set_allocator": (ctypes.c_int, [vp, vp, vp]),
        "spmv_reserve": (ctypes.c_int, [u64, vp]),
        "spmv_analyze": (ctypes.c_int, [P(_CrsT), P(_StatsT), vp]),
        "spmv_validate": (ctypes.c_int, [P(_CrsT), vp]),
        "spmv_ell_bytes": (u64, [i32, i32]),
        "spmv_transform": (ctypes.c_int, [P(_CrsT), ctypes.c_int, ctypes.c_int, u64, P(vp), vp]),
        "spmv_transform_from": (ctypes.c_int, [vp, ctypes.c_int, u64, P(vp), vp]),
        "spmv_apply": (ctypes.c_int, [vp, vp, vp, vp]),
        "spmv_transform_apply": (ctypes.c_int, [P(_CrsT), vp, vp, u64, P(vp), vp]),
        "spmv_describe": (ctypes.c_int, [vp, P(_DescT)]),
        "spmv_matrix_status": (ctypes.c_int, [vp, vp]),
        "spmv_destroy": (None, [vp]),
        "spmv_r_ell": (dbl, [dbl, dbl, dbl]),
        "spmv_dstar_from_points": (ctypes.c_int, [i32, P(dbl), P(dbl), dbl, i32, P(dbl)]),
        "spmv_measure": (ctypes.c_int, [P(_CrsT), P(_AtParamsT), P(_TimingT), vp]),
        "spmv_calibrate": (ctypes.c_int, [P(P(_CrsT)), i32, P(_AtParamsT), P(dbl), P(dbl), P(dbl), vp]),
        "spmv_autotune": (ctypes.c_int, [P(_CrsT), P(_AtParamsT), P(vp), P(_StatsT), vp]),
        "spmv_autotune_choose": (ctypes.c_int, [P(_CrsT), P(_AtParamsT), P(i32), P(i32), P(_StatsT), vp]),
        "spmv_apply_coo_row_noalloc": (ctypes.c_int, [i32, i32, i64, vp, vp, vp, vp, vp, vp]),
        "spmv_launch_count": (u64, []),
        "spmv_set_hint": (ctypes.c_int, [i32, i32]),
        "spmv_get_hint": (i32, [i32]),
        "spmv_profile_enable": (ctypes.c_int, [i32]),
        "spmv_profile_read": (i32, [P(_KernelTimeT), i32, i32]),
        "spmv_debug_scan_timeout": (ctypes.c_int, [i32, i32, P(i32), vp]),
        "spmv_batch_create": (ctypes.c_int, [P(_CrsT), i32, P(_AtParamsT), vp, vp, P(vp), vp]),
        "spmv_batch_apply": (ctypes.c_int, [vp, vp, vp, vp]),
        "spmv_batch_apply_multi": (ctypes.c_int, [vp, vp, i64, vp, i64, i32, vp]),
        "spmv_batch_info_get": (ctypes.c_int, [vp, P(_BatchInfoT)]),
        "spmv_batch_plan_get": (ctypes.c_int, [vp, i32, i32, P(_BatchPlanT)]),
        "spmv_batch_destroy": (None, [vp]),
        "spmv_batch_prepare": (ctypes.c_int, [P(_CrsT), i32, P(_AtParamsT), P(vp), vp]),
        "spmv_batch_build": (ctypes.c_int, [vp, vp, vp, vp]),
        "spmv_batch_status": (ctypes.c_int, [vp]),
        "spmv_batch_schedule_set": (ctypes.c_int, [P(i32), i32]),
        "spmv_batch_schedule_get": (ctypes.c_int, [P(i32), i32]),
        "spmv_batch_time": (ctypes.c_int, [vp, vp, vp, i32, i32, P(dbl), vp]),
        "spmv_measure_atomics": (ctypes.c_int, [i64, i64, i32, P(dbl), vp]),
        "spmv_server_create": (ctypes.c_int, [P(_ServerParamsT), P(vp)]),
        "spmv_server_add_matrix": (ctypes.c_int, [vp, P(_CrsT), P(i32)]),
        "spmv_server_submit": (ctypes.c_int, [vp, i32, i32, vp, vp, vp, P(u64)]),
        "spmv_server_wait": (ctypes.c_int, [vp, u64, i32, P(dbl), P(i32)]),
        "spmv_server_drain": (ctypes.c_int, [vp, i32]),
        "spmv_server_stats_get": (ctypes.c_int, [vp, P(_ServerStatsT), i32]),
        "spmv_server_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(st: int, where: str):
    if st != SPMV_OK:
        raise SpmvError(st, where)


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else ctypes.c_void_p(0)


class Crs:
    """A CRS matrix held in torch CUDA tensors (Sec. 2.1 VAL / ICOL / IRP)."""

    def __init__(self, n_rows, n_cols, irp, icol, val):
        import torch
        for t, dt in ((irp, torch.int32), (icol, torch.int32), (val, torch.float64)):
            if t.dtype != dt or not t.is_cuda or not t.is_contiguous():
                raise TypeError("Crs wants contiguous CUDA tensors: irp/icol int32, val float64")
        self.n_rows, self.n_cols = int(n_rows), int(n_cols)
        self.irp, self.icol, self.val = irp, icol, val
        self.nnz = int(icol.numel())
        self._c = _CrsT(self.n_rows, self.n_cols, self.nnz, _ptr(irp).value, _ptr(icol).value, _ptr(val).value)

    @classmethod
    def from_host(cls, A, device="cuda"):
        """Copy a host CRS (numpy arrays: irp, icol, val, n_rows, n_cols) to the device."""
        import torch
        return cls(A.n_rows, A.n_cols, torch.from_numpy(A.irp).to(device), torch.from_numpy(A.icol).to(device),
                   torch.from_numpy(A.val).to(device))

    @property
    def c(self):
        return self._c

    @classmethod
    def batch_from_host(cls, mats, device="cuda"):
        """Copy host CRS matrices into three device tensors (one per array)
        and return one Crs per matrix viewing its part of them."""
        import numpy as np
        import torch
        nnz = [int(A.irp[-1]) for A in mats]
        e_off = np.concatenate(([0], np.cumsum(nnz)))
        p_off = np.concatenate(([0], np.cumsum([A.n_rows + 1 for A in mats])))
        irp = torch.from_numpy(np.concatenate([A.irp for A in mats]).astype(np.int32)).to(device)
        icol = torch.from_numpy(np.concatenate([A.icol for A in mats]).astype(np.int32)).to(device)
        val = torch.from_numpy(np.concatenate([A.val for A in mats]).astype(np.float64)).to(device)
        return [cls(A.n_rows, A.n_cols, irp[p_off[i]:p_off[i + 1]], icol[e_off[i]:e_off[i + 1]],
                    val[e_off[i]:e_off[i + 1]]) for i, A in enumerate(mats)]


class Matrix:
    """Owning wrapper of an spmv_matrix handle; keeps borrowed tensors alive."""

    def __init__(self, handle, keep=()):
        self.handle = ctypes.c_void_p(handle)
        self._keep = tuple(keep)
        # vector lengths, known from the descriptors (no device query, so that
        # products can be captured in a CUDA graph)
        self.total_rows = sum(int(A.n_rows) for A in self._keep)
        self.total_cols = sum(int(A.n_cols) for A in self._keep)

    def close(self):
        if self.handle and self.handle.value:
            load_library().spmv_destroy(self.handle)
            self.handle = ctypes.c_void_p(0)
            self._keep = ()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def describe(self):
        return spmv_describe(self)

    def arrays(self) -> dict:
        """Zero-copy torch views of the handle's device arrays (valid while
        the handle lives): ptr, idx, idx2, val, as present for the format."""
        import torch
        d = spmv_describe(self)
        lines = d["n_rows"] if d["layout"] == SPMV_ROWWISE else d["n_cols"]
        out = {}
        if d["format"] == SPMV_ELL:
            nslot = d["width"] * d["ld"]
            out["idx"] = device_view(d["idx"], nslot, torch.int32)
            out["val"] = device_view(d["val"], nslot, torch.float64)
            return out
        if d["ptr"]:
            out["ptr"] = device_view(d["ptr"], lines + 1, torch.int32)
        out["idx"] = device_view(d["idx"], d["nnz"], torch.int32)
        if d["idx2"]:
            out["idx2"] = device_view(d["idx2"], d["nnz"], torch.int32)
        out["val"] = device_view(d["val"], d["nnz"], torch.float64)
        return out


class Batch:
    """Owning wrapper of an spmv_batch handle; keeps the borrowed CRS alive."""

    def __init__(self, handle, keep=()):
        self.handle = ctypes.c_void_p(handle)
        self._keep = tuple(keep)
        # vector lengths, known from the descriptors (no device query, so that
        # products can be captured in a CUDA graph)
        self.total_rows = sum(int(A.n_rows) for A in self._keep)
        self.total_cols = sum(int(A.n_cols) for A in self._keep)

    def close(self):
        if self.handle and self.handle.value:
            load_library().spmv_batch_destroy(self.handle)
            self.handle = ctypes.c_void_p(0)
            self._keep = ()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply(self, x, y, stream=None):
        spmv_batch_apply(self, x, y, stream)

    def apply_multi(self, x, y, nvec, ldx=None, ldy=None, stream=None):
        """nvec products: vector j of x at j * ldx, of y at j * ldy."""
        ldx = self.total_cols if ldx is None else ldx
        ldy = self.total_rows if ldy is None else ldy
        _check(load_library().spmv_batch_apply_multi(self.handle, _ptr(x), int(ldx), _ptr(y), int(ldy), int(nvec),
                                                     _stream(stream)), "spmv_batch_apply_multi")

    def info(self) -> dict:
        return spmv_batch_info_get(self)

    def build(self, x=None, y=None, stream=None):
        """Device-planned batch: enqueue the whole build (and with x, y the
        first product); no synchronisation, capturable in a CUDA graph."""
        spmv_batch_build(self, x, y, stream)

    def status(self) -> None:
        _check(load_library().spmv_batch_status(self.handle), "spmv_batch_status")

    def time(self, x, y, warm=3, reps=20, stream=None) -> float:
        return spmv_batch_time(self, x, y, warm, reps, stream)

    def plans(self, first=0, count=None) -> list:
        return spmv_batch_plan_get(self, first, count)


class _CudaArray:
    def __init__(self, ptr, count, typestr):
        self.__cuda_array_interface__ = {"shape": (int(count),), "typestr": typestr,
                                         "data": (int(ptr or 0), False), "version": 3}


def device_view(ptr, count, dtype):
    """A torch CUDA tensor viewing `count` elements at device address `ptr`."""
    import torch
    typestr = {torch.int32: "<i4", torch.float64: "<f8"}[dtype]
    if not count:
        return torch.empty(0, dtype=dtype, device="cuda")
    return torch.as_tensor(_CudaArray(ptr, count, typestr), device="cuda")


# ---------------------------------------------------------------- the C ABI
def spmv_version() -> int:
    return load_library().spmv_version()


def spmv_status_string(status: int) -> str:
    return load_library().spmv_status_string(int(status)).decode()


_alloc_keepalive = []


def spmv_reserve(nbytes: int, stream=None) -> None:
    """Grow the library's private memory pool by nbytes (kept for reuse)."""
    _check(load_library().spmv_reserve(int(nbytes), _stream(stream)), "spmv_reserve")


def spmv_set_allocator(alloc=None, free=None, ctx=None):
    """Install Python callables alloc(bytes, ctx, stream) -> int and
    free(ptr, bytes, ctx, stream), or restore the default pool (both None)."""
    L = load_library()
    if alloc is None and free is None:
        _check(L.spmv_set_allocator(None, None, None), "spmv_set_allocator")
        return
    a, f = _ALLOC_FN(alloc), _FREE_FN(free)
    # kept for the life of the process: a buffer allocated through a hook is
    # freed through the same hook, possibly after the hook was replaced
    _alloc_keepalive.extend([a, f])
    _check(L.spmv_set_allocator(ctypes.cast(a, ctypes.c_void_p), ctypes.cast(f, ctypes.c_void_p), ctx),
           "spmv_set_allocator")


def _stats_dict(s: _StatsT) -> dict:
    return {"mu": s.mu, "sigma": s.sigma, "dmat": s.dmat, "W": s.max_row_len, "min_len": s.min_row_len,
            "n_empty": s.n_empty_rows, "ell_bytes": s.ell_bytes, "hist": list(s.row_len_hist)}


def spmv_analyze(A: Crs, stream=None) -> dict:
    s = _StatsT()
    _check(load_library().spmv_analyze(ctypes.byref(A.c), ctypes.byref(s), _stream(stream)), "spmv_analyze")
    return _stats_dict(s)


def spmv_validate(A: Crs, stream=None) -> None:
    _check(load_library().spmv_validate(ctypes.byref(A.c), _stream(stream)), "spmv_validate")


def spmv_ell_bytes(n_lines: int, width: int) -> int:
    return int(load_library().spmv_ell_bytes(int(n_lines), int(width)))


def spmv_transform(A: Crs, fmt: int, layout: int, mem_cap_bytes: int = 0, stream=None) -> Matrix:
    h = ctypes.c_void_p()
    _check(load_library().spmv_transform(ctypes.byref(A.c), int(fmt), int(layout), int(mem_cap_bytes),
                                         ctypes.byref(h), _stream(stream)), "spmv_transform")
    return Matrix(h.value, keep=(A,))


def spmv_transform_from(src: Matrix, fmt: int, mem_cap_bytes: int = 0, stream=None) -> Matrix:
    h = ctypes.c_void_p()
    _check(load_library().spmv_transform_from(src.handle, int(fmt), int(mem_cap_bytes), ctypes.byref(h),
                                              _stream(stream)), "spmv_transform_from")
    return Matrix(h.value, keep=src._keep)


def spmv_apply(M: Matrix, x, y, stream=None) -> None:
    _check(load_library().spmv_apply(M.handle, _ptr(x), _ptr(y), _stream(stream)), "spmv_apply")


def spmv_transform_apply(A: Crs, x, y, mem_cap_bytes: int = 0, stream=None) -> Matrix:
    h = ctypes.c_void_p()
    _check(load_library().spmv_transform_apply(ctypes.byref(A.c), _ptr(x), _ptr(y), int(mem_cap_bytes),
                                               ctypes.byref(h), _stream(stream)), "spmv_transform_apply")
    return Matrix(h.value, keep=(A,))


def spmv_describe(M: Matrix) -> dict:
    d = _DescT()
    _check(load_library().spmv_describe(M.handle, ctypes.byref(d)), "spmv_describe")
    return {f: getattr(d, f) for f, _ in _DescT._fields_}


def spmv_matrix_status(M: Matrix, stream=None) -> None:
    _check(load_library().spmv_matrix_status(M.handle, _stream(stream)), "spmv_matrix_status")


def spmv_destroy(M: Matrix) -> None:
    M.close()


def spmv_r_ell(t_crs: float, t_ell: float, t_trans: float) -> float:
    return float(load_library().spmv_r_ell(float(t_crs), float(t_ell), float(t_trans)))


def spmv_dstar_from_points(dmat, rell, c: float = 1.0, rule: int = SPMV_DSTAR_PREFIX) -> float:
    m = len(dmat)
    D = (ctypes.c_double * max(m, 1))(*[float(v) for v in dmat])
    R = (ctypes.c_double * max(m, 1))(*[float(v) for v in rell])
    out = ctypes.c_double()
    _check(load_library().spmv_dstar_from_points(m, D, R, float(c), int(rule), ctypes.byref(out)),
           "spmv_dstar_from_points")
    return out.value


def _params(c=1.0, dstar=math.inf, mem_cap_bytes=0, timing_reps=20, warmup_reps=3,
            dstar_rule=SPMV_DSTAR_PREFIX, flags=0) -> _AtParamsT:
    return _AtParamsT(float(c), float(dstar), int(mem_cap_bytes), int(timing_reps), int(warmup_reps),
                      int(dstar_rule), int(flags))


def spmv_measure(A: Crs, stream=None, **params) -> dict:
    t = _TimingT()
    p = _params(**params)
    _check(load_library().spmv_measure(ctypes.byref(A.c), ctypes.byref(p), ctypes.byref(t), _stream(stream)),
           "spmv_measure")
    return {f: getattr(t, f) for f, _ in _TimingT._fields_}


def spmv_calibrate(mats, stream=None, **params):
    """Returns (D*, [D_mat^i], [R_ell^i])."""
    m = len(mats)
    arr = (ctypes.POINTER(_CrsT) * max(m, 1))(*[ctypes.pointer(A.c) for A in mats])
    D = (ctypes.c_double * max(m, 1))()
    R = (ctypes.c_double * max(m, 1))()
    out = ctypes.c_double()
    p = _params(**params)
    _check(load_library().spmv_calibrate(arr, m, ctypes.byref(p), D, R, ctypes.byref(out), _stream(stream)),
           "spmv_calibrate")
    return out.value, list(D)[:m], list(R)[:m]


def spmv_autotune(A: Crs, stream=None, **params):
    """Returns (Matrix chosen, stats dict)."""
    h = ctypes.c_void_p()
    s = _StatsT()
    p = _params(**params)
    _check(load_library().spmv_autotune(ctypes.byref(A.c), ctypes.byref(p), ctypes.byref(h), ctypes.byref(s),
                                        _stream(stream)), "spmv_autotune")
    return Matrix(h.value, keep=(A,)), _stats_dict(s)


def spmv_autotune_choose(A: Crs, stream=None, **params):
    """Returns ((format, layout), stats dict) of the on-line rule, building nothing."""
    f, l = ctypes.c_int32(), ctypes.c_int32()
    s = _StatsT()
    p = _params(**params)
    _check(load_library().spmv_autotune_choose(ctypes.byref(A.c), ctypes.byref(p), ctypes.byref(f), ctypes.byref(l),
                                               ctypes.byref(s), _stream(stream)), "spmv_autotune_choose")
    return (f.value, l.value), _stats_dict(s)


SPMV_NOALLOC_SCRATCH_BYTES = (1 << 20) + 256
SPMV_NOALLOC_COO_MAX_NNZ = 134217728


def _noalloc_check(n_rows: int, n_cols: int, irow, icol, val, x, y) -> int:
    """Checks the caller's tensors before their raw pointers reach the
    kernels (which trust sizes and dtypes): returns nnz."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    want = (("irow", irow, torch.int32), ("icol", icol, torch.int32), ("val", val, torch.float64),
            ("x", x, torch.float64), ("y", y, torch.float64))
    for name, t, dt in want:
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name} must be a torch tensor")
        if t.dtype != dt:
            raise TypeError(f"{name} must be {dt}, got {t.dtype}")
        if t.device != dev:
            raise ValueError(f"{name} must be on the current CUDA device {dev}, got {t.device}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    nnz = icol.numel()
    if irow.numel() != nnz or val.numel() != nnz:
        raise ValueError(f"irow, icol and val must have the same length ({irow.numel()}, {nnz}, {val.numel()})")
    if x.numel() < n_cols or y.numel() < n_rows:
        raise ValueError(f"x needs {n_cols} and y {n_rows} elements, got {x.numel()} and {y.numel()}")
    return nnz


def spmv_apply_coo_row_noalloc(n_rows: int, n_cols: int, irow, icol, val, x, y, stream=None) -> None:
    """COO-Row SpMV from caller-owned device tensors, with no device allocation
    (temporaries in a fixed device array shared by all calls). The tensors are
    checked (dtype, device, contiguity, lengths) before the call."""
    nnz = _noalloc_check(int(n_rows), int(n_cols), irow, icol, val, x, y)
    _check(load_library().spmv_apply_coo_row_noalloc(int(n_rows), int(n_cols), int(nnz), _ptr(irow),
                                                     _ptr(icol), _ptr(val), _ptr(x), _ptr(y), _stream(stream)),
           "spmv_apply_coo_row_noalloc")


def spmv_set_hint(hint: int, value: int) -> None:
    _check(load_library().spmv_set_hint(int(hint), int(value)), "spmv_set_hint")


def spmv_get_hint(hint: int) -> int:
    return int(load_library().spmv_get_hint(int(hint)))


class hint:
    """Context manager: `with hint(SPMV_HINT_PHASE1, SPMV_PHASE1_GROUPED): ...`
    forces one schedule choice and restores the previous value on exit."""

    def __init__(self, which: int, value: int):
        self.which, self.value = int(which), int(value)

    def __enter__(self):
        self.prev = spmv_get_hint(self.which)
        spmv_set_hint(self.which, self.value)
        return self

    def __exit__(self, *exc):
        spmv_set_hint(self.which, self.prev)
        return False


def spmv_launch_count() -> int:
    return int(load_library().spmv_launch_count())


def spmv_profile_enable(on: bool) -> None:
    _check(load_library().spmv_profile_enable(1 if on else 0), "spmv_profile_enable")


def spmv_profile_read(reset: bool = False) -> dict:
    L = load_library()
    buf = (_KernelTimeT * 64)()
    n = L.spmv_profile_read(buf, 64, 1 if reset else 0)
    return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms)) for i in range(min(n, 64))}


def spmv_debug_scan_timeout(n: int, spin_limit: int, stream=None) -> int:
    obs = ctypes.c_int32()
    _check(load_library().spmv_debug_scan_timeout(int(n), int(spin_limit), ctypes.byref(obs), _stream(stream)),
           "spmv_debug_scan_timeout")
    return int(obs.value)


def spmv_batch_create(mats, x=None, y=None, stream=None, **params) -> Batch:
    """One batch over the Crs list `mats` (on-line rule per matrix with the
    AT parameters given); with x and y also the first product."""
    m = len(mats)
    arr = (_CrsT * max(m, 1))(*[A.c for A in mats])
    h = ctypes.c_void_p()
    p = _params(**params)
    _check(load_library().spmv_batch_create(arr, m, ctypes.byref(p), _ptr(x), _ptr(y), ctypes.byref(h),
                                            _stream(stream)), "spmv_batch_create")
    return Batch(h.value, keep=tuple(mats))


def spmv_batch_apply(B: Batch, x, y, stream=None) -> None:
    _check(load_library().spmv_batch_apply(B.handle, _ptr(x), _ptr(y), _stream(stream)), "spmv_batch_apply")


def spmv_batch_info_get(B: Batch) -> dict:
    i = _BatchInfoT()
    _check(load_library().spmv_batch_info_get(B.handle, ctypes.byref(i)), "spmv_batch_info_get")
    return {f: getattr(i, f) for f, _ in _BatchInfoT._fields_ if f != "pad"}


def spmv_batch_plan_get(B: Batch, first: int = 0, count=None) -> list:
    if count is None:
        count = spmv_batch_info_get(B)["n_matrices"] - first
    out = (_BatchPlanT * max(count, 1))()
    _check(load_library().spmv_batch_plan_get(B.handle, int(first), int(count), out), "spmv_batch_plan_get")
    return [{f: getattr(out[i], f) for f, _ in _BatchPlanT._fields_} for i in range(count)]


def spmv_batch_destroy(B: Batch) -> None:
    B.close()


class Server:
    """Owning wrapper of an spmv_server (continuous batching over a matrix
    pool); keeps the registered matrices alive."""

    FIXED_THRESHOLD = 1
    PLAIN = 2

    def __init__(self, mem_budget_bytes=0, dstar=0.0, n_streams=4, amortize_products=2, flags=0):
        p = _ServerParamsT(int(mem_budget_bytes), float(dstar), int(n_streams), int(amortize_products), int(flags), 0)
        h = ctypes.c_void_p()
        _check(load_library().spmv_server_create(ctypes.byref(p), ctypes.byref(h)), "spmv_server_create")
        self.handle = h
        self._mats = []

    def add_matrix(self, A: Crs) -> int:
        i = ctypes.c_int32()
        _check(load_library().spmv_server_add_matrix(self.handle, ctypes.byref(A.c), ctypes.byref(i)),
               "spmv_server_add_matrix")
        self._mats.append(A)
        return i.value

    def submit(self, mat_id: int, k: int, x, y, after=None) -> int:
        """Queue k products with matrix mat_id: x (k * n_cols), y (k * n_rows)
        device tensors; `after`: a stream whose current work must finish first
        (default: the current torch stream)."""
        r = ctypes.c_uint64()
        s = _stream(after)
        if not s.value:
            s = ctypes.c_void_p(1)  # cudaStreamLegacy: torch's default stream has handle 0, which means "none"
        _check(load_library().spmv_server_submit(self.handle, int(mat_id), int(k), _ptr(x), _ptr(y), s,
                                                 ctypes.byref(r)), "spmv_server_submit")
        return r.value

    def wait(self, req: int, timeout_ms: int = -1):
        """Returns (latency_ms, format) of a completed request."""
        lat, fmt = ctypes.c_double(), ctypes.c_int32()
        _check(load_library().spmv_server_wait(self.handle, ctypes.c_uint64(req), int(timeout_ms),
                                               ctypes.byref(lat), ctypes.byref(fmt)), "spmv_server_wait")
        return lat.value, fmt.value

    def drain(self, timeout_ms: int = -1) -> None:
        _check(load_library().spmv_server_drain(self.handle, int(timeout_ms)), "spmv_server_drain")

    def stats(self, reset: bool = False) -> dict:
        st = _ServerStatsT()
        _check(load_library().spmv_server_stats_get(self.handle, ctypes.byref(st), int(bool(reset))),
               "spmv_server_stats_get")
        return {f: getattr(st, f) for f, _ in _ServerStatsT._fields_}

    def close(self):
        if self.handle and self.handle.value:
            load_library().spmv_server_destroy(self.handle)
            self.handle = ctypes.c_void_p(0)
            self._mats = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def spmv_server_create(**kw) -> Server:
    return Server(**kw)


def spmv_batch_apply_multi(B: Batch, x, y, nvec: int, ldx=None, ldy=None, stream=None) -> None:
    B.apply_multi(x, y, nvec, ldx, ldy, stream)


SPMV_BATCH_SCHED_CLASSES = 10


def spmv_batch_prepare(mats, stream=None, **params) -> Batch:
    """Host part of a device-planned batch over the Crs list `mats` (no
    launches); then Batch.build() enqueues the rest."""
    m = len(mats)
    arr = (_CrsT * max(m, 1))(*[A.c for A in mats])
    h = ctypes.c_void_p()
    p = _params(**params)
    _check(load_library().spmv_batch_prepare(arr, m, ctypes.byref(p), ctypes.byref(h), _stream(stream)),
           "spmv_batch_prepare")
    return Batch(h.value, keep=tuple(mats))


def spmv_batch_build(B: Batch, x=None, y=None, stream=None) -> None:
    _check(load_library().spmv_batch_build(B.handle, _ptr(x), _ptr(y), _stream(stream)), "spmv_batch_build")


def spmv_batch_status(B: Batch) -> None:
    B.status()


def spmv_batch_schedule_set(tpr_by_class) -> None:
    t = (ctypes.c_int32 * max(len(tpr_by_class), 1))(*[int(v) for v in tpr_by_class])
    _check(load_library().spmv_batch_schedule_set(t, len(tpr_by_class)), "spmv_batch_schedule_set")


def spmv_batch_schedule_get() -> list:
    t = (ctypes.c_int32 * SPMV_BATCH_SCHED_CLASSES)()
    _check(load_library().spmv_batch_schedule_get(t, SPMV_BATCH_SCHED_CLASSES), "spmv_batch_schedule_get")
    return list(t)


def spmv_batch_time(B: Batch, x, y, warm=3, reps=20, stream=None) -> float:
    ms = ctypes.c_double()
    _check(load_library().spmv_batch_time(B.handle, _ptr(x), _ptr(y), int(warm), int(reps), ctypes.byref(ms),
                                          _stream(stream)), "spmv_batch_time")
    return ms.value


def spmv_measure_atomics(n_targets: int, n_adds: int, reps: int = 10, stream=None) -> float:
    """Median ms of n_adds coalesced FP64 atomic adds into n_targets doubles."""
    ms = ctypes.c_double()
    _check(load_library().spmv_measure_atomics(int(n_targets), int(n_adds), int(reps), ctypes.byref(ms),
                                               _stream(stream)), "spmv_measure_atomics")
    return ms.value
