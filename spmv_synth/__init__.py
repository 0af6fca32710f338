"""Seeded synthetic inputs: CRS matrices and vectors.

This module only draws numbers and lays out sparsity patterns. It holds none
of the arithmetic of the sparse-format transformation method (no analysis,
no transformation, no SpMV), so both the CPU oracle tests and the CUDA path
may use it as their common input source.

Random numbers come from a counter-based generator: splitmix64 (Steele, Lea
and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014)
evaluated at state ``key(seed, stream) + (index + 1) * 0x9E3779B97F4A7C15``
and passed through the splitmix64 output mix. Every value is a pure function
of ``(seed, stream, index)``; no hidden state is carried between calls.

The matrices are stored as CRS (the paper's VAL / ICOL / IRP, Sec. 2.1), with
0-based int32 indices and float64 values.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "CRS",
    "counter_u64",
    "uniform01",
    "uniform_pm1",
    "normal",
    "laplacian_2d_5pt",
    "stencil_3d_27pt",
    "power_law",
    "power_law_xmin",
    "random_crs",
    "banded_random_crs",
    "batch_matrix",
    "batch_set",
    "serve_matrix",
    "vector_pm1",
]

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


@dataclass
class CRS:
    """A square-or-rectangular sparse matrix in CRS layout (host arrays)."""

    n_rows: int
    n_cols: int
    irp: np.ndarray  # int32[n_rows + 1], irp[0] = 0, irp[n_rows] = nnz
    icol: np.ndarray  # int32[nnz], column of each entry
    val: np.ndarray  # float64[nnz]

    @property
    def nnz(self) -> int:
        return int(self.irp[-1])

    def row_slice(self, r0: int, r1: int) -> "CRS":
        """Rows [r0, r1) as a CRS matrix with the same column count."""
        a, b = int(self.irp[r0]), int(self.irp[r1])
        return CRS(r1 - r0, self.n_cols,
                   (self.irp[r0:r1 + 1] - a).astype(np.int32),
                   self.icol[a:b].copy(), self.val[a:b].copy())


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _key(seed: int, stream: int) -> np.uint64:
    s = np.array([(int(seed) & 0xFFFFFFFF) | ((int(stream) & 0xFFFFFFFF) << 32)],
                 dtype=np.uint64)
    return _mix(s)[0]


def counter_u64(seed: int, stream: int, idx) -> np.ndarray:
    """64 random bits for each counter value in ``idx`` (any int array)."""
    i = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _key(seed, stream) + (i + np.uint64(1)) * _GOLDEN
    return _mix(z)


def uniform01(seed: int, stream: int, idx) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits."""
    return (counter_u64(seed, stream, idx) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_pm1(seed: int, stream: int, idx) -> np.ndarray:
    """Uniform doubles in [-1, 1)."""
    return uniform01(seed, stream, idx) * 2.0 - 1.0


def normal(seed: int, stream: int, idx) -> np.ndarray:
    """Standard normal doubles by the Box-Muller transform (cosine branch).

    Draw ``idx`` uses counters 2*idx and 2*idx+1; the logarithm, square root
    and cosine are the platform libm's (through numpy).
    """
    i = np.asarray(idx, dtype=np.uint64)
    u1 = 1.0 - uniform01(seed, stream, i * np.uint64(2))  # (0, 1]
    u2 = uniform01(seed, stream, i * np.uint64(2) + np.uint64(1))
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def vector_pm1(n: int, seed: int, stream: int = 0) -> np.ndarray:
    """A length-n vector with entries uniform in [-1, 1)."""
    return uniform_pm1(seed, stream, np.arange(n, dtype=np.uint64))


def _compress(cols: np.ndarray, mask: np.ndarray, n_rows: int, n_cols: int) -> tuple:
    """Flatten a padded (n_rows, K) column table, keeping entries where mask."""
    lens = mask.sum(axis=1, dtype=np.int64)
    irp = np.zeros(n_rows + 1, dtype=np.int64)
    np.cumsum(lens, out=irp[1:])
    if irp[-1] >= 2 ** 31:
        raise ValueError("nnz does not fit int32 indexing")
    icol = cols[mask].astype(np.int32)
    return irp.astype(np.int32), icol


def laplacian_2d_5pt(nx: int, ny: int | None = None) -> CRS:
    """2-D 5-point Laplacian on an nx-by-ny grid, natural (row-major) order.

    Diagonal 4, each existing grid neighbour -1; columns ascend in each row.
    """
    ny = nx if ny is None else ny
    n = nx * ny
    i = np.arange(n, dtype=np.int64)
    x, y = i % nx, i // nx
    offs = [(-nx, y > 0), (-1, x > 0), (0, np.ones(n, bool)), (1, x < nx - 1), (nx, y < ny - 1)]
    cols = np.stack([i + o for o, _ in offs], axis=1)
    mask = np.stack([m for _, m in offs], axis=1)
    irp, icol = _compress(cols, mask, n, n)
    vals = np.where(np.stack([np.full(n, o == 0) for o, _ in offs], axis=1), 4.0, -1.0)
    val = vals[mask].astype(np.float64)
    return CRS(n, n, irp, icol, val)


def stencil_3d_27pt(N: int, seed: int = 1, diag_rule: str = "abs_sum") -> CRS:
    """27-point stencil on an N^3 grid, lexicographic order (x fastest).

    Off-diagonal values are N(0, 1) draws keyed by their CRS position
    (stream 0). The diagonal is 27 plus |sum of the row's off-diagonals|
    (``diag_rule="abs_sum"``) or 27 plus the sum of their absolute values
    (``diag_rule="sum_abs"``).
    """
    n = N * N * N
    i = np.arange(n, dtype=np.int64)
    x, y, z = i % N, (i // N) % N, i // (N * N)
    colslist, masklist, isdiag = [], [], []
    for dz in (-1, 0, 1):
        mz = (z + dz >= 0) & (z + dz < N)
        for dy in (-1, 0, 1):
            my = mz & (y + dy >= 0) & (y + dy < N)
            for dx in (-1, 0, 1):
                m = my & (x + dx >= 0) & (x + dx < N)
                colslist.append((i + (dz * N + dy) * N + dx).astype(np.int32))
                masklist.append(m)
                isdiag.append(dz == 0 and dy == 0 and dx == 0)
    cols = np.stack(colslist, axis=1)
    mask = np.stack(masklist, axis=1)
    del colslist, masklist
    irp, icol = _compress(cols, mask, n, n)
    del cols
    nnz = int(irp[-1])
    val = normal(seed, 0, np.arange(nnz, dtype=np.uint64))
    diagpos = np.stack([np.full(n, d) for d in isdiag], axis=1)[mask]
    del mask
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(irp).astype(np.int64))
    off = np.where(diagpos, 0.0, val)
    if diag_rule == "abs_sum":
        rs = np.abs(np.bincount(rows, weights=off, minlength=n))
    elif diag_rule == "sum_abs":
        rs = np.bincount(rows, weights=np.abs(off), minlength=n)
    else:
        raise ValueError(diag_rule)
    val[diagpos] = 27.0 + rs
    return CRS(n, n, irp, icol, val)


def power_law_xmin(mean: float = 16.0, kmax: float = 20000.0) -> float:
    """Lower cut-off a of a continuous pdf ~ k^-2 on [a, kmax] with the given mean.

    The mean of that law is ln(kmax/a) / (1/a - 1/kmax); it rises with a, so
    bisection on [1, mean] finds the root.
    """
    lo, hi = 1.0, float(mean)
    f = lambda a: math.log(kmax / a) / (1.0 / a - 1.0 / kmax) - mean
    if f(lo) > 0:
        return lo
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(mid) > 0:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


def _sorted_unique_cols(lens: np.ndarray, n_cols: int, seed: int, stream: int) -> np.ndarray:
    """For each row, lens[i] distinct columns uniform on [0, n_cols), ascending.

    First pass, all rows at once: sorted uniforms from normalised exponential
    spacings (the k-th of L sorted uniforms is S_k / S_{L+1}, S the running
    sum of L+1 unit exponentials), floored to columns; counter
    row * 2^32 + slot. Rows whose floors collide are drawn again one by one:
    iid uniform columns (counters row * 2^32 + 2^31 + j) until at least L are
    distinct, then a uniformly random L-subset of those (ordered by a keyed
    draw on the column value), which is a uniform L-subset of [0, n_cols).
    Rows asking for n_cols or more columns get every column.
    """
    n = lens.shape[0]
    lens = np.minimum(lens.astype(np.int64), n_cols)
    out_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=out_ptr[1:])
    out = np.empty(int(out_ptr[-1]), dtype=np.int32)
    todo = np.nonzero(lens > 0)[0]
    if todo.size:
        L = lens[todo]
        gp = np.zeros(todo.size + 1, dtype=np.int64)
        np.cumsum(L + 1, out=gp[1:])
        tot = int(gp[-1])
        slot = np.arange(tot, dtype=np.int64) - np.repeat(gp[:-1], L + 1)
        ctr = np.repeat(todo.astype(np.uint64) << np.uint64(32), L + 1) + slot.astype(np.uint64)
        e = -np.log(1.0 - uniform01(seed, stream, ctr))
        del ctr, slot
        cs = np.cumsum(e)
        del e
        start = np.repeat(np.concatenate(([0.0], cs[gp[1:-1] - 1])), L + 1)
        part = cs - start  # running sum within the row
        del cs, start
        total = part[gp[1:] - 1]
        keep = np.ones(tot, dtype=bool)
        keep[gp[1:] - 1] = False
        u = part[keep] / np.repeat(total, L)
        del part, keep
        c = np.minimum((u * n_cols).astype(np.int64), n_cols - 1)
        rowid = np.repeat(np.arange(todo.size), L)
        dup = np.zeros(c.size, dtype=bool)
        dup[1:] = (c[1:] == c[:-1]) & (rowid[1:] == rowid[:-1])
        bad = np.zeros(todo.size, dtype=bool)
        bad[rowid[dup]] = True
        good = np.nonzero(~bad)[0]
        if good.size:
            src = np.nonzero(~bad[rowid])[0]  # entries of good rows, row order
            dst_rows = todo[good]
            out[_ranges(out_ptr[dst_rows], lens[dst_rows])] = c[src].astype(np.int32)
        for r in todo[bad]:
            out[out_ptr[r]:out_ptr[r + 1]] = _row_unique(int(lens[r]), n_cols, seed, stream, int(r))
    return out


def _row_unique(L: int, n_cols: int, seed: int, stream: int, r: int) -> np.ndarray:
    if L >= n_cols:
        return np.arange(n_cols, dtype=np.int32)
    base = (np.uint64(r) << np.uint64(32)) + np.uint64(1 << 31)
    got = np.zeros(0, dtype=np.int64)
    used = 0
    while got.size < L:
        m = (L - got.size) * 2 + 64
        ctr = base + np.arange(used, used + m, dtype=np.uint64)
        used += m
        c = np.minimum((uniform01(seed, stream, ctr) * n_cols).astype(np.int64), n_cols - 1)
        got = np.union1d(got, c)
    if got.size > L:
        key = counter_u64(seed, stream + 1000, got.astype(np.uint64) + (np.uint64(r) << np.uint64(32)))
        got = np.sort(got[np.argsort(key, kind="stable")[:L]])
    return got.astype(np.int32)


def _ranges(starts: np.ndarray, lens: np.ndarray) -> np.ndarray:
    """Concatenation of arange(s, s + l) for each (s, l)."""
    tot = int(lens.sum())
    if tot == 0:
        return np.zeros(0, dtype=np.int64)
    p = np.zeros(lens.size + 1, dtype=np.int64)
    np.cumsum(lens, out=p[1:])
    return np.arange(tot, dtype=np.int64) - np.repeat(p[:-1] - starts, lens)


def power_law(n: int, mean: float = 16.0, kmax: int = 20000, seed: int = 3,
              n_cols: int | None = None) -> CRS:
    """Rows with lengths from a truncated power law (exponent 2), random columns.

    Lengths: inverse-CDF samples of the continuous pdf ~ k^-2 on
    [a, min(kmax, n_cols)], with a chosen so the mean is ``mean``, rounded to
    the nearest integer and raised to at least 1 (stream 1). Columns: distinct,
    uniform on [0, n_cols), ascending (stream 2). Values: N(0, 1) (stream 3).
    """
    n_cols = n if n_cols is None else n_cols
    b = float(min(kmax, n_cols))
    a = min(power_law_xmin(mean, b), b)
    u = uniform01(seed, 1, np.arange(n, dtype=np.uint64))
    inv_a, inv_b = 1.0 / a, 1.0 / b
    xs = 1.0 / (inv_a - u * (inv_a - inv_b))
    lens = np.clip(np.rint(xs), 1, n_cols).astype(np.int64)
    irp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=irp[1:])
    if irp[-1] >= 2 ** 31:
        raise ValueError("nnz does not fit int32 indexing")
    icol = _sorted_unique_cols(lens, n_cols, seed, 2)
    val = normal(seed, 3, np.arange(int(irp[-1]), dtype=np.uint64))
    return CRS(n, n_cols, irp.astype(np.int32), icol, val)


def random_crs(n_rows: int, n_cols: int, mean_len: float, seed: int,
               empty_frac: float = 0.0, dup: bool = False,
               long_rows: int = 0, long_len: int = 0) -> CRS:
    """A general random CRS for tests.

    Row lengths are uniform on [0, 2*mean_len] (stream 10), a fraction
    ``empty_frac`` of rows is emptied (stream 11), ``long_rows`` rows get
    ``long_len`` entries. Columns are distinct and ascending (stream 12)
    unless ``dup``, in which case each row's columns are drawn with
    replacement and kept in ascending order, so repeated (i, j) entries
    occur. Values are N(0, 1) (stream 13).
    """
    idx = np.arange(n_rows, dtype=np.uint64)
    lens = np.floor(uniform01(seed, 10, idx) * (2 * mean_len + 1)).astype(np.int64)
    if empty_frac > 0:
        lens[uniform01(seed, 11, idx) < empty_frac] = 0
    if long_rows:
        pick = (counter_u64(seed, 14, np.arange(long_rows, dtype=np.uint64)) % np.uint64(max(n_rows, 1))).astype(np.int64)
        lens[pick] = long_len
    lens = np.minimum(lens, n_cols)
    irp = np.zeros(n_rows + 1, dtype=np.int64)
    np.cumsum(lens, out=irp[1:])
    nnz = int(irp[-1])
    if dup:
        c = np.minimum((uniform01(seed, 12, np.arange(nnz, dtype=np.uint64)) * n_cols).astype(np.int64), n_cols - 1)
        rows = np.repeat(np.arange(n_rows, dtype=np.int64), lens)
        order = np.lexsort((c, rows))
        icol = c[order].astype(np.int32)
    else:
        icol = _sorted_unique_cols(lens, n_cols, seed, 12)
    val = normal(seed, 13, np.arange(nnz, dtype=np.uint64))
    return CRS(n_rows, n_cols, irp.astype(np.int32), icol, val)


def banded_random_crs(n: int, nnz: int, sigma: float, seed: int, band: int | None = None) -> CRS:
    """A square matrix shaped by (n, nnz, sigma): row lengths log-normal with
    mean nnz/n and deviation sigma (stream 20), rounded and clipped to
    [0, W]; columns distinct and ascending inside a window of W = min(n,
    2*band + 1) columns centred on the diagonal and shifted inwards at the
    matrix edges (stream 21); values N(0, 1) (stream 22).

    The default band, max(4*mean, mean + 6*sigma, 64), gives the
    neighbourhood locality of discretised operators while leaving room for
    the long rows a large deviation implies; clipping to the window can
    still lower the achieved nnz and deviation a little.
    """
    mu = nnz / n
    if band is None:
        band = int(max(4.0 * mu, mu + 6.0 * sigma, 64.0))
    W = int(min(n, 2 * int(band) + 1))
    if sigma > 0:
        s2 = math.log1p((sigma / mu) ** 2)
        z = normal(seed, 20, np.arange(n, dtype=np.uint64))
        lens = np.rint(np.exp(math.log(mu) - 0.5 * s2 + math.sqrt(s2) * z)).astype(np.int64)
    else:
        lens = np.full(n, int(round(mu)), np.int64)
    lens = np.clip(lens, 0, W)
    irp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=irp[1:])
    if irp[-1] >= 2 ** 31:
        raise ValueError("nnz does not fit int32 indexing")
    lo = np.clip(np.arange(n, dtype=np.int64) - int(band), 0, n - W)
    rel = _sorted_distinct_shift(lens, W, seed, 21)
    icol = (rel.astype(np.int64) + np.repeat(lo, lens)).astype(np.int32)
    val = normal(seed, 22, np.arange(int(irp[-1]), dtype=np.uint64))
    return CRS(n, n, irp.astype(np.int32), icol, val)


def _sorted_distinct_shift(lens: np.ndarray, width: int, seed: int, stream: int) -> np.ndarray:
    """For each row, lens[i] <= width distinct ascending columns in [0, width):
    L sorted uniforms (normalised exponential spacings, counter row * 2^32 +
    slot) floored onto [0, width - L + 1), plus their rank 0..L-1. Never
    collides, so no row is redrawn; the subsets are spread a little more
    evenly than uniform L-subsets (fine for synthetic sparsity patterns)."""
    n = lens.shape[0]
    L = lens.astype(np.int64)
    out = np.empty(int(L.sum()), dtype=np.int32)
    gp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(L + 1, out=gp[1:])
    ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(L, out=ptr[1:])
    step = 1 << 24  # entries per chunk of rows, bounds the temporaries
    r0 = 0
    while r0 < n:
        r1 = int(np.searchsorted(gp, gp[r0] + step, side="right")) - 1
        r1 = min(max(r1, r0 + 1), n)
        rows = np.arange(r0, r1, dtype=np.int64)
        Lc = L[r0:r1]
        g0 = gp[r0:r1 + 1] - gp[r0]
        tot = int(g0[-1])
        slot = np.arange(tot, dtype=np.int64) - np.repeat(g0[:-1], Lc + 1)
        ctr = (np.repeat(rows.astype(np.uint64), Lc + 1) << np.uint64(32)) + slot.astype(np.uint64)
        cs = np.cumsum(-np.log(1.0 - uniform01(seed, stream, ctr)))
        start = np.repeat(np.concatenate(([0.0], cs[g0[1:-1] - 1])), Lc + 1)
        part = cs - start
        total = part[g0[1:] - 1]
        keep = np.ones(tot, dtype=bool)
        keep[g0[1:] - 1] = False
        u = part[keep] / np.repeat(total, Lc)
        span = np.repeat(width - Lc + 1, Lc)
        rank = slot[keep]
        c = np.minimum((u * span).astype(np.int64), span - 1) + rank
        out[ptr[r0]:ptr[r1]] = c.astype(np.int32)
        r0 = r1
    return out


def _poisson_inv(lam: float, u: np.ndarray) -> np.ndarray:
    """Poisson(lam) by inversion of its CDF at uniforms u."""
    kmax = int(lam + 12.0 * math.sqrt(lam) + 12.0)
    k = np.arange(kmax + 1, dtype=np.float64)
    logp = k * math.log(lam) - lam - np.array([math.lgamma(v + 1.0) for v in k])
    cdf = np.cumsum(np.exp(logp))
    return np.minimum(np.searchsorted(cdf, u, side="right"), kmax).astype(np.int64)


def batch_matrix(idx: int, seed: int = 5, n_lo: int = 100, n_hi: int = 20000) -> CRS:
    """Matrix `idx` of a batch of small uneven matrices, drawn with seed
    seed + idx: n = round(exp(U[ln n_lo, ln n_hi])) (stream 30). Even idx: a
    2-D 5-point stencil (diagonal 4, neighbours -1) on a ceil(sqrt(n)) square
    grid, natural order, cut to its first n rows and columns. Odd idx: row
    lengths Poisson(8) (stream 31, at most n), distinct ascending uniform
    columns (stream 32), values N(0, 1) (stream 33)."""
    sd = seed + int(idx)
    u = float(uniform01(sd, 30, np.zeros(1, dtype=np.uint64))[0])
    n = int(round(math.exp(math.log(n_lo) + u * (math.log(n_hi) - math.log(n_lo)))))
    n = max(1, n)
    if idx % 2 == 0:
        g = int(math.ceil(math.sqrt(n)))
        i = np.arange(n, dtype=np.int64)
        gx, gy = i % g, i // g
        offs = [(-g, gy > 0), (-1, gx > 0), (0, np.ones(n, bool)), (1, (gx < g - 1) & (i + 1 < n)), (g, i + g < n)]
        cols = np.stack([i + o for o, _ in offs], axis=1)
        mask = np.stack([m for _, m in offs], axis=1)
        irp, icol = _compress(cols, mask, n, n)
        vals = np.where(np.stack([np.full(n, o == 0) for o, _ in offs], axis=1), 4.0, -1.0)
        return CRS(n, n, irp, icol, vals[mask].astype(np.float64))
    lens = np.minimum(_poisson_inv(8.0, uniform01(sd, 31, np.arange(n, dtype=np.uint64))), n)
    irp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=irp[1:])
    icol = _sorted_unique_cols(lens, n, sd, 32)
    val = normal(sd, 33, np.arange(int(irp[-1]), dtype=np.uint64))
    return CRS(n, n, irp.astype(np.int32), icol, val)


def batch_set(count: int, seed: int = 5, n_lo: int = 100, n_hi: int = 20000) -> list:
    """Matrices 0..count-1 of batch_matrix."""
    return [batch_matrix(i, seed, n_lo, n_hi) for i in range(count)]


def serve_matrix(idx: int, seed: int = 6, n_lo: int = 1000, n_hi: int = 2000000) -> CRS:
    """Matrix `idx` of a serving pool, drawn with seed seed + idx: n =
    round(exp(U[ln n_lo, ln n_hi])) (stream 40). Even idx: the cut 2-D
    5-point stencil of batch_matrix. Odd idx: power_law(n) with mean 16 and
    longest row min(20000, n)."""
    sd = seed + int(idx)
    u = float(uniform01(sd, 40, np.zeros(1, dtype=np.uint64))[0])
    n = max(1, int(round(math.exp(math.log(n_lo) + u * (math.log(n_hi) - math.log(n_lo))))))
    if idx % 2 == 0:
        g = int(math.ceil(math.sqrt(n)))
        i = np.arange(n, dtype=np.int64)
        gx, gy = i % g, i // g
        offs = [(-g, gy > 0), (-1, gx > 0), (0, np.ones(n, bool)), (1, (gx < g - 1) & (i + 1 < n)), (g, i + g < n)]
        cols = np.stack([i + o for o, _ in offs], axis=1)
        mask = np.stack([m for _, m in offs], axis=1)
        irp, icol = _compress(cols, mask, n, n)
        vals = np.where(np.stack([np.full(n, o == 0) for o, _ in offs], axis=1), 4.0, -1.0)
        return CRS(n, n, irp, icol, vals[mask].astype(np.float64))
    return power_law(n, mean=16.0, kmax=min(20000, n), seed=sd)
