"""Host side of the off-line calibration module: the Table 1 shapes agree
with the golden fixture, the banded generator gives valid CRS of the asked
shape, and D* survives a save/load round trip."""

import math
import os

import numpy as np
import pytest

import spmv_synth as synth
from paper_2407_00019_gb300 import calibrate as C

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_test_matrices.txt")


def _golden_rows():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        rows.append((int(f[2]), int(f[3]), float(f[5])))
    return rows


def test_table1_shapes_match_fixture():
    assert C.TABLE1_SHAPES == _golden_rows()


def _check_crs(H):
    assert H.irp[0] == 0 and np.all(np.diff(H.irp) >= 0) and H.irp[-1] == H.icol.size
    assert H.icol.min() >= 0 and H.icol.max() < H.n_cols
    d = np.diff(H.icol.astype(np.int64))
    inner = np.ones(d.size, dtype=bool)
    st = H.irp[1:-1]
    st = st[(st > 0) & (st <= d.size)]
    inner[st - 1] = False
    assert np.all(d[inner] > 0)  # distinct and ascending within a row


@pytest.mark.parametrize("n,nnz,sigma", [(5000, 70000, 2.69), (4000, 20000, 0.14), (3000, 90000, 40.0),
                                         (2000, 14000, 22.0)])
def test_banded_shape(n, nnz, sigma):
    H = synth.banded_random_crs(n, nnz, sigma, seed=7)
    _check_crs(H)
    lens = np.diff(H.irp)
    assert abs(H.nnz / nnz - 1) < 0.05
    if sigma >= 1:
        assert abs(lens.std() / sigma - 1) < 0.25
    band = int(max(4 * nnz / n, nnz / n + 6 * sigma, 64))
    rows = np.repeat(np.arange(n), lens)
    W = min(n, 2 * band + 1)
    lo = np.clip(rows - band, 0, n - W)
    assert np.all(H.icol >= lo) and np.all(H.icol < lo + W)


def test_banded_deterministic():
    a = synth.banded_random_crs(3000, 40000, 5.0, seed=3)
    b = synth.banded_random_crs(3000, 40000, 5.0, seed=3)
    c = synth.banded_random_crs(3000, 40000, 5.0, seed=4)
    assert np.array_equal(a.icol, b.icol) and np.array_equal(a.val, b.val)
    assert not np.array_equal(a.icol, c.icol)


def test_full_window_rows():
    # lengths equal to the window: every column of it, in order
    H = synth.banded_random_crs(64, 64 * 64, 0.0, seed=1, band=100)
    _check_crs(H)
    assert np.array_equal(H.icol.reshape(64, 64), np.tile(np.arange(64, dtype=np.int32), (64, 1)))


def test_dstar_save_load(tmp_path):
    p = str(tmp_path / "d.json")
    res = {"dstar": 0.61, "rule": 1, "c": 1.0, "points": [(0.1, 0.9)], "device": "GPU X"}
    C.save_dstar(p, res)
    assert C.load_dstar(p) == 0.61
    assert C.load_dstar(p, device="GPU X") == 0.61
    with pytest.raises(ValueError):
        C.load_dstar(p, device="GPU Y")
    C.save_dstar(p, dict(res, dstar=math.inf))
    assert C.load_dstar(p) == math.inf


def test_schedule_files_round_trip_and_refuse_another_device(tmp_path):
    from paper_2407_00019_gb300 import calibrate as cal
    res = {"table": [1, 1, 1, 1, 1, 8, 8, 8, 32, 32], "times_ms": {}, "device": "NVIDIA GB300"}
    p = tmp_path / "s.json"
    cal.save_schedule(str(p), res)
    assert cal.load_schedule(str(p), "NVIDIA GB300") == res["table"]
    with pytest.raises(ValueError):
        cal.load_schedule(str(p), "another GPU")
    bad = dict(res, table=[3] * 10)
    cal.save_schedule(str(p), bad)
    with pytest.raises(ValueError):
        cal.load_schedule(str(p))


def test_schedule_calibration_sets_cover_every_class():
    from paper_2407_00019_gb300 import calibrate as cal
    for c in (0, 3, 9):
        mats = cal.schedule_set_for_class(c, entries=200_000, rows=512)
        mu = sum(H.nnz for H in mats) / sum(H.n_rows for H in mats)
        lo, hi = (0.0, 1.0) if c == 0 else (2.0 ** (c - 1), 2.0 ** c)
        assert lo * 0.8 <= mu < hi * 1.2, (c, mu)


def test_committed_calibrations_are_for_the_gpu_and_readable():
    from paper_2407_00019_gb300 import calibrate as cal
    for rule in ("prefix", "maxpass"):
        d = cal.load_dstar(cal.committed_path(rule), "NVIDIA GB300")
        assert d >= 0.0
