"""Off-line phase of the run-time AT method (Katagiri & Sato, Sec. 2.2) on this
GPU: measure R_ell and D_mat over a set of matrices, take D* by the rule,
and keep the result in a JSON file that the on-line phase reads.

    python -m paper_2407_00019_gb300.calibrate --out dstar.json [--scale 1.0]
    python -m paper_2407_00019_gb300.calibrate --schedule --out schedule.json

The default set is shaped by the statistics of the paper's Table 1 (N, NNZ
and deviation of each of its 22 test matrices, Sec. 4.2): synthetic banded
matrices with gamma-distributed row lengths stand in for the matrices
themselves, which are not used. All measurement runs in the CUDA library
(spmv_calibrate); this module only builds inputs and stores results.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import time

# (N, NNZ, deviation) of the 22 test matrices, Table 1 (Sec. 4.2).
TABLE1_SHAPES = [
    (20082, 281150, 2.69), (40401, 201201, 0.14), (116158, 8516500, 419.58), (115067, 1033473, 0.58),
    (259156, 4429042, 4.39), (17758, 126150, 22.03), (12005, 259879, 12.28), (13514, 352762, 13.76),
    (85623, 2374949, 14.71), (14214, 259688, 3.94), (32769, 381326, 13.95), (48600, 1181120, 4.25),
    (157464, 3866688, 4.06), (26064, 177168, 0.43), (26068, 177016, 0.43), (51993, 380415, 3.35),
    (12504, 874887, 34.92), (29067, 2081063, 37.06), (42930, 3148656, 36.98), (14734, 95053, 0.57),
    (25228, 175027, 6.38), (84617, 463625, 0.54),
]


def table1_shaped_set(scale: float = 1.0, seed: int = 100):
    """Host CRS matrices with Table 1's shapes; `scale` multiplies N and NNZ."""
    import spmv_synth as synth
    mats = []
    for i, (n, nnz, sg) in enumerate(TABLE1_SHAPES):
        ns, nnzs = max(64, int(n * scale)), max(64, int(nnz * scale))
        mats.append(synth.banded_random_crs(ns, nnzs, sg, seed=seed + i))
    return mats


def run_offline(host_mats, c: float = 1.0, rule: int = 0, timing_reps: int = 20, warmup_reps: int = 3,
                mem_cap_bytes: int = 0):
    """Returns a dict: dstar, rule, c, points [(D_mat, R_ell)], device."""
    import torch

    import paper_2407_00019_gb300 as L
    dev = [L.Crs.from_host(H) for H in host_mats]
    dstar, d, r = L.spmv_calibrate(dev, c=c, dstar_rule=rule, timing_reps=timing_reps,
                                   warmup_reps=warmup_reps, mem_cap_bytes=mem_cap_bytes)
    return {"dstar": dstar, "rule": rule, "c": c, "points": list(zip(d, r)),
            "device": torch.cuda.get_device_name(), "library_version": L.spmv_version(),
            "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())}


CALIBRATION_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "calibration")


def committed_path(rule: str = "prefix", device: str = "NVIDIA GB300") -> str:
    """Path of the committed calibration of `device` under `rule` ("prefix" or
    "maxpass"): made with this module on that device, 30 timed repetitions."""
    return os.path.join(CALIBRATION_DIR, device.replace(" ", "_") + f"_{rule}.json")


def save_dstar(path: str, result: dict) -> None:
    res = dict(result)
    res["dstar"] = res["dstar"] if math.isfinite(res["dstar"]) else "inf"
    with open(path, "w") as f:
        json.dump(res, f, indent=1)


def load_dstar(path: str, device: str | None = None) -> float:
    """D* from a saved calibration; raises if it was made on another device."""
    with open(path) as f:
        res = json.load(f)
    if device is not None and res.get("device") != device:
        raise ValueError(f"calibration made on {res.get('device')!r}, not {device!r}")
    d = res["dstar"]
    return math.inf if d == "inf" else float(d)


# ---- the batch schedule (lanes per row by mean row length), Sec. 2.2 style --
SCHED_CLASSES = 10
SCHED_LANES = (1, 8, 32)


def schedule_class_mean(c: int) -> float:
    """A mean row length inside class c (class 0: below 1; c >= 1: [2^(c-1), 2^c))."""
    return 0.6 if c == 0 else 1.5 * 2.0 ** (c - 1)


def schedule_set_for_class(c: int, seed: int = 200, entries: int = 16_000_000, rows: int = 4096):
    """Host matrices of one schedule class: banded random rows of that mean
    length (log-normal lengths, deviation half the mean), about `entries`
    entries in all."""
    import spmv_synth as synth
    mu = schedule_class_mean(c)
    count = int(min(1000, max(8, entries // max(1, int(rows * mu)))))
    return [synth.banded_random_crs(rows, max(1, int(rows * mu)), 0.5 * mu, seed=seed + 1000 * c + i)
            for i in range(count)]


def run_schedule(reps: int = 20, warm: int = 3, classes=range(SCHED_CLASSES)):
    """Off-line phase of the batch schedule: for each class, the batch product
    of a calibration batch (all CRS) timed with 1, 8 and 32 lanes per row
    (spmv_batch_time, medians of CUDA-event times); the fastest is the class's
    entry. Returns dict(table, times_ms, device, when)."""
    import torch

    import paper_2407_00019_gb300 as L
    import spmv_synth as synth
    table = list(L.spmv_batch_schedule_get())
    times = {}
    for c in classes:
        host = schedule_set_for_class(c)
        dev = L.Crs.batch_from_host(host)
        nc, nr = sum(H.n_cols for H in host), sum(H.n_rows for H in host)
        x = torch.from_numpy(synth.vector_pm1(nc, seed=5)).cuda()
        y = torch.empty(nr, dtype=torch.float64, device="cuda")
        t = {}
        for lanes in SCHED_LANES:
            with L.hint(L.SPMV_HINT_BATCH_TPR, lanes):
                B = L.spmv_batch_create(dev, dstar=0.0)
            t[lanes] = B.time(x, y, warm=warm, reps=reps)
            B.close()
        times[c] = t
        table[c] = min(t, key=t.get)
        del dev, x, y
        torch.cuda.empty_cache()
    return {"table": table, "times_ms": {str(c): {str(k): v for k, v in t.items()} for c, t in times.items()},
            "device": torch.cuda.get_device_name(), "library_version": L.spmv_version(),
            "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())}


def committed_schedule_path(device: str = "NVIDIA GB300") -> str:
    return os.path.join(CALIBRATION_DIR, device.replace(" ", "_") + "_batch_schedule.json")


def save_schedule(path: str, result: dict) -> None:
    with open(path, "w") as f:
        json.dump(result, f, indent=1)


def load_schedule(path: str, device: str | None = None) -> list:
    """The lanes-per-row table of a saved schedule calibration; raises if it
    was made on another device."""
    with open(path) as f:
        res = json.load(f)
    if device is not None and res.get("device") != device:
        raise ValueError(f"schedule made on {res.get('device')!r}, not {device!r}")
    table = [int(v) for v in res["table"]]
    if len(table) != SCHED_CLASSES or any(v not in SCHED_LANES for v in table):
        raise ValueError("malformed schedule table")
    return table


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default="dstar.json")
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--rule", type=int, default=0)
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--detail", action="store_true", help="also print t_crs, t_ell, t_trans, SP and TT per matrix")
    ap.add_argument("--schedule", action="store_true",
                    help="calibrate the batch schedule table (lanes per row by mean row length) instead of D*")
    args = ap.parse_args()
    if args.schedule:
        res = run_schedule(reps=args.reps)
        save_schedule(args.out, res)
        print(json.dumps({"table": res["table"]}))
        for c, t in res["times_ms"].items():
            print(f"class {c} (mean {schedule_class_mean(int(c)):.1f}): " +
                  "  ".join(f"{k} lanes {v:.3f} ms" for k, v in t.items()))
        return
    mats = table1_shaped_set(args.scale)
    res = run_offline(mats, rule=args.rule, timing_reps=args.reps)
    save_dstar(args.out, res)
    print(json.dumps({"dstar": res["dstar"] if math.isfinite(res["dstar"]) else "inf", "n": len(mats)}))
    detail = [None] * len(mats)
    if args.detail:
        import paper_2407_00019_gb300 as L
        detail = [L.spmv_measure(L.Crs.from_host(H), timing_reps=args.reps) for H in mats]
    for (dm, r), (n, nnz, sg), t in zip(res["points"], TABLE1_SHAPES, detail):
        line = f"N={n:7d} NNZ={nnz:8d} sigma={sg:7.2f}  D_mat={dm:.3f}  R_ell={r:.3f}"
        if t is not None:
            line += (f"  t_crs={t['t_crs_ms'] * 1e3:.1f}us t_ell={t['t_ell_ms'] * 1e3:.1f}us"
                     f" t_trans={t['t_trans_ms'] * 1e3:.1f}us SP={t['sp']:.2f} TT={t['tt']:.2f}")
        print(line)


if __name__ == "__main__":
    main()
