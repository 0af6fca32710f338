"""Off-line phase of the run-time AT method (Katagiri & Sato, Sec. 2.2) on this
GPU: measure R_ell and D_mat over a set of matrices, take D* by the rule,
and keep the result in a JSON file that the on-line phase reads.

    python -m paper_2407_00019_gb300.calibrate --out dstar.json [--scale 1.0]

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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default="dstar.json")
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--rule", type=int, default=0)
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--detail", action="store_true", help="also print t_crs, t_ell, t_trans, SP and TT per matrix")
    args = ap.parse_args()
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
