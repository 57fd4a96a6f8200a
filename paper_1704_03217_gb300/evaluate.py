"""Accuracy of the exported matches against synthetic ground truth.

The paper reports average end-point error on datasets that are not available
here (Tables 1, 3-7); this module measures the same kind of quantities on the
seeded synthetic pairs of ``synth``: for every exported match (x1, y1, x2, y2)
the end-point error |(x2 - x1, y2 - y1) - flow(x1, y1)|.

    python -m paper_1704_03217_gb300.evaluate            # the ablation and stability tables
    python -m paper_1704_03217_gb300.evaluate --out results/accuracy_1024x436.json
"""
import argparse
import json

import numpy as np
import torch

from . import api, synth

# Philox keys of the random search for the stability experiment (any distinct keys)
KEYS = (0x5EED5EED1234ABCD, 0x1111222233334444, 0x9999AAAABBBBCCCC)

ABLATIONS = {"complete": 0, "no refinement of the initial field": 1,
             "propagate inliers and outliers": 2, "no outlier-record propagation": 4}


def match_accuracy(rows: np.ndarray, flow: np.ndarray, n_seeds: int) -> dict:
    """rows [n, 4] int32 matches, flow (H, W, 2) ground truth of frame 1."""
    if len(rows) == 0:
        return {"matches": 0, "density": 0.0, "epe": float("nan"), "outliers_3px": float("nan")}
    g = flow[rows[:, 1], rows[:, 0]]
    epe = np.hypot(rows[:, 2] - rows[:, 0] - g[:, 0], rows[:, 3] - rows[:, 1] - g[:, 1])
    return {"matches": int(len(rows)), "density": len(rows) / max(n_seeds, 1),
            "epe": float(epe.mean()), "outliers_3px": float((epe > 3).mean())}


def run(params: api.Params, pairs, stream_id0=0) -> dict:
    """Match each (frame1, frame2, flow) on the GPU and average the accuracy."""
    acc = []
    for k, (f1, f2, fl) in enumerate(pairs):
        P1 = api.build_pyramid(params, torch.from_numpy(f1).cuda())
        P2 = api.build_pyramid(params, torch.from_numpy(f2).cuda())
        ws = api.match(params, P1, P2, stream_id=stream_id0 + k)
        rows, _ = api.filter_matches(params, ws)
        nx, ny, *_ = ws.layout(0, 0)
        acc.append(match_accuracy(rows.cpu().numpy(), fl, nx * ny))
    keys = acc[0].keys()
    return {k: float(np.mean([a[k] for a in acc])) for k in keys}


def dense_accuracy(params: api.Params, pairs, ip: api.InterpParams = None) -> dict:
    """The exported matches densified (pgm_interpolate, Sec. III-G) against the
    ground truth at every pixel: mean and median end-point error and the
    share above 3 px, averaged over the pairs."""
    acc = []
    for k, (f1, f2, fl) in enumerate(pairs):
        P1 = api.build_pyramid(params, torch.from_numpy(f1).cuda())
        P2 = api.build_pyramid(params, torch.from_numpy(f2).cuda())
        ws = api.match(params, P1, P2, stream_id=k)
        nx, ny, *_ = ws.layout(0, 0)
        rows = torch.empty((nx * ny, 4), dtype=torch.int32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
        api.filter_into(params, ws, rows, cnt)
        flow, _ = api.interpolate(params, P1, rows, cnt, ip)
        epe = np.hypot(*(flow.cpu().numpy() - fl).transpose(2, 0, 1))
        acc.append({"epe": float(epe.mean()), "epe_median": float(np.median(epe)),
                    "outliers_3px": float((epe > 3).mean())})
    return {m: float(np.mean([a[m] for a in acc])) for m in acc[0]}


def ablation_table(pairs, base: api.Params) -> dict:
    return {name: run(base.replace(ablation=bits), pairs) for name, bits in ABLATIONS.items()}


def stability_stats(fields, flow: np.ndarray, sigma: int) -> dict:
    """Secret (3) of Sec. III-C (Fig. 4) on one pair: `fields` are the level-0
    forward fields of the same pair matched under different random-search
    keys (dicts of (ny, nx) arrays ux, uy, valid, outlier, as Workspace.field
    and the oracle's Match.field give them).  A seed valid under every key is
    stable when its final displacement is the same under every key, else
    unstable.  Returns the counts, and for each class the share of seeds whose
    displacement (under the first key) is more than 3 px from the ground
    truth at the seed centre and the share flagged by the consistency check
    (Eq. 6); and per key the mean end-point error and > 3 px share over the
    seeds valid under that key."""
    ux = [np.asarray(f["ux"], np.int64) for f in fields]
    uy = [np.asarray(f["uy"], np.int64) for f in fields]
    valid = np.all([np.asarray(f["valid"]) == 1 for f in fields], axis=0)
    ny, nx = ux[0].shape
    jj, ii = np.mgrid[0:ny, 0:nx]
    g = flow[sigma // 2 + sigma * jj, sigma // 2 + sigma * ii]
    same = np.ones((ny, nx), bool)
    for k in range(1, len(fields)):
        same &= (ux[k] == ux[0]) & (uy[k] == uy[0])
    stable, unstable = valid & same, valid & ~same
    epe = [np.hypot(ux[k] - g[..., 0], uy[k] - g[..., 1]) for k in range(len(fields))]
    out0 = epe[0] > 3
    cons0 = np.asarray(fields[0]["outlier"]) == 1

    def share(m, sel):
        return float(m[sel].mean()) if sel.any() else float("nan")

    per_key = []
    for k, f in enumerate(fields):
        v = np.asarray(f["valid"]) == 1
        per_key.append({"valid": int(v.sum()), "epe": share(epe[k], v),
                        "outliers_3px": share(epe[k] > 3, v)})
    return {"seeds_valid": int(valid.sum()), "stable": int(stable.sum()),
            "unstable": int(unstable.sum()),
            "outliers_3px_stable": share(out0, stable), "outliers_3px_unstable": share(out0, unstable),
            "consistency_outliers_stable": share(cons0, stable),
            "consistency_outliers_unstable": share(cons0, unstable),
            "per_key": per_key}


def stability(params: api.Params, pairs, keys=KEYS, stream_id0=0) -> dict:
    """The stability experiment on the GPU: every pair matched under each key
    (same stream ids), statistics per pair (stability_stats) and summed over
    the pairs."""
    per_pair = []
    for k, (f1, f2, fl) in enumerate(pairs):
        P1 = api.build_pyramid(params, torch.from_numpy(f1).cuda())
        P2 = api.build_pyramid(params, torch.from_numpy(f2).cuda())
        fields = []
        for key in keys:
            ws = api.match(params.replace(philox_key=key), P1, P2, stream_id=stream_id0 + k)
            fields.append({n: v.cpu().numpy() for n, v in ws.field(0, 0).items()})
        per_pair.append(stability_stats(fields, fl, params.seed_stride))
    tot = {n: sum(r[n] for r in per_pair) for n in ("seeds_valid", "stable", "unstable")}
    for cls in ("stable", "unstable"):
        for m in ("outliers_3px", "consistency_outliers"):
            w = [(r[m + "_" + cls], r[cls]) for r in per_pair if r[cls] > 0]
            tot[m + "_" + cls] = (sum(a * b for a, b in w) / sum(b for _, b in w)) if w else float("nan")
    tot["stable_share"] = tot["stable"] / max(1, tot["seeds_valid"])
    tot["per_key"] = [{"epe": float(np.mean([r["per_key"][i]["epe"] for r in per_pair])),
                       "outliers_3px": float(np.mean([r["per_key"][i]["outliers_3px"] for r in per_pair]))}
                      for i in range(len(keys))]
    tot["keys"] = ["0x%016X" % k for k in keys]
    return {"total": tot, "per_pair": per_pair}


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--pairs", type=int, default=8)
    ap.add_argument("--out", default="", help="write both tables to this JSON file")
    a = ap.parse_args()
    from . import build
    build.build()
    pairs = [synth.sintel_like_pair(100 + s) for s in range(a.pairs)]
    base = api.Params(levels=5, color=1)
    abl = ablation_table(pairs, base)
    for name, r in abl.items():
        print("%-36s matches %7.0f  density %.3f  EPE %.3f  >3px %.4f"
              % (name, r["matches"], r["density"], r["epe"], r["outliers_3px"]))
    dense = dense_accuracy(base, pairs)
    print("dense (interpolated) flow: EPE %.3f  median %.3f  >3px %.4f"
          % (dense["epe"], dense["epe_median"], dense["outliers_3px"]))
    st = stability(base, pairs)
    t = st["total"]
    print("stability over %d keys: %d valid seeds, %.3f stable; >3px outliers: stable %.4f, "
          "unstable %.4f; consistency outliers: stable %.4f, unstable %.4f"
          % (len(KEYS), t["seeds_valid"], t["stable_share"], t["outliers_3px_stable"],
             t["outliers_3px_unstable"], t["consistency_outliers_stable"],
             t["consistency_outliers_unstable"]))
    if a.out:
        import os
        os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
        with open(a.out, "w") as f:
            json.dump({"workload": "%d sintel-like 1024x436 RGB pairs (seeds 100..%d), PGM-C, "
                                   "L=5" % (a.pairs, 99 + a.pairs),
                       "ablation": abl, "dense_interpolation": dense, "stability": st},
                      f, indent=1)
            f.write("\n")
