"""Accuracy of the exported matches against synthetic ground truth.

The paper reports average end-point error on datasets that are not available
here (Tables 1, 3-7); this module measures the same kind of quantities on the
seeded synthetic pairs of ``synth``: for every exported match (x1, y1, x2, y2)
the end-point error |(x2 - x1, y2 - y1) - flow(x1, y1)|.

    python -m paper_1704_03217_gb300.evaluate            # the ablation table
"""
import numpy as np
import torch

from . import api, synth

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


def ablation_table(pairs, base: api.Params) -> dict:
    return {name: run(base.replace(ablation=bits), pairs) for name, bits in ABLATIONS.items()}


if __name__ == "__main__":
    from . import build
    build.build()
    pairs = [synth.sintel_like_pair(100 + s) for s in range(8)]
    base = api.Params(levels=5, color=1)
    for name, r in ablation_table(pairs, base).items():
        print("%-36s matches %7.0f  density %.3f  EPE %.3f  >3px %.4f"
              % (name, r["matches"], r["density"], r["epe"], r["outliers_3px"]))
