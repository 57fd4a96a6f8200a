"""Helpers of the GPU parity tests: run one pair through the C-ABI library
and through the CPU oracle on the same seeded inputs, and compare every
result element by element (everything is integer, so the bar is bit-exact)."""
import numpy as np
import torch

import oracle as O


def gpu_params(api, d):
    return api.Params(**{k: v for k, v in d.items()})


def oracle_params(d):
    return O.make_params(d)


def run_gpu(api, prm, img1, img2, stream_id=0):
    p = gpu_params(api, prm)
    t1 = torch.from_numpy(np.ascontiguousarray(img1)).cuda()
    t2 = torch.from_numpy(np.ascontiguousarray(img2)).cuda()
    P1 = api.build_pyramid(p, t1)
    P2 = api.build_pyramid(p, t2)
    ws = api.match(p, P1, P2, stream_id=stream_id)
    rows, keep = api.filter_matches(p, ws)
    torch.cuda.synchronize()
    ws.sync_status()
    return P1, P2, ws, rows.cpu().numpy(), keep.cpu().numpy()


def compare_pyramid(gpu_pyr, orc_pyr, what=""):
    for s in range(orc_pyr.schemes):
        for l in range(orc_pyr.levels):
            g = gpu_pyr.desc(s, l).cpu().numpy()              # (h, w, nch)
            o = orc_pyr.desc(s, l)                            # (nch, h, w)
            assert g.shape == (o.shape[1], o.shape[2], o.shape[0]), (what, s, l)
            bad = np.argwhere(g != o.transpose(1, 2, 0))
            assert bad.size == 0, "%s desc scheme %d level %d differs at %s" % (what, s, l, bad[:5])
            gi = gpu_pyr.cimage(s, l).cpu().numpy()
            oi = orc_pyr.cimage(s, l)
            assert (gi == oi).all(), "%s image scheme %d level %d" % (what, s, l)


def compare_fields(ws, M, levels, what=""):
    for l in range(levels):
        for d in (0, 1):
            g = {k: v.cpu().numpy() for k, v in ws.field(l, d).items()}
            o = M.field(l, d)
            assert g["valid"].shape == o["valid"].shape, (what, l, d)
            for k in ("valid", "outlier", "oinit"):
                bad = np.argwhere(g[k] != o[k])
                assert bad.size == 0, "%s level %d dir %d %s differs at %s" % (what, l, d, k, bad[:5])
            m = o["valid"].astype(bool)
            for k in ("ux", "uy"):
                bad = np.argwhere((g[k].astype(np.int32) != o[k]) & m)
                assert bad.size == 0, "%s level %d dir %d %s differs at %s" % (what, l, d, k, bad[:5])
            gc = g["cost"].view(np.uint64)
            bad = np.argwhere((gc != o["cost"]) & m)
            assert bad.size == 0, "%s level %d dir %d cost differs at %s" % (what, l, d, bad[:5])


def run_both(api, prm, img1, img2, stream_id=0, schedule=O.SCHED_CHECKERBOARD):
    P1, P2, ws, rows, keep = run_gpu(api, prm, img1, img2, stream_id)
    op = oracle_params(prm)
    Q1, Q2 = O.Pyramid(op, img1), O.Pyramid(op, img2)
    M = O.Match(op, Q1, Q2, schedule, stream_id)
    orows, okeep = M.filter()
    return (P1, P2, ws, rows, keep), (Q1, Q2, M, orows, okeep)


def assert_parity(api, prm, img1, img2, stream_id=0, what=""):
    (P1, P2, ws, rows, keep), (Q1, Q2, M, orows, okeep) = run_both(api, prm, img1, img2, stream_id)
    compare_pyramid(P1, Q1, what + " img1")
    compare_pyramid(P2, Q2, what + " img2")
    compare_fields(ws, M, prm.get("levels", 3), what)
    assert (keep == okeep).all(), what
    assert rows.shape == orows.shape and (rows == orows).all(), what
    return rows, M
