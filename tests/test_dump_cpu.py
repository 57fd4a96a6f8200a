"""Workspace.dump / load_fields: the debugging dump of a match workspace holds
every level's and direction's fields exactly as the workspace views show them.
Runs on a workspace buffer in host memory filled with random bytes (the layout
queries are host-only), so no GPU is needed."""
import os

import numpy as np
import pytest
import torch


def test_dump_round_trip(tmp_path):
    from paper_1704_03217_gb300 import api, build
    build.build()
    prm = api.Params(levels=3, color=0, patch_fwd=8, patch_bwd=8, iters_level=(6, -1, 3))
    ws = api.Workspace(prm, 61, 47, 53, 40, device="cpu")
    g = torch.Generator().manual_seed(3)
    ws.buf.copy_(torch.randint(0, 256, ws.buf.shape, dtype=torch.uint8, generator=g))
    path = os.path.join(tmp_path, "fields.npz")
    ws.dump(path)
    params, dims, fields = api.load_fields(path)
    assert dims == (61, 47, 53, 40)
    assert api.Params(**dict(params, iters_level=tuple(params["iters_level"]))) == prm
    assert sorted(fields) == [(l, d) for l in range(3) for d in (0, 1)]
    for (level, d), f in fields.items():
        v = ws.field(level, d)
        nx, ny = ws.layout(level, d)[:2]
        assert f["ux"].shape == f["uy"].shape == f["cost"].shape == f["flags"].shape == (ny, nx)
        assert (f["ux"] == v["ux"].numpy()).all() and (f["uy"] == v["uy"].numpy()).all()
        assert (f["cost"] == v["cost"].numpy().view(np.uint64)).all()
        flags = f["flags"]
        assert ((flags & 1) == v["valid"].numpy()).all()
        assert (((flags >> 1) & 1) == v["outlier"].numpy()).all()
        assert (((flags >> 2) & 1) == v["oinit"].numpy()).all()
    # the lattice of each level and direction: stride 3, offset 1
    assert fields[(0, 0)]["ux"].shape == ((47 - 2) // 3 + 1, (61 - 2) // 3 + 1)
    assert fields[(0, 1)]["ux"].shape == ((40 - 2) // 3 + 1, (53 - 2) // 3 + 1)


def test_load_rejects_missing_file(tmp_path):
    from paper_1704_03217_gb300 import api
    with pytest.raises(FileNotFoundError):
        api.load_fields(os.path.join(tmp_path, "none.npz"))
