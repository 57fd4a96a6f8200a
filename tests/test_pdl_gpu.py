"""Programmatic dependent launch along the matching loop is a launch option
only: with the attribute turned off (PGM_PDL=0, read once when the library
loads, so each setting runs in its own child process) a graph-captured batch
of full-size pairs gives exactly the same matches, counts and evaluation
counters as with it on (the default)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import torch
sys.path.insert(0, %(root)r)
from paper_1704_03217_gb300 import api, synth
out = []
for prm, n in ((dict(levels=5, color=1), 3), (dict(levels=5, color=1, descriptor=1), 2)):
    p = api.Params(**prm)
    pairs = [synth.sintel_like_pair(70 + k) for k in range(n)]
    m = api.PairMatcher(p, 1024, 436, batch=n)
    i1 = [torch.from_numpy(a[0]).cuda() for a in pairs]
    i2 = [torch.from_numpy(a[1]).cuda() for a in pairs]
    m.capture(i1, i2)
    m.replay()
    torch.cuda.synchronize()
    for ws in m.ws:
        ws.sync_status()
    out.append({"rows": [r.cpu().numpy().tolist() for r in m.results()],
                "evals": [ws.evals() for ws in m.ws]})
print(json.dumps(out))
"""


def run(pdl):
    env = dict(os.environ)
    env["PGM_PDL"] = "1" if pdl else "0"
    r = subprocess.run([sys.executable, "-c", CHILD % {"root": ROOT}], capture_output=True,
                       text=True, env=env, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_pdl_off_gives_the_same_results():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_03217_gb300 import build
    build.build()
    on, off = run(True), run(False)
    assert len(on) == len(off) == 2
    for a, b in zip(on, off):
        assert a["rows"] == b["rows"]
        assert a["evals"] == b["evals"]
        assert all(len(r) > 0 for r in a["rows"])
