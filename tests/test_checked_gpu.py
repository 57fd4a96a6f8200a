"""The checked build (libpgm_checked.so, device index checks that report
PGM_ERR_DEVICE_BOUNDS) on in-bounds work: no check fires, and every export
equals the regular build's.  The checked library runs in a child process
(PGM_CHECKED=1 selects it at load time)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (params, size, pairs): the int16 search with its global-memory path, the
# bit-plane search with one seed per lane (level 0 of three full-size pairs
# has more than 12 tiles per SM), and gray bit-planes at a small size
CASES = [(dict(levels=4, color=1), (512, 218), 2),
         (dict(levels=5, color=1, descriptor=1), (1024, 436), 3),
         (dict(levels=3, color=0, descriptor=1), (320, 240), 2)]

CHILD = r"""
import json, sys
import numpy as np
import torch
sys.path.insert(0, %(root)r)
from paper_1704_03217_gb300 import api, synth, _lib
cases = json.loads(sys.argv[1])
out = {"checked": int(_lib.load().pgm_checked_build()), "rows": []}
for prm, (w, h), n in cases:
    p = api.Params(**prm)
    pairs = [synth.sintel_like_pair(40 + k, w, h, t_max=min(150.0, w / 8), rgb=bool(p.color))
             for k in range(n)]
    m = api.PairMatcher(p, w, h, batch=n)
    m.enqueue([torch.from_numpy(a[0]).cuda() for a in pairs], [torch.from_numpy(a[1]).cuda() for a in pairs])
    torch.cuda.synchronize()
    for ws in m.ws:
        ws.sync_status()                  # raises on PGM_ERR_DEVICE_BOUNDS
    out["rows"].append([r.cpu().numpy().tolist() for r in m.results()])
print(json.dumps(out))
"""


def run(env_checked):
    env = dict(os.environ)
    env["PGM_CHECKED"] = "1" if env_checked else "0"
    r = subprocess.run([sys.executable, "-c", CHILD % {"root": ROOT}, json.dumps(CASES)],
                       capture_output=True, text=True, env=env, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_checked_build_is_silent_and_identical():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_03217_gb300 import build
    build.build()
    build.build(checked=True)
    plain, checked = run(False), run(True)
    assert plain["checked"] == 0 and checked["checked"] == 1
    for a, b in zip(plain["rows"], checked["rows"]):
        assert a == b
        assert sum(len(x) for x in a) > 0
