"""Served results equal the results of the same pairs matched alone: batching,
overlap on several streams and mixed sizes change no match."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_mix_equals_alone():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_03217_gb300 import build
    build.build()
    from paper_1704_03217_gb300 import api, serve, synth
    prm = api.Params(levels=4, color=1)
    sizes = [(320, 240), (256, 160), (400, 150)]
    reqs = []
    for k in range(10):
        w, h = sizes[k % 3]
        f1, f2, _ = synth.sintel_like_pair(50 + k, w, h, t_max=30.0)
        reqs.append(serve.Request(k, 0.002 * k, f1, f2, stream_id=100 + k))
    ex = serve.GpuExecutor(prm, streams=3)
    sch = serve.Scheduler(budget_bytes=6 * ex.bytes_of(reqs[0]), max_batch=4, bytes_of=ex.bytes_of)
    done = serve.serve(reqs, sch, ex)
    assert len(ex.streams) == 3 and sch.peak <= sch.budget
    for r in done:
        P1 = api.build_pyramid(prm, torch.from_numpy(r.img1).cuda())
        P2 = api.build_pyramid(prm, torch.from_numpy(r.img2).cuda())
        ws = api.match(prm, P1, P2, stream_id=r.stream_id)
        rows, _ = api.filter_matches(prm, ws)
        assert np.array_equal(rows.cpu().numpy(), r.matches), r.rid
