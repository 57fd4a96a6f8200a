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


def test_faults_evict_only_their_requests():
    """With an injected allocation failure (request 4) and an injected device
    error (request 7), those two are evicted with an error and every other
    served request still equals the same pair matched alone; the executor's
    resident slots are reused across batches."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_03217_gb300 import build
    build.build()
    from paper_1704_03217_gb300 import api, serve, synth
    prm = api.Params(levels=4, color=1)
    sizes = [(320, 240), (256, 160)]
    reqs = []
    for k in range(12):
        w, h = sizes[k % 2]
        f1, f2, _ = synth.sintel_like_pair(70 + k, w, h, t_max=30.0)
        reqs.append(serve.Request(k, 0.003 * k, f1, f2, stream_id=200 + k))
    ex = serve.GpuExecutor(prm, streams=2, faults=serve.Faults(alloc_fail={4}, device_error={7}))
    sch = serve.Scheduler(budget_bytes=5 * ex.bytes_of(reqs[0]), max_batch=3, bytes_of=ex.bytes_of)
    done = serve.serve(reqs, sch, ex)
    assert [r.rid for r in done if r.error] == [4, 7]
    assert ex.slots_made < len(reqs)
    for r in done:
        if r.error:
            assert r.matches is None
            continue
        P1 = api.build_pyramid(prm, torch.from_numpy(r.img1).cuda())
        P2 = api.build_pyramid(prm, torch.from_numpy(r.img2).cuda())
        ws = api.match(prm, P1, P2, stream_id=r.stream_id)
        rows, _ = api.filter_matches(prm, ws)
        assert np.array_equal(rows.cpu().numpy(), r.matches), r.rid
