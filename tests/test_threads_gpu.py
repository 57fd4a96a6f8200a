"""Calls from several host threads at once.  The ABI allows concurrent calls
on different workspaces: four threads, each with its own CUDA stream, build
the pyramids of their own Sintel-like pair, match it and filter it three
times over, and every result equals the same pair run alone."""
import threading

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_1704_03217_gb300 import synth

W, H = 512, 218
PRM = dict(levels=4, color=1)


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_03217_gb300 import build
    build.build()
    from paper_1704_03217_gb300 import api as A
    return A


def _run(api, p, pair, sid, stream):
    with torch.cuda.stream(stream):
        i1 = torch.from_numpy(pair[0]).cuda()
        i2 = torch.from_numpy(pair[1]).cuda()
        p1 = api.build_pyramid(p, i1, stream)
        p2 = api.build_pyramid(p, i2, stream)
        ws = api.match(p, p1, p2, sid, stream=stream)
        rows, _ = api.filter_matches(p, ws, stream=stream)
        ws.sync_status(stream)
        return rows.cpu().numpy()


def test_concurrent_host_threads(api):
    p = api.Params(**PRM)
    pairs = [synth.sintel_like_pair(sd, W, H) for sd in range(4)]
    alone = [_run(api, p, pairs[k], 40 + k, torch.cuda.Stream()) for k in range(4)]
    out = [[None] * 3 for _ in range(4)]
    errs = []

    def work(k):
        try:
            torch.cuda.set_device(0)
            st = torch.cuda.Stream()
            for r in range(3):
                out[k][r] = _run(api, p, pairs[k], 40 + k, st)
        except Exception as e:                       # reported below
            errs.append("thread %d: %r" % (k, e))

    threads = [threading.Thread(target=work, args=(k,)) for k in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errs, errs
    for k in range(4):
        assert len(alone[k]) > 0
        for r in range(3):
            assert np.array_equal(out[k][r], alone[k]), (k, r)


def test_many_caller_streams(api):
    """More caller streams than the library keeps auxiliary stream sets for
    (32 per host thread): calls on the later streams run without forking,
    and every result still equals the first."""
    p = api.Params(**PRM)
    pair = synth.sintel_like_pair(7, W, H)
    ref = _run(api, p, pair, 47, torch.cuda.Stream())
    streams = [torch.cuda.Stream() for _ in range(40)]
    for k, st in enumerate(streams):
        got = _run(api, p, pair, 47, st)
        assert np.array_equal(got, ref), k


def test_kernel_limits_shared_across_threads(api):
    """Kernel attributes (the shared-memory limit of a launch) belong to the
    device, not to a host thread: after worker threads ran small pairs, the
    main thread's larger pair still launches and equals its first result."""
    p = api.Params(**PRM)
    big = synth.sintel_like_pair(11, 512, 300)
    small = synth.sintel_like_pair(12, 256, 120)
    first = _run(api, p, big, 50, torch.cuda.Stream())
    errs = []

    def work(k):
        try:
            torch.cuda.set_device(0)
            _run(api, p, small, 60 + k, torch.cuda.Stream())
        except Exception as e:                       # reported below
            errs.append("thread %d: %r" % (k, e))

    threads = [threading.Thread(target=work, args=(k,)) for k in range(3)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errs, errs
    assert np.array_equal(_run(api, p, big, 50, torch.cuda.Stream()), first)
