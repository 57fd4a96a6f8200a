"""Failure detection on the device without a GPU fault: the search kernel's
bounded waits.  With a wait limit of a few cycles the first wait of every
search launch runs out; the kernel then records PGM_ERR_TIMEOUT in the
workspace status word and ends early (copies already in flight still land),
and the host reads the status.  The context stays usable: with the default
limit restored the same pair matches exactly as before."""
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_03217_gb300 import build
    build.build()
    from paper_1704_03217_gb300 import api as A
    return A


def test_wait_limit_timeout_is_reported_and_recovered(api):
    from paper_1704_03217_gb300 import _lib, synth
    L = _lib.load()
    prm = api.Params(levels=3, color=1)
    f1, f2, _ = synth.sintel_like_pair(91, 320, 240, t_max=30.0)
    P1 = api.build_pyramid(prm, torch.from_numpy(f1).cuda())
    P2 = api.build_pyramid(prm, torch.from_numpy(f2).cuda())
    ref = api.match(prm, P1, P2, stream_id=3)
    ref.sync_status()
    want = {k: v.clone() for k, v in ref.field(0, 0).items()}
    try:
        assert L.pgm_set_wait_limit(2) == 0
        ws = api.match(prm, P1, P2, stream_id=3)
        torch.cuda.synchronize()
        with pytest.raises(_lib.PGMError) as e:
            ws.sync_status()
        assert e.value.code == 5                 # PGM_ERR_TIMEOUT
        ws.sync_status()                         # read once, then cleared
    finally:
        assert L.pgm_set_wait_limit(0) == 0
    assert L.pgm_set_wait_limit(-1) == 1         # PGM_ERR_ARG
    again = api.match(prm, P1, P2, stream_id=3)
    again.sync_status()
    got = again.field(0, 0)
    for k in want:
        assert torch.equal(got[k], want[k]), k


@pytest.mark.parametrize("name,extra,pairs", [("PGM-C", {}, 2), ("PGM-CD", dict(descriptor=1), 3)])
def test_wait_limit_timeout_in_large_phases(api, name, extra, pairs):
    """The same at full size, where the search runs its per-direction
    launches (and, for the direction descriptor, the one-seed-per-lane
    kernel with its per-consumer barriers): every workspace reports the
    timeout, and afterwards the batch matches exactly as before."""
    from paper_1704_03217_gb300 import _lib, synth
    L = _lib.load()
    prm = api.Params(levels=5, color=1, **extra)
    data = [synth.sintel_like_pair(60 + k) for k in range(pairs)]
    i1 = [torch.from_numpy(d[0]).cuda() for d in data]
    i2 = [torch.from_numpy(d[1]).cuda() for d in data]
    m = api.PairMatcher(prm, 1024, 436, batch=pairs)
    m.enqueue(i1, i2)
    torch.cuda.synchronize()
    want = [r.clone() for r in m.results()]
    try:
        assert L.pgm_set_wait_limit(2) == 0
        m.enqueue(i1, i2)
        torch.cuda.synchronize()
        for ws in m.ws:
            with pytest.raises(_lib.PGMError) as e:
                ws.sync_status()
            assert e.value.code == 5
    finally:
        assert L.pgm_set_wait_limit(0) == 0
    m.enqueue(i1, i2)
    torch.cuda.synchronize()
    for ws in m.ws:
        ws.sync_status()
    for a, b in zip(m.results(), want):
        assert torch.equal(a, b), name
