"""Host-side fault injection into the matching schedule
(pgm_inject_launch_failure): a launch step refused part-way through a call
makes the call return PGM_ERR_CUDA, and everything the call had enqueued
before -- also what it had forked onto its auxiliary streams (the finer
levels' box sums, the backward search phases) -- is joined back to the
caller's stream.  The check is a CUDA-graph capture of the failing call: a
capture ends cleanly only when nothing forked from its stream is left
unjoined.  The same failure on an eagerly running call leaves the device
usable: the next call on the same workspace matches exactly as before."""
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# 1024x436, L = 5, PGM-C: 5 box-sum steps, then 9 visits of (transfer or
# initialisation, 2 T colour phases, consistency): 99 steps.  Step 1 is the
# coarsest level's box sums (nothing forked yet), 2 the first forked one, 6
# the initialisation (four levels' box sums pending), 90 a level-0 colour
# phase (backward phases pending), 99 the last consistency check.
STEPS = (1, 2, 6, 90, 99)


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_03217_gb300 import build
    build.build()
    from paper_1704_03217_gb300 import api, synth
    prm = api.Params(levels=5, color=1)
    f1, f2, _ = synth.sintel_like_pair(93)
    P1 = api.build_pyramid(prm, torch.from_numpy(f1).cuda())
    P2 = api.build_pyramid(prm, torch.from_numpy(f2).cuda())
    ref = api.match(prm, P1, P2, stream_id=4)
    ref.sync_status()
    want = {(l, d): {k: v.clone() for k, v in ref.field(l, d).items()}
            for l in range(5) for d in (0, 1)}
    return api, prm, P1, P2, want


def _same(ws, want):
    for (l, d), f in want.items():
        got = ws.field(l, d)
        for k in f:
            assert torch.equal(got[k], f[k]), (l, d, k)


@pytest.mark.parametrize("step", STEPS)
def test_failure_in_a_capture_leaves_nothing_unjoined(setup, step):
    from paper_1704_03217_gb300 import _lib
    api, prm, P1, P2, want = setup
    L = _lib.load()
    ws = api.Workspace(prm, 1024, 436, 1024, 436)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    assert L.pgm_inject_launch_failure(step) == 0
    try:
        with pytest.raises(_lib.PGMError) as e:
            with torch.cuda.graph(g):
                api.match(prm, P1, P2, stream_id=4, ws=ws)
    finally:
        assert L.pgm_inject_launch_failure(0) == 0
    assert e.value.code == 4 and "injected launch failure" in str(e.value)
    del g
    api.match(prm, P1, P2, stream_id=4, ws=ws)
    ws.sync_status()
    _same(ws, want)


def test_failure_in_an_eager_call_then_recovery(setup):
    from paper_1704_03217_gb300 import _lib
    api, prm, P1, P2, want = setup
    L = _lib.load()
    assert L.pgm_inject_launch_failure(-1) == 1            # PGM_ERR_ARG
    ws = api.Workspace(prm, 1024, 436, 1024, 436)
    for step in (90, 6):
        assert L.pgm_inject_launch_failure(step) == 0
        try:
            with pytest.raises(_lib.PGMError) as e:
                api.match(prm, P1, P2, stream_id=4, ws=ws)
        finally:
            assert L.pgm_inject_launch_failure(0) == 0
        assert e.value.code == 4
        torch.cuda.synchronize()
        api.match(prm, P1, P2, stream_id=4, ws=ws)
        ws.sync_status()
        _same(ws, want)
    # armed beyond the call's steps: the call runs whole, and stays correct
    assert L.pgm_inject_launch_failure(1000) == 0
    try:
        api.match(prm, P1, P2, stream_id=4, ws=ws)
        ws.sync_status()
    finally:
        assert L.pgm_inject_launch_failure(0) == 0
    _same(ws, want)
