"""Tuning knobs: the search logic on the CPU with a fake timer, and on the GPU
that every setting gives bit-identical results."""
import pytest


def test_search_picks_the_fastest_setting():
    from paper_1704_03217_gb300 import tune
    cost = lambda sl, ch: abs(sl - 8) + abs(ch - 16) / 8.0
    best, times = tune.search(cost)
    assert best == (8, 16) and len(times) == len(tune.SLACKS) * len(tune.CHUNKS)


def test_tuning_roundtrip_and_range_checks():
    from paper_1704_03217_gb300 import build, tune, _lib
    build.build()
    tune.set(4, 8)
    assert tune.get() == (4, 8)
    with pytest.raises(_lib.PGMError):
        tune.set(33, 8)
    with pytest.raises(_lib.PGMError):
        tune.set(4, 0)
    tune.set()                                   # defaults
    assert tune.get() == (2, 32)


@pytest.mark.gpu
def test_every_setting_gives_identical_results():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_03217_gb300 import api, build, synth, tune
    build.build()
    prm = api.Params(levels=4, color=1)
    pairs = [synth.sintel_like_pair(60 + k, 320, 200, t_max=40.0) for k in range(5)]
    t1 = [torch.from_numpy(p[0]).cuda() for p in pairs]
    t2 = [torch.from_numpy(p[1]).cuda() for p in pairs]
    ref = None
    try:
        for sl, ch in [(2, 32), (0, 32), (6, 3), (12, 1), (32, 5)]:
            tune.set(sl, ch)
            m = api.PairMatcher(prm, 320, 200, batch=5)
            m.enqueue(t1, t2, list(range(5)))
            torch.cuda.synchronize()
            res = [r.clone() for r in m.results()]
            if ref is None:
                ref = res
            for a, b in zip(res, ref):
                assert torch.equal(a, b), (sl, ch)
    finally:
        tune.set()
