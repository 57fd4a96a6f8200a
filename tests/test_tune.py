"""Tuning knobs: the search logic on the CPU with a fake timer, and on the GPU
that every setting gives bit-identical results."""
import pytest


def test_search_picks_the_fastest_setting():
    from paper_1704_03217_gb300 import tune
    cost = lambda sl, ch, tw: abs(sl - 8) + abs(ch - 16) / 8.0 + abs(tw - 4)
    best, times = tune.search(cost)
    assert best == (8, 16, 4)
    assert len(times) == len(tune.SLACKS) * len(tune.CHUNKS) * len(tune.TILES)


def test_tuning_roundtrip_and_range_checks():
    from paper_1704_03217_gb300 import build, tune, _lib
    build.build()
    tune.set(4, 8, 16)
    assert tune.get() == (4, 8, 16)
    with pytest.raises(_lib.PGMError):
        tune.set(33, 8)
    with pytest.raises(_lib.PGMError):
        tune.set(4, 0)
    for bad_tile in (2, 6, 32):
        with pytest.raises(_lib.PGMError):
            tune.set(4, 8, bad_tile)
    tune.set()                                   # defaults
    assert tune.get() == (2, 32, 8)


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
        for sl, ch, tw in [(2, 32, 8), (0, 32, 4), (6, 3, 16), (12, 1, 4), (32, 5, 16),
                           (2, 32, 16), (4, 16, 4)]:
            tune.set(sl, ch, tw)
            m = api.PairMatcher(prm, 320, 200, batch=5)
            m.enqueue(t1, t2, list(range(5)))
            torch.cuda.synchronize()
            res = [r.clone() for r in m.results()]
            if ref is None:
                ref = res
            for a, b in zip(res, ref):
                assert torch.equal(a, b), (sl, ch, tw)
    finally:
        tune.set()


def test_pick_schedule_keeps_accuracy_within_margins():
    """The fastest schedule wins only if its accuracy is within the margins
    of the reference schedule's; otherwise the reference stays."""
    from paper_1704_03217_gb300 import tune
    ref = (6, 4, 4, 4, 4)
    base = {"ms": 10.0, "epe": 1.00, "outliers_3px": 0.020, "density": 0.90}
    table = {ref: base,
             (6, 2, 2, 2, 2): dict(base, ms=7.0, epe=1.05, outliers_3px=0.023),
             (3, 3, 3, 3, 3): dict(base, ms=5.0, epe=1.30),                  # EPE too high
             (4, 2, 2, 2, 2): dict(base, ms=6.0, outliers_3px=0.030),        # outliers too high
             (4, 4, 4, 4, 4): dict(base, ms=6.5, density=0.85)}              # too sparse
    assert tune.pick_schedule(table, ref) == (6, 2, 2, 2, 2)
    table[(6, 2, 2, 2, 2)]["epe"] = 1.2
    assert tune.pick_schedule(table, ref) == ref
    seen = []
    best, tab = tune.tune_schedule(
        __import__("paper_1704_03217_gb300.api", fromlist=["Params"]).Params(levels=5),
        lambda p: seen.append(p.iters_level) or 10.0 - sum(p.iters_level) / 10.0,
        lambda p: {"epe": 1.0, "outliers_3px": 0.0, "density": 1.0},
        schedules=((6, 4, 4, 4, 4), (3, 3, 3, 3, 3)))
    assert seen == [(6, 4, 4, 4, 4), (3, 3, 3, 3, 3)] and best == (6, 4, 4, 4, 4)


@pytest.mark.gpu
def test_tuned_schedule_matches_the_oracle():
    """Schedule tuning on a small Sintel-shaped batch, then the chosen
    per-level counts run through the CPU oracle: the GPU result at those
    counts is bit-exact with it, as for the paper's counts."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import numpy as np
    from paper_1704_03217_gb300 import api, build, evaluate, synth, tune
    from pgm_compare import assert_parity
    build.build()
    prm = api.Params(levels=4, color=1)
    pairs = [synth.sintel_like_pair(80 + k, 320, 200, t_max=40.0) for k in range(3)]
    t1 = [torch.from_numpy(p[0]).cuda() for p in pairs]
    t2 = [torch.from_numpy(p[1]).cuda() for p in pairs]

    def run(p):
        m = api.PairMatcher(p, 320, 200, batch=3)
        m.enqueue(t1, t2, list(range(3)))
        torch.cuda.synchronize()
        return m

    def time_schedule(p):
        m = run(p)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        m.enqueue(t1, t2, list(range(3)))
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    def accuracy(p):
        m = run(p)
        acc = [evaluate.match_accuracy(r.cpu().numpy(), pr[2], m.cap) for r, pr in zip(m.results(), pairs)]
        return {k: float(np.mean([a[k] for a in acc])) for k in ("epe", "outliers_3px", "density")}

    scheds = ((6, 4, 4, 4), (6, 2, 2, 2), (4, 3, 3, 3), (3, 1, 1, 1))
    best, table = tune.tune_schedule(prm, time_schedule, accuracy, schedules=scheds)
    assert best in table and set(table) == set(scheds)
    ref = table[scheds[0]]
    assert table[best]["epe"] <= ref["epe"] + tune.MARGINS["epe"]
    assert_parity(api, dict(levels=4, color=1, iters_level=best), pairs[0][0], pairs[0][1],
                  stream_id=0, what="tuned %s" % (best,))
