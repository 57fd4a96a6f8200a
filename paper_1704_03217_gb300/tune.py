"""Autotuners.

Launch knobs (``pgm_set_tuning``): the shared-memory window margin of the
search kernels, the number of pairs that share a launch and the shape of a
search tile (64 seeds as 4 x 16, 8 x 8 or 16 x 4).  Every setting gives
bit-identical results; only the time differs, so the tuner times one
graph-captured step per setting on the caller's workload and keeps the
fastest.

Per-level iteration schedules (``Params.iters_level``) change the results:
they are method parameters.  ``tune_schedule`` times candidate schedules and
scores each against synthetic ground truth, and keeps the fastest one whose
accuracy stays within stated margins of the paper's schedule; the caller
checks the chosen schedule against the CPU oracle (bit-exact parity holds for
any schedule).
"""
import ctypes as C
import itertools

from . import _lib

SLACKS = (2, 4, 6, 8, 12)
CHUNKS = (8, 16, 32)
TILES = (4, 8, 16)


def get():
    t = _lib.CTuning()
    _lib.check(_lib.load().pgm_get_tuning(C.byref(t)), "pgm_get_tuning")
    return t.window_slack, t.pairs_per_launch, t.tile_w


def set(window_slack=2, pairs_per_launch=32, tile_w=8):
    t = _lib.CTuning(int(window_slack), int(pairs_per_launch), int(tile_w))
    _lib.check(_lib.load().pgm_set_tuning(C.byref(t)), "pgm_set_tuning")


def search(time_setting, slacks=SLACKS, chunks=CHUNKS, tiles=TILES):
    """Try every (slack, chunk, tile width) with ``time_setting(slack, chunk,
    tile_w) -> seconds``; return (best setting, {setting: seconds})."""
    times = {}
    for sl, ch, tw in itertools.product(slacks, chunks, tiles):
        times[(sl, ch, tw)] = time_setting(sl, ch, tw)
    best = min(times, key=times.get)
    return best, times


def autotune(matcher, imgs1, imgs2, reps=3, slacks=SLACKS, chunks=CHUNKS, tiles=TILES):
    """Tune on a PairMatcher workload (CUDA events around graph replays), set
    the fastest knobs and return (best, times in ms)."""
    import torch

    def time_setting(sl, ch, tw):
        set(sl, ch, tw)
        matcher.capture(imgs1, imgs2)
        matcher.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            matcher.replay()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    best, times = search(time_setting, slacks, chunks, tiles)
    set(*best)
    return best, times


# Candidate per-level schedules (level 0 first) for a 5-level pyramid: the
# paper's (6 at full resolution, 4 above) and cheaper or redistributed ones.
SCHEDULES_L5 = ((6, 4, 4, 4, 4), (6, 3, 3, 3, 3), (6, 2, 2, 2, 2), (5, 3, 3, 3, 3),
                (4, 4, 4, 4, 4), (4, 3, 3, 3, 3), (4, 2, 2, 2, 2), (6, 4, 4, 2, 2),
                (3, 3, 3, 3, 3))

# accuracy margins against the paper's schedule: mean end-point error of the
# exported matches, their > 3 px share, and their density (matches per seed)
MARGINS = {"epe": 0.10, "outliers_3px": 0.005, "density": 0.02}


def pick_schedule(table, reference, margins=MARGINS):
    """table: {schedule: {"ms": t, "epe": e, "outliers_3px": o, "density": d}};
    the fastest schedule whose accuracy is within `margins` of
    table[reference] (EPE and outlier share no more than that much higher,
    density no more than that much lower); the reference itself otherwise."""
    ref = table[reference]
    ok = [s for s, r in table.items()
          if r["epe"] <= ref["epe"] + margins["epe"]
          and r["outliers_3px"] <= ref["outliers_3px"] + margins["outliers_3px"]
          and r["density"] >= ref["density"] - margins["density"]]
    return min(ok, key=lambda s: table[s]["ms"]) if ok else reference


def tune_schedule(params, time_schedule, accuracy, schedules=SCHEDULES_L5, margins=MARGINS):
    """Score every per-level schedule: ``time_schedule(params') -> ms`` and
    ``accuracy(params') -> {"epe", "outliers_3px", "density"}`` with params' =
    params with that schedule; the first schedule is the reference.  Returns
    (chosen schedule, table)."""
    table = {}
    for s in schedules:
        p = params.replace(iters_level=tuple(s))
        r = dict(accuracy(p))
        r["ms"] = float(time_schedule(p))
        table[tuple(s)] = r
    return pick_schedule(table, tuple(schedules[0]), margins), table
