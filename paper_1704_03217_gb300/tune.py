"""Autotuner of the result-invariant launch knobs (``pgm_set_tuning``): the
shared-memory window margin of the tile kernels and the number of pairs that
share a launch.  Every setting gives bit-identical results; only the time
differs, so the tuner times one graph-captured step per setting on the caller's
workload and keeps the fastest.

Per-level iteration counts would change the results: they are method
parameters (``Params.iters_coarse`` / ``iters_fine``), not tuning knobs.
"""
import ctypes as C
import itertools

from . import _lib

SLACKS = (2, 4, 6, 8, 12)
CHUNKS = (8, 16, 32)


def get():
    t = _lib.CTuning()
    _lib.check(_lib.load().pgm_get_tuning(C.byref(t)), "pgm_get_tuning")
    return t.window_slack, t.pairs_per_launch


def set(window_slack=2, pairs_per_launch=32):
    t = _lib.CTuning(int(window_slack), int(pairs_per_launch))
    _lib.check(_lib.load().pgm_set_tuning(C.byref(t)), "pgm_set_tuning")


def search(time_setting, slacks=SLACKS, chunks=CHUNKS):
    """Try every (slack, chunk) with ``time_setting(slack, chunk) -> seconds``;
    return (best setting, {setting: seconds})."""
    times = {}
    for sl, ch in itertools.product(slacks, chunks):
        times[(sl, ch)] = time_setting(sl, ch)
    best = min(times, key=times.get)
    return best, times


def autotune(matcher, imgs1, imgs2, reps=3, slacks=SLACKS, chunks=CHUNKS):
    """Tune on a PairMatcher workload (CUDA events around graph replays), set
    the fastest knobs and return (best, times in ms)."""
    import torch

    def time_setting(sl, ch):
        set(sl, ch)
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

    best, times = search(time_setting, slacks, chunks)
    set(*best)
    return best, times
