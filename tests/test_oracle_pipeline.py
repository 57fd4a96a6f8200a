"""Pins of the CPU oracle's whole pipeline: pure-Python brute force on tiny
images, and the invariants the method must satisfy at any size (identity,
additive bias, exact integer translation, fixed point, monotone cost).  Plus
the statistical margins between the checkerboard and the paper's sequential
schedule.  CPU only."""
import numpy as np
import pytest

import oracle as O
import brute
from paper_1704_03217_gb300 import synth

BASE = dict(levels=2, seed_stride=2, patch_fwd=3, patch_bwd=4, iters_coarse=2, iters_fine=3,
            refine_rounds=1, rs_W=2, tau2=1, min_region=3, region_dmax2=4)


def _tiny_pair(seed, w=18, h=14, rgb=False):
    rng = np.random.default_rng(seed)
    shape = (h, w, 3) if rgb else (h, w)
    a = rng.integers(0, 256, size=shape).astype(np.uint8)
    b = np.roll(a, (1, 2), axis=(0, 1))
    noise = rng.integers(-6, 7, size=shape)
    b = np.clip(b.astype(int) + noise, 0, 255).astype(np.uint8)
    return a, b


def _compare_fields(M, F, L):
    for l in range(L):
        for d in (0, 1):
            got = M.field(l, d)
            ref = F[(l, d)]
            ny, nx = got["ux"].shape
            assert (nx, ny) == (ref.nx, ref.ny)
            v = np.array(ref.valid).reshape(ny, nx)
            assert (got["valid"] == v).all(), (l, d)
            assert (got["outlier"] == np.array(ref.outl).reshape(ny, nx)).all(), (l, d)
            m = v.astype(bool)
            assert (got["ux"][m] == np.array(ref.ux).reshape(ny, nx)[m]).all(), (l, d)
            assert (got["uy"][m] == np.array(ref.uy).reshape(ny, nx)[m]).all(), (l, d)
            cost = np.array([c if c is not None else 0 for c in ref.cost], np.uint64).reshape(ny, nx)
            assert (got["cost"][m] == cost[m]).all(), (l, d)


@pytest.mark.parametrize("case", [
    dict(),
    dict(norm=1, rs_mode=1, seed_stride=1, levels=2, iters_fine=2),
    dict(descriptor=1, sobel=3, rs_W=3),
    dict(color=1, levels=3, seed_stride=1, patch_fwd=3, patch_bwd=2, iters_coarse=1, iters_fine=1),
    dict(ablation=2, refine_rounds=2),
    dict(ablation=4, tau2=2),
    dict(ablation=1, levels=3, seed_stride=1, iters_coarse=1, iters_fine=1),
    dict(descriptor=2, color=1, seed_stride=1, patch_fwd=3, patch_bwd=3),
    dict(rs_grid=3, seed_stride=1, iters_fine=2),
])
@pytest.mark.parametrize("schedule", [O.SCHED_CHECKERBOARD, O.SCHED_SEQUENTIAL])
def test_pipeline_brute(case, schedule):
    prm = dict(BASE, **case)
    prm.setdefault("philox_key", 0x1234_5678_9ABC_DEF0)
    rgb = prm.get("color", 0) == 1
    a, b = _tiny_pair(7, rgb=rgb)
    p = O.make_params(prm)
    P1, P2 = O.Pyramid(p, a), O.Pyramid(p, b)
    M = O.Match(p, P1, P2, schedule, stream_id=3)
    D1 = [[P1.desc(s, l) for l in range(prm["levels"])] for s in range(P1.schemes)]
    D2 = [[P2.desc(s, l) for l in range(prm["levels"])] for s in range(P2.schemes)]
    full = dict(O.FIELDS)
    full.update(prm)
    F = brute.run_pipeline(full, D1, D2, lambda c, k: O.philox4x32_10(c, k), schedule, 3)
    _compare_fields(M, F, prm["levels"])
    rows, keep = M.filter()
    want = brute.region_keep(F[(0, 0)], full["region_dmax2"], full["min_region"])
    assert (keep == want).all()
    assert len(rows) == int(want.sum())


def test_init_is_global_nearest_neighbour():
    """L = 1, sigma = 1: the exhaustive init is the global minimum of Eq. 3 for
    every seed, so propagation and search cannot improve it (fixed point)."""
    a, b = _tiny_pair(11, w=16, h=12)
    prm = dict(BASE, levels=1, seed_stride=1, iters_fine=3)
    p = O.make_params(prm)
    M = O.Match(p, O.Pyramid(p, a), O.Pyramid(p, b))
    p0 = O.make_params(dict(prm, iters_fine=0))
    M0 = O.Match(p0, O.Pyramid(p0, a), O.Pyramid(p0, b))
    D1 = O.Pyramid(p, a).desc(0, 0); D2 = O.Pyramid(p, b).desc(0, 0)
    f, f0 = M.field(0, 0), M0.field(0, 0)
    assert (f["ux"] == f0["ux"]).all() and (f["uy"] == f0["uy"]).all()
    for y in range(0, 12, 3):
        for x in range(0, 16, 3):
            costs = [(brute.patch_dist(D1, D2, (x, y), (qx, qy), 3), qy, qx)
                     for qy in range(12) for qx in range(16)]
            c, qy, qx = min(costs)
            assert (f0["ux"][y, x], f0["uy"][y, x], f0["cost"][y, x]) == (qx - x, qy - y, c)


def test_identity_pair_gives_zero_flow():
    f1, _, _ = synth.noise_affine_pair(3, w=96, h=64)
    prm = dict(levels=3, seed_stride=3, patch_fwd=8, patch_bwd=8, iters_coarse=3, iters_fine=3)
    P1, P2, M, rows = O.run_pair(prm, f1, f1.copy())
    for l in range(3):
        for d in (0, 1):
            f = M.field(l, d)
            assert (f["ux"] == 0).all() and (f["uy"] == 0).all() and (f["cost"] == 0).all()
            assert not f["outlier"].any()
    assert len(rows) == M.dims(0, 0)[0] * M.dims(0, 0)[1]
    assert (rows[:, 0] == rows[:, 2]).all() and (rows[:, 1] == rows[:, 3]).all()


def test_additive_bias_invariance():
    """(sum k (I + b) + 128) >> 8 = ((sum k I + 128) >> 8) + b and the Sobel taps
    sum to zero, so a bias without clipping changes no gradient and no field."""
    rng = np.random.default_rng(9)
    f1, f2, _ = synth.noise_affine_pair(4, w=80, h=60)
    f1 = (f1 // 2).astype(np.uint8); f2 = (f2 // 2).astype(np.uint8)
    prm = dict(levels=3, seed_stride=3, patch_fwd=8, patch_bwd=6, iters_coarse=2, iters_fine=2)
    _, _, M, rows = O.run_pair(prm, f1, f2)
    _, _, Mb, rowsb = O.run_pair(prm, f1 + 60, f2 + 60)
    for l in range(3):
        for d in (0, 1):
            a, b = M.field(l, d), Mb.field(l, d)
            for k in a:
                assert (a[k] == b[k]).all()
    assert (rows == rowsb).all()


@pytest.mark.parametrize("dx,dy", [(8, -4), (-12, 16)])
def test_integer_translation_is_exact(dx, dy):
    """A shift by multiples of 2^(L-1) is an exact shift at every level, so
    interior seeds find u = d with cost 0 and no consistency outliers."""
    L = 3
    w, h = 120, 96
    f1, f2, _ = synth.translate_pair(5, w, h, dx, dy)
    prm = dict(levels=L, seed_stride=3, patch_fwd=8, patch_bwd=8, iters_coarse=4, iters_fine=4)
    _, _, M, rows = O.run_pair(prm, f1, f2)
    f = M.field(0, 0)
    ny, nx = f["ux"].shape
    jj, ii = np.mgrid[0:ny, 0:nx]
    px, py = 1 + 3 * ii, 1 + 3 * jj
    m = 24 + max(abs(dx), abs(dy))
    interior = (px >= m) & (px < w - m) & (py >= m) & (py < h - m)
    assert interior.sum() > 50
    assert (f["ux"][interior] == dx).all() and (f["uy"][interior] == dy).all()
    assert (f["cost"][interior] == 0).all()
    assert not f["outlier"][interior].any()


def test_cost_non_increasing_within_visit():
    f1, f2, _ = synth.noise_affine_pair(6, w=96, h=72)
    base = dict(levels=2, seed_stride=3, patch_fwd=8, patch_bwd=8, refine_rounds=0,
                iters_coarse=2, max_visits=2)
    prev = None
    for T in range(0, 4):
        p = O.make_params(dict(base, iters_fine=T))
        M = O.Match(p, O.Pyramid(p, f1), O.Pyramid(p, f2))
        f = M.field(0, 0)
        if prev is not None:
            both = (f["valid"] == 1) & (prev["valid"] == 1)
            assert (f["cost"][both] <= prev["cost"][both]).all()
            assert (f["valid"] >= prev["valid"]).all()
        prev = f


def test_per_level_iterations_select_the_count():
    """iters_level[l] replaces the iteration count of every visit at level l
    and -1 keeps iters_coarse / iters_fine: the paper's schedule written per
    level gives the same fields, and one level's count written per level
    equals the same count given as iters_fine / iters_coarse."""
    f1, f2, _ = synth.noise_affine_pair(4, w=128, h=96)
    base = dict(levels=3, seed_stride=3, patch_fwd=8, patch_bwd=8)

    def fields(extra):
        p = O.make_params(dict(base, **extra))
        M = O.Match(p, O.Pyramid(p, f1), O.Pyramid(p, f2))
        return [M.field(l, d) for l in range(3) for d in (0, 1)]

    def same(a, b):
        return all((x[k] == y[k]).all() for x, y in zip(a, b) for k in ("ux", "uy", "valid", "cost"))

    ref = fields({})
    assert same(ref, fields(dict(iters_level=(6, 4, 4))))
    assert same(ref, fields(dict(iters_level=(-1, 4, -1))))
    assert same(fields(dict(iters_fine=2)), fields(dict(iters_level=(2,))))
    assert same(fields(dict(iters_coarse=1, iters_fine=3)), fields(dict(iters_level=(3, 1, 1))))
    assert not same(ref, fields(dict(iters_level=(6, 0, 4))))


@pytest.mark.slow
@pytest.mark.parametrize("name", ["c1", "c2", "c3"])
def test_checkerboard_vs_sequential_margins(name):
    """The checkerboard order reorders the paper's scan (Sec. III-B), so it
    must not lose accuracy against it.  Per workload, on 10 seeds: the
    checkerboard at the calibrated iteration counts against the paper's
    sequential scan at the paper's counts (Sec. IV).  Frozen margins, one-sided
    (both schedules are local searches of Eq. 3-5 and either may end in the
    better optimum): mean end-point error of the inliers at most 0.25 px
    higher, share of inliers with EPE > 3 px at most 2 points higher, at most
    5 % fewer inliers."""
    import multiprocessing as mp
    import margins
    jobs = []
    for seed in range(10):
        jobs.append((name, seed, O.SCHED_CHECKERBOARD, margins.CALIBRATED[name]))
        jobs.append((name, seed, O.SCHED_SEQUENTIAL, {}))
    with mp.get_context("spawn").Pool(min(8, mp.cpu_count())) as pool:
        res = pool.map(margins.stats, jobs)
    for seed in range(10):
        (e0, o0, n0), (e1, o1, n1) = res[2 * seed], res[2 * seed + 1]
        assert e0 - e1 <= 0.25, (seed, e0, e1)
        assert o0 - o1 <= 0.02, (seed, o0, o1)
        assert n0 >= 0.95 * n1, (seed, n0, n1)
