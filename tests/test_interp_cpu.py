"""Pins of the oracle's sparse-to-dense interpolation (Sec. III-G, readings
R23-R25) against independent definitions: per-source shortest paths from a
library graph routine, Manhattan distances for a constant cost, the constant
and affine fields that NW and LA must reproduce, and the paper's NW/LA
selection rule."""
import numpy as np
import pytest

import oracle as O

sp = pytest.importorskip("scipy.sparse")
csgraph = pytest.importorskip("scipy.sparse.csgraph")


def grid_graph(cost):
    """4-connected grid, edge p-q weighted cost[p] + cost[q]."""
    h, w = cost.shape
    idx = np.arange(h * w).reshape(h, w)
    c = cost.astype(np.float64).ravel()
    a = np.concatenate([idx[:, :-1].ravel(), idx[:-1, :].ravel()])
    b = np.concatenate([idx[:, 1:].ravel(), idx[1:, :].ravel()])
    wt = c[a] + c[b]
    g = sp.coo_matrix((np.concatenate([wt, wt]), (np.concatenate([a, b]), np.concatenate([b, a]))),
                      shape=(h * w, h * w))
    return g.tocsr()


def brute_knn(cost, sx, sy, K):
    h, w = cost.shape
    keep = []
    seen = set()
    for i, (x, y) in enumerate(zip(sx, sy)):        # a position given twice keeps the first index
        if (x, y) not in seen:
            seen.add((x, y))
            keep.append(i)
    D = csgraph.dijkstra(grid_graph(cost), indices=[int(sy[i]) * w + int(sx[i]) for i in keep])
    out = np.full((h * w, K), np.iinfo(np.uint64).max, np.uint64)
    for p in range(h * w):
        lst = sorted((int(D[r, p]), keep[r]) for r in range(len(keep)) if np.isfinite(D[r, p]))
        for k, (d, i) in enumerate(lst[:K]):
            out[p, k] = np.uint64((d << 32) | i)
    return out.reshape(h, w, K)


@pytest.mark.parametrize("seed,K", [(0, 1), (1, 3), (2, 5), (3, 8)])
def test_knn_equals_per_source_shortest_paths(seed, K):
    rng = np.random.default_rng(seed)
    h, w = 9 + seed, 13
    cost = rng.integers(1, 40, size=(h, w)).astype(np.uint32)
    n = 6 + seed
    sx = rng.integers(0, w, n).astype(np.int32)
    sy = rng.integers(0, h, n).astype(np.int32)
    sx[-1], sy[-1] = sx[0], sy[0]                   # one duplicate position
    got = O.interp_knn(cost, sx, sy, K)
    assert (got == brute_knn(cost, sx, sy, K)).all()


def test_constant_cost_gives_manhattan_distances():
    h, w, K = 11, 17, 4
    desc = np.zeros((2, h, w), np.int16)            # cost 1 everywhere: a step costs 2
    cost = O.interp_cost(desc, 6)
    assert (cost == 1).all()
    sx = np.array([0, 16, 8, 3, 12], np.int32)
    sy = np.array([0, 10, 5, 9, 2], np.int32)
    keys = O.interp_knn(cost, sx, sy, K)
    yy, xx = np.mgrid[0:h, 0:w]
    d = 2 * (np.abs(xx[..., None] - sx) + np.abs(yy[..., None] - sy))
    order = np.lexsort((np.broadcast_to(np.arange(5), d.shape), d), axis=-1)[..., :K]
    want = (np.take_along_axis(d, order, -1).astype(np.uint64) << np.uint64(32)) | order.astype(np.uint64)
    assert (keys == want).all()


def test_cost_is_one_plus_shifted_l1_magnitude():
    rng = np.random.default_rng(5)
    desc = rng.integers(-5000, 5000, size=(6, 7, 9)).astype(np.int16)
    for shift in (0, 4, 6):
        want = 1 + (np.abs(desc.astype(np.int64)).sum(0) >> shift)
        assert (O.interp_cost(desc, shift) == want).all()


def lattice_rows(w, h, fxy):
    ys, xs = np.mgrid[1:h:3, 1:w:3]
    xs, ys = xs.ravel(), ys.ravel()
    fx, fy = fxy(xs, ys)
    return np.stack([xs, ys, xs + fx, ys + fy], 1).astype(np.int32)


def test_single_match_gives_a_constant_field():
    desc = np.random.default_rng(1).integers(-900, 900, size=(2, 20, 30)).astype(np.int16)
    rows = np.array([[7, 9, 12, 4]], np.int32)
    for mode in (1, 2):
        _, flow, _ = O.interpolate(desc, rows, K=4, mode=mode)
        assert np.abs(flow - np.array([5, -5])).max() < 1e-12


def test_affine_flow_is_reproduced_by_la_not_by_nw():
    """Matches of an affine flow on a grid: the weighted affine fit returns
    that flow at every pixel; the weighted average does not."""
    w, h = 40, 31
    desc = np.random.default_rng(2).integers(-2000, 2000, size=(6, h, w)).astype(np.int16)
    desc[:, :, 20:] = 0                                 # textured left half, flat right half
    aff = lambda x, y: (x - 2 * y + 3, -x + y // 1 + 1)
    rows = lattice_rows(w, h, aff)
    yy, xx = np.mgrid[0:h, 0:w]
    _, la, used = O.interpolate(desc, rows, K=8, mode=2)
    assert used
    assert np.abs(la[..., 0] - (xx - 2 * yy + 3)).max() < 1e-6
    assert np.abs(la[..., 1] - (-xx + yy + 1)).max() < 1e-6
    _, nw, used = O.interpolate(desc, rows, K=8, mode=1)
    assert not used and np.abs(nw[..., 0] - (xx - 2 * yy + 3)).max() > 0.5


def test_nw_is_the_weighted_mean_of_the_neighbours():
    rng = np.random.default_rng(3)
    w, h, K, lam = 25, 18, 5, 7.0
    desc = rng.integers(-3000, 3000, size=(2, h, w)).astype(np.int16)
    rows = np.stack([rng.integers(0, w, 12), rng.integers(0, h, 12),
                     rng.integers(0, w, 12), rng.integers(0, h, 12)], 1).astype(np.int32)
    keys, flow, _ = O.interpolate(desc, rows, K=K, lam=lam, mode=1, shift=6)
    f = rows[:, 2:] - rows[:, :2]
    for y, x in ((0, 0), (17, 24), (9, 11)):
        k = keys[y, x][keys[y, x] != O.EMPTY_KEY]
        d = (k >> np.uint64(32)).astype(np.float64)
        i = (k & np.uint64(0xffffffff)).astype(np.int64)
        wt = np.exp(-d / lam)                           # any common factor cancels
        assert np.allclose(flow[y, x], (wt[:, None] * f[i]).sum(0) / wt.sum(), rtol=0, atol=1e-12)


def test_la_when_matches_exceed_the_paper_density():
    """Sec. III-G: LA with more than 2.2 % of the image size in matches, else NW
    (decided in integers: n * 10^4 > 220 w h)."""
    desc = np.zeros((2, 50, 50), np.int16)             # 2500 pixels: LA needs more than 55
    rng = np.random.default_rng(4)
    for n, la in ((55, False), (56, True)):
        rows = np.stack([rng.permutation(2500)[:n] % 50, rng.permutation(2500)[:n] // 50,
                         np.zeros(n), np.zeros(n)], 1).astype(np.int32)
        assert O.interpolate(desc, rows, K=3)[2] == la
