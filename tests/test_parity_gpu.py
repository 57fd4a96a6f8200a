"""Parity of the CUDA path (called through the C ABI) with the CPU oracle:
bit-exact on every integer result -- descriptors, colour-converted images,
fields of every level and direction (displacement, cost, flags), the kept
mask and the exported matches.  Sizes span several seed tiles and ragged
tails; the full-size Sintel- and KITTI-shaped pairs are compared whole."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle as O
from paper_1704_03217_gb300 import synth
from pgm_compare import assert_parity, compare_fields, compare_pyramid, run_both, run_gpu

C1 = dict(levels=3, seed_stride=3, patch_fwd=8, patch_bwd=8, color=0, iters_coarse=6,
          iters_fine=6, tau2=1)


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_03217_gb300 import build
    build.build()
    from paper_1704_03217_gb300 import api as A
    return A


def _rgb_pair(seed, w, h):
    f1, f2, _ = synth.sintel_like_pair(seed, w, h, t_max=min(150.0, w / 6))
    return f1, f2


@pytest.mark.parametrize("prm,shape", [
    (dict(levels=3, color=0), (192, 256)),
    (dict(levels=5, color=1), (436, 1024, 3)),
    (dict(levels=5, color=1, descriptor=1), (436, 1024, 3)),
    (dict(levels=4, color=0, sobel=3), (23, 37, 3)),          # RGB input -> gray
    (dict(levels=4, color=1, cs_sched=1, sobel=3), (31, 17, 3)),
    (dict(levels=6, color=1), (97, 131, 3)),                  # Table 2 cycled past level 2
])
def test_pyramid_parity(api, prm, shape):
    rng = np.random.default_rng(len(shape) * 100 + shape[0])
    img = rng.integers(0, 256, size=shape, dtype=np.uint8)
    p = api.Params(**prm)
    P = api.build_pyramid(p, torch.from_numpy(img).cuda())
    torch.cuda.synchronize()
    compare_pyramid(P, O.Pyramid(O.make_params(prm), img), str(prm))


@pytest.mark.parametrize("prm,shape", [
    (dict(levels=4, color=0), (157, 301)),       # level 2 is 76 x 40: h = 8 (mod 16)
    (dict(levels=3, color=1), (99, 211, 3)),
    (dict(levels=2, color=1), (24, 56, 3)),      # w = 24 (mod 32), h = 8 (mod 16)
    (dict(levels=2, color=0, descriptor=1), (40, 88)),
])
def test_descriptor_border(api, prm, shape):
    """The replicated border of the padded descriptor arrays (patches read
    outside the image take the nearest image pixel, Sec. III-B): every border
    pixel equals the oracle's descriptor at the clamped position."""
    rng = np.random.default_rng(shape[0] * 7 + shape[1])
    img = rng.integers(0, 256, size=shape, dtype=np.uint8)
    p = api.Params(**prm)
    P = api.build_pyramid(p, torch.from_numpy(img).cuda())
    torch.cuda.synchronize()
    Q = O.Pyramid(O.make_params(prm), img)
    for s in range(Q.schemes):
        for l in range(Q.levels):
            g = P.desc_padded(s, l).cpu().numpy()
            o = Q.desc(s, l).transpose(1, 2, 0)
            B = P.desc_layout(s, l)["border"]
            h, w = o.shape[:2]
            ys = np.clip(np.arange(-B, h + B), 0, h - 1)
            xs = np.clip(np.arange(-B, w + B), 0, w - 1)
            bad = np.argwhere((g != o[ys][:, xs]).any(-1))
            assert bad.size == 0, (prm, s, l, (bad[:5] - B).tolist())


def test_match_every_visit_c1(api):
    """256x192 gray (noise-affine workload): the state after each of the 7
    visits of the L = 3 schedule, at every level and in both directions."""
    f1, f2, _ = synth.noise_affine_pair(0)
    for v in range(1, 8):
        prm = dict(C1, max_visits=v)
        (_, _, ws, _, _), (_, _, M, _, _) = run_both(api, prm, f1, f2, stream_id=5)
        compare_fields(ws, M, 3, "visits=%d" % v)


@pytest.mark.parametrize("name,prm,size", [
    ("c1", C1, None),
    ("PGM-C", dict(levels=4, color=1), (384, 164)),
    ("PGM-CD", dict(levels=4, color=1, descriptor=1), (384, 164)),
    ("PGM-G", dict(levels=4, color=0), (301, 157)),
    ("PGM-GD", dict(levels=4, color=0, descriptor=1), (301, 157)),
    ("L1+floor", dict(levels=3, color=1, norm=1, rs_mode=1, rs_W=5), (200, 120)),
    ("plain-rgb", dict(levels=3, color=1, cs_sched=1, sobel=3, tau2=2), (211, 99)),
    ("dense", dict(levels=3, color=0, seed_stride=1, patch_fwd=5, patch_bwd=4), (96, 64)),
    ("stride2-even", dict(levels=3, color=0, seed_stride=2, patch_fwd=16, patch_bwd=6), (130, 94)),
    ("no-refine", dict(levels=4, color=0, ablation=1), (256, 140)),
    ("prop-all", dict(levels=4, color=0, ablation=2), (256, 140)),
    ("no-oprop", dict(levels=4, color=0, ablation=4, refine_rounds=3), (256, 140)),
    ("L1-level", dict(levels=1, color=0, patch_fwd=7, patch_bwd=5, iters_fine=3), (64, 48)),
    ("sector", dict(levels=4, color=1, descriptor=2), (384, 164)),
    ("sector-gray", dict(levels=4, color=0, descriptor=2), (301, 157)),
    ("C3-dense", dict(levels=3, color=1, seed_stride=1, rs_grid=3, patch_fwd=7, patch_bwd=5),
     (160, 96)),
    ("G3", dict(levels=4, color=0, rs_grid=3), (301, 157)),
    ("per-level-iters", dict(levels=4, color=1, iters_level=(3, 1, 5, 0)), (384, 164)),
])
def test_pipeline_parity(api, name, prm, size):
    if size is None:
        f1, f2, _ = synth.noise_affine_pair(1)
    elif prm.get("color", 1) == 1:
        f1, f2 = _rgb_pair(2, *size)
    else:
        f1, f2, _ = synth.noise_affine_pair(3, *size)
    assert_parity(api, prm, f1, f2, stream_id=11, what=name)


def test_different_sizes_pair(api):
    """I1 and I2 of different sizes (the ABI allows it)."""
    rng = np.random.default_rng(4)
    f1 = rng.integers(0, 256, size=(90, 120), dtype=np.uint8)
    f2 = rng.integers(0, 256, size=(77, 131), dtype=np.uint8)
    assert_parity(api, dict(levels=3, color=0, patch_fwd=7, patch_bwd=5), f1, f2, what="sizes")


def test_degenerate_constant_images(api):
    """All gradients zero: every cost is 0, so every choice is decided by the
    tie rules (lowest target raster index at init, strict improvement after)."""
    f1 = np.full((40, 52), 77, np.uint8)
    f2 = np.full((40, 52), 200, np.uint8)
    assert_parity(api, dict(levels=2, color=0, patch_fwd=5, patch_bwd=5), f1, f2, what="const")


def test_identity_pair(api):
    f1, _, _ = synth.noise_affine_pair(8, 160, 96)
    rows, M = assert_parity(api, dict(C1), f1, f1.copy(), what="identity")
    assert (rows[:, 0] == rows[:, 2]).all() and (rows[:, 1] == rows[:, 3]).all()


def test_tiny_images(api):
    rng = np.random.default_rng(5)
    for (h, w), prm in [((7, 9), dict(levels=1, seed_stride=1, patch_fwd=3, patch_bwd=3)),
                        ((11, 13), dict(levels=2, seed_stride=1, patch_fwd=4, patch_bwd=2)),
                        ((5, 5), dict(levels=1, seed_stride=3, patch_fwd=1, patch_bwd=1))]:
        f1 = rng.integers(0, 256, size=(h, w), dtype=np.uint8)
        f2 = rng.integers(0, 256, size=(h, w), dtype=np.uint8)
        assert_parity(api, dict(prm, color=0, iters_coarse=2, iters_fine=2, min_region=2), f1, f2,
                      what="tiny %dx%d" % (w, h))


@pytest.mark.slow
@pytest.mark.parametrize("cfg,prm", [
    ("c2", dict(levels=5, color=1, descriptor=0)),
    ("c2", dict(levels=5, color=0, descriptor=1)),
    ("c3", dict(levels=5, color=1, descriptor=1)),
    ("c3", dict(levels=5, color=0, descriptor=0)),
])
def test_full_size_parity(api, cfg, prm):
    """The 1024x436 Sintel-shaped and 1242x375 KITTI-shaped pairs, whole."""
    f1, f2, _ = synth.config_pair(cfg, 0)
    assert_parity(api, prm, f1, f2, stream_id=1, what=cfg + str(prm))


def test_batch_equals_single(api):
    """pgm_match_batch over pairs of different sizes gives each pair exactly
    what pgm_match gives it alone (and the oracle)."""
    prm = dict(levels=4, color=1)
    p = api.Params(**prm)
    pairs = [_rgb_pair(10 + k, w, h) for k, (w, h) in enumerate([(320, 240), (257, 131), (400, 150)])]
    P1 = [api.build_pyramid(p, torch.from_numpy(a).cuda()) for a, _ in pairs]
    P2 = [api.build_pyramid(p, torch.from_numpy(b).cuda()) for _, b in pairs]
    W = [api.Workspace(p, a.w, a.h, b.w, b.h) for a, b in zip(P1, P2)]
    api.match_batch(p, P1, P2, [7, 8, 9], W)
    for k in range(3):
        ws1 = api.match(p, P1[k], P2[k], stream_id=7 + k)
        torch.cuda.synchronize()
        for l in range(4):
            for d in (0, 1):
                a, b = W[k].field(l, d), ws1.field(l, d)
                for key in a:
                    assert torch.equal(a[key], b[key]), (k, l, d, key)
    op = O.make_params(prm)
    M = O.Match(op, O.Pyramid(op, pairs[1][0]), O.Pyramid(op, pairs[1][1]), 0, 8)
    compare_fields(W[1], M, 4, "batch")


def test_deterministic_and_stream_id(api):
    f1, f2, _ = synth.noise_affine_pair(12)
    a = run_gpu(api, C1, f1, f2, stream_id=3)
    b = run_gpu(api, C1, f1, f2, stream_id=3)
    c = run_gpu(api, C1, f1, f2, stream_id=4)
    assert (a[3] == b[3]).all()
    fa, fc = a[2].field(0, 0), c[2].field(0, 0)
    assert not (torch.equal(fa["ux"], fc["ux"]) and torch.equal(fa["uy"], fc["uy"]))


def test_max_matches_truncates(api):
    f1, f2, _ = synth.noise_affine_pair(13)
    _, _, ws, rows, _ = run_gpu(api, C1, f1, f2)
    p = api.Params(**C1)
    out = torch.zeros((17, 4), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    api.filter_into(p, ws, out, cnt)
    torch.cuda.synchronize()
    assert int(cnt.item()) == len(rows) and (out.cpu().numpy() == rows[:17]).all()


def test_batched_pyramid_and_filter_equal_single(api):
    """pgm_build_pyramid_batch / pgm_filter_batch over images of different
    sizes give each exactly what the single calls give."""
    prm = api.Params(levels=4, color=1)
    imgs = [_rgb_pair(30 + k, w, h)[k % 2] for k, (w, h) in
            enumerate([(320, 240), (257, 131), (400, 150), (199, 301)])]
    T = [torch.from_numpy(x).cuda() for x in imgs]
    batched = [api.Pyramid(prm, x.shape[1], x.shape[0]) for x in imgs]
    api.build_pyramids(prm, T, batched)
    single = [api.build_pyramid(prm, t) for t in T]
    torch.cuda.synchronize()
    for a, b in zip(batched, single):
        for s in range(2):
            for l in range(4):
                assert torch.equal(a.desc(s, l), b.desc(s, l))
                assert torch.equal(a.cimage(s, l), b.cimage(s, l))
    pairs = [(0, 2), (1, 3)]
    W = [api.match(prm, single[i], single[j], stream_id=k) for k, (i, j) in enumerate(pairs)]
    rows = [torch.full((w.layout(0, 0)[0] * w.layout(0, 0)[1], 4), -1, dtype=torch.int32,
                       device="cuda") for w in W]
    cnts = [torch.zeros(1, dtype=torch.int32, device="cuda") for _ in W]
    api.filter_batch(prm, W, rows, cnts)
    for w, r, c in zip(W, rows, cnts):
        want, _ = api.filter_matches(prm, w)
        torch.cuda.synchronize()
        n = int(c.item())
        assert n == want.shape[0] and torch.equal(r[:n], want)


def test_graph_replay_equals_eager(api):
    """A step captured as a CUDA graph and replayed on new images gives the
    same matches as eager launches on those images."""
    prm = api.Params(levels=4, color=1)
    a = [_rgb_pair(40 + k, 256, 160) for k in range(3)]
    t1 = [torch.from_numpy(x[0]).cuda() for x in a[:2]]
    t2 = [torch.from_numpy(x[1]).cuda() for x in a[:2]]
    m = api.PairMatcher(prm, 256, 160, batch=2)
    n = m.capture(t1, t2, [5, 6])
    assert n > 20
    t1[1].copy_(torch.from_numpy(a[2][0]))          # new content, same buffers
    t2[1].copy_(torch.from_numpy(a[2][1]))
    m.replay()
    torch.cuda.synchronize()
    got = [r.clone() for r in m.results()]
    e = api.PairMatcher(prm, 256, 160, batch=2)
    e.enqueue(t1, t2, [5, 6])
    torch.cuda.synchronize()
    want = e.results()
    for g, w in zip(got, want):
        assert torch.equal(g, w)
