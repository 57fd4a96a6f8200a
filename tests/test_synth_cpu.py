"""The seeded input generators and the accuracy measure (CPU only).  The
generators feed both the CUDA path and the oracle, and their ground-truth
flows are what the end-point errors, the checkerboard-versus-scan margins and
the autotuner's accuracy bounds are measured against, so each flow is checked
against its own images: frame 2 sampled at p + flow(p) reproduces frame 1 at
p (exactly for the integer shift, to rounding for the warps)."""
import numpy as np
import pytest
from scipy import ndimage

from paper_1704_03217_gb300 import evaluate, synth


def _pull(f2, flow, ys, xs):
    """Frame 2 sampled (bilinear) at p + flow(p) for the pixels (ys, xs)."""
    qx = xs + flow[ys, xs, 0]
    qy = ys + flow[ys, xs, 1]
    img = f2.astype(np.float64)
    if img.ndim == 2:
        return ndimage.map_coordinates(img, [qy, qx], order=1, mode="nearest")
    return np.stack([ndimage.map_coordinates(img[..., c], [qy, qx], order=1, mode="nearest")
                     for c in range(img.shape[2])], -1)


def _interior(flow, h, w, margin):
    ys, xs = np.mgrid[0:h, 0:w]
    qx, qy = xs + flow[..., 0], ys + flow[..., 1]
    ok = (qx >= margin) & (qx <= w - 1 - margin) & (qy >= margin) & (qy <= h - 1 - margin)
    ok &= (xs >= margin) & (xs <= w - 1 - margin) & (ys >= margin) & (ys <= h - 1 - margin)
    return ys[ok], xs[ok]


@pytest.mark.parametrize("dx,dy,ch", [(5, -3, 1), (-12, 7, 3), (0, 0, 1)])
def test_translate_pair_is_an_exact_shift(dx, dy, ch):
    f1, f2, flow = synth.translate_pair(4, 97, 61, dx, dy, channels=ch)
    assert f1.dtype == np.uint8 and flow.shape == (61, 97, 2)
    assert (flow[..., 0] == dx).all() and (flow[..., 1] == dy).all()
    h, w = 61, 97
    y0, y1 = max(0, -dy), min(h, h - dy)
    x0, x1 = max(0, -dx), min(w, w - dx)
    assert (f2[y0 + dy:y1 + dy, x0 + dx:x1 + dx] == f1[y0:y1, x0:x1]).all()


def test_noise_affine_flow_matches_its_images():
    f1, f2, flow = synth.noise_affine_pair(3)
    assert f1.shape == f2.shape == (192, 256) and flow.shape == (192, 256, 2)
    ys, xs = _interior(flow, 192, 256, 3)
    d = np.median(np.abs(_pull(f2, flow, ys, xs) - f1[ys, xs]))
    # the same flow one pixel off, either way, explains the images far worse
    for off in ((1, 0), (0, 1)):
        d_off = np.median(np.abs(_pull(f2, flow + np.float32(off), ys, xs) - f1[ys, xs]))
        assert d < 0.3 * d_off
    assert d < 5.0        # bilinear resampling twice (the generator, then here) of fine noise
    # the motion stays within the stated bounds: |t| <= 12 px, |theta| <= 3 degrees
    assert np.abs(flow).max() <= 12 * np.sqrt(2) + np.deg2rad(3) * np.hypot(128, 96) + 1e-3


def test_sintel_like_flow_matches_its_images_where_visible():
    f1, f2, flow = synth.sintel_like_pair(5, 320, 200, t_max=30.0, blur=False)
    again = synth.sintel_like_pair(5, 320, 200, t_max=30.0, blur=False)
    assert all((a == b).all() for a, b in zip((f1, f2, flow), again))       # seeded
    assert f1.shape == (200, 320, 3) and f1.dtype == np.uint8
    ys, xs = _interior(flow, 200, 320, 3)
    d = np.abs(_pull(f2, flow, ys, xs) - f1[ys, xs]).max(-1)
    d_off = np.abs(_pull(f2, flow + np.float32((1, 0)), ys, xs) - f1[ys, xs]).max(-1)
    # occlusions and layer edges break the equality, visible pixels keep it
    assert np.mean(d <= 8) > 0.8 and np.mean(d_off <= 8) < 0.3


def test_kitti_like_flow_is_the_stated_expansion():
    f1, f2, flow = synth.kitti_like_pair(2, 311, 94, max_disp=50.0)
    h, w = 94, 311
    corner = np.hypot(flow[0, 0, 0], flow[0, 0, 1])
    assert corner == pytest.approx(50.0, rel=1e-5)
    c = np.hypot(flow[h // 2, w // 2, 0], flow[h // 2, w // 2, 1])
    assert c < 1.0
    ys, xs = _interior(flow, h, w, 3)
    a = _pull(f2, flow, ys, xs).reshape(-1)
    b = f1[ys, xs].astype(np.float64).reshape(-1)
    gain, bias = np.polyfit(b, a, 1)                     # frame 2 = gain * frame 1 + bias
    assert 0.8 - 0.02 <= gain <= 1.2 + 0.02 and -20 - 2 <= bias <= 20 + 2
    a_off = _pull(f2, flow + np.float32((1, 0)), ys, xs).reshape(-1)
    assert np.corrcoef(a, b)[0, 1] > 0.98 > np.corrcoef(a_off, b)[0, 1]


def test_match_accuracy_by_hand():
    flow = np.zeros((10, 10, 2), np.float32)
    flow[..., 0] = 1.0
    rows = np.array([[2, 3, 3, 3],          # exact: EPE 0
                     [4, 4, 5, 8],          # off by (0, 4): EPE 4, an outlier
                     [1, 1, 5, 4]],         # (4, 3) against (1, 0): EPE sqrt(9 + 9)
                    np.int32)
    r = evaluate.match_accuracy(rows, flow, n_seeds=6)
    assert r["matches"] == 3 and r["density"] == 0.5
    assert r["epe"] == pytest.approx((0 + 4 + np.sqrt(18)) / 3)
    assert r["outliers_3px"] == pytest.approx(2 / 3)
    empty = evaluate.match_accuracy(np.zeros((0, 4), np.int32), flow, 6)
    assert empty["matches"] == 0 and np.isnan(empty["epe"])
