"""Seeded synthetic image pairs shaped like the paper's benchmarks.

This module only makes inputs: it holds none of the matching method's
arithmetic, so the CUDA path and the CPU oracle can both be fed from it.
MPI Sintel and KITTI are not available here; these generators stand in for
them with the same image shapes and similar motion statistics:

* ``noise_affine_pair`` -- 256x192 gray, Gaussian-smoothed uniform noise
  (sigma 1.5), frame 2 = frame 1 under a known affine flow (translation up to
  12 px, rotation up to 3 degrees), bilinear sampling, rounded to uint8.
* ``translate_pair`` -- an exact integer shift (crop of one larger texture).
* ``sintel_like_pair`` -- 1024x436 RGB: 3-6 layered, textured, convex polygons
  over a noise background, each moving rigidly (translation up to 150 px, small
  rotation and scale), occlusion by layer order, optional motion blur.
* ``kitti_like_pair`` -- 1242x375 RGB road-plane texture, forward ego-motion
  expansion flow about the image centre (up to 200 px at the borders) and a
  gain 0.8-1.2 / bias +-20 illumination change on frame 2.

Every function returns ``(frame1, frame2, flow)``: uint8 images (H, W) or
(H, W, 3) and the ground-truth flow of frame-1 pixels, float32 (H, W, 2).
"""
import numpy as np
from scipy import ndimage


def _smooth_noise(rng, h, w, sigma, channels=1):
    """Uniform noise smoothed by a Gaussian and stretched to 0..255."""
    out = []
    for _ in range(channels):
        n = rng.uniform(0.0, 255.0, size=(h, w))
        s = ndimage.gaussian_filter(n, sigma, mode="reflect")
        lo, hi = np.percentile(s, 0.5), np.percentile(s, 99.5)
        out.append(np.clip((s - lo) * (255.0 / max(hi - lo, 1e-6)), 0, 255))
    return out[0] if channels == 1 else np.stack(out, axis=-1)


def _sample(img, ys, xs):
    """Bilinear sampling with edge replication; img (H, W) or (H, W, C)."""
    if img.ndim == 2:
        return ndimage.map_coordinates(img, [ys, xs], order=1, mode="nearest")
    return np.stack([ndimage.map_coordinates(img[..., c], [ys, xs], order=1, mode="nearest")
                     for c in range(img.shape[2])], axis=-1)


def _to_u8(a):
    return np.clip(np.rint(a), 0, 255).astype(np.uint8)


def noise_affine_pair(seed, w=256, h=192, t_max=12.0, rot_max_deg=3.0, sigma=1.5):
    rng = np.random.default_rng(seed)
    f1 = _smooth_noise(rng, h, w, sigma)
    tx, ty = rng.uniform(-t_max, t_max, size=2)
    th = np.deg2rad(rng.uniform(-rot_max_deg, rot_max_deg))
    cx, cy = (w - 1) / 2.0, (h - 1) / 2.0
    c, s = np.cos(th), np.sin(th)
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    # frame-1 point p moves to R (p - c) + c + t; frame 2 samples the inverse
    qx, qy = xx - cx - tx, yy - cy - ty
    px = c * qx + s * qy + cx
    py = -s * qx + c * qy + cy
    f2 = _sample(f1, py, px)
    fx = c * (xx - cx) - s * (yy - cy) + cx + tx - xx
    fy = s * (xx - cx) + c * (yy - cy) + cy + ty - yy
    return _to_u8(f1), _to_u8(f2), np.stack([fx, fy], -1).astype(np.float32)


def translate_pair(seed, w, h, dx, dy, channels=1, sigma=1.5):
    """frame2(q) = frame1(q - d) exactly, both cropped from one texture."""
    rng = np.random.default_rng(seed)
    m = int(max(abs(dx), abs(dy))) + 4
    big = _smooth_noise(rng, h + 2 * m, w + 2 * m, sigma, channels)
    f1 = big[m:m + h, m:m + w]
    f2 = big[m - dy:m - dy + h, m - dx:m - dx + w]
    flow = np.zeros((h, w, 2), np.float32)
    flow[..., 0], flow[..., 1] = dx, dy
    return _to_u8(f1), _to_u8(f2), flow


def _convex_polygon(rng, cx, cy, radius):
    k = int(rng.integers(5, 9))
    ang = np.sort(rng.uniform(0, 2 * np.pi, size=k))
    rad = radius * rng.uniform(0.75, 1.0, size=k)
    return np.stack([cx + rad * np.cos(ang), cy + rad * np.sin(ang)], -1)


def _inside_convex(poly, xs, ys):
    """Intersection of the half-planes left of each counter-clockwise edge."""
    inside = np.ones(xs.shape, bool)
    k = len(poly)
    for i in range(k):
        x0, y0 = poly[i]
        x1, y1 = poly[(i + 1) % k]
        inside &= ((x1 - x0) * (ys - y0) - (y1 - y0) * (xs - x0)) >= 0
    return inside


def sintel_like_pair(seed, w=1024, h=436, t_max=150.0, blur=True, rgb=True):
    rng = np.random.default_rng(seed)
    ch = 3 if rgb else 1
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    # background: textured noise with a small global translation
    bg = _smooth_noise(rng, h, w, rng.uniform(1.0, 2.5), ch)
    bt = rng.uniform(-8, 8, size=2)
    f1 = bg.copy()
    f2 = _sample(bg, yy - bt[1], xx - bt[0])
    flow = np.zeros((h, w, 2))
    flow[..., 0], flow[..., 1] = bt
    nl = int(rng.integers(3, 7))
    cover2 = np.zeros((h, w), bool)
    for _ in range(nl):                      # later layers are in front
        tex = _smooth_noise(rng, h, w, rng.uniform(0.8, 2.0), ch)
        if rgb:
            tex = np.clip(tex * rng.uniform(0.5, 1.0, size=3) + rng.uniform(0, 80, size=3), 0, 255)
        r = rng.uniform(0.12, 0.3) * min(w, h)
        cx, cy = rng.uniform(r, w - r), rng.uniform(r, h - r)
        poly = _convex_polygon(rng, cx, cy, r)
        t = rng.uniform(-t_max, t_max, size=2)
        th = np.deg2rad(rng.uniform(-4, 4))
        sc = rng.uniform(0.93, 1.07)
        c, s = sc * np.cos(th), sc * np.sin(th)
        # frame 1: the polygon in place, texture sampled directly
        in1 = _inside_convex(poly, xx, yy)
        f1 = np.where(in1[..., None] if rgb else in1, tex, f1)
        fx = c * (xx - cx) - s * (yy - cy) + cx + t[0] - xx
        fy = s * (xx - cx) + c * (yy - cy) + cy + t[1] - yy
        flow[in1, 0] = fx[in1]
        flow[in1, 1] = fy[in1]
        # frame 2: pull back each pixel through the inverse similarity
        det = c * c + s * s
        qx, qy = xx - cx - t[0], yy - cy - t[1]
        px = (c * qx + s * qy) / det + cx
        py = (-s * qx + c * qy) / det + cy
        in2 = _inside_convex(poly, px, py)
        moved = _sample(tex, py, px)
        f2 = np.where(in2[..., None] if rgb else in2, moved, f2)
        cover2 |= in2
    if blur:                                  # final-pass-like mild motion blur
        f2 = ndimage.uniform_filter1d(f2, size=3, axis=1)
    return _to_u8(f1), _to_u8(f2), flow.astype(np.float32)


def kitti_like_pair(seed, w=1242, h=375, max_disp=200.0, rgb=True):
    rng = np.random.default_rng(seed)
    ch = 3 if rgb else 1
    # road-plane texture: fine noise plus lane-like stripes, slight tint
    tex = _smooth_noise(rng, h, w, rng.uniform(0.8, 1.6), ch)
    stripes = 40.0 * (np.sin(np.arange(w) * rng.uniform(0.02, 0.05))[None, :] > 0.7)
    tex = np.clip(tex * 0.8 + (stripes[..., None] if rgb else stripes), 0, 255)
    cx, cy = (w - 1) / 2.0, (h - 1) / 2.0
    rmax = np.hypot(cx, cy)
    k = max_disp / rmax                       # u(p) = k (p - c): expansion
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    f1 = tex
    f2 = _sample(tex, cy + (yy - cy) / (1 + k), cx + (xx - cx) / (1 + k))
    gain, bias = rng.uniform(0.8, 1.2), rng.uniform(-20, 20)
    f2 = f2 * gain + bias
    flow = np.stack([k * (xx - cx), k * (yy - cy)], -1)
    return _to_u8(f1), _to_u8(f2), flow.astype(np.float32)


def config_pair(name, seed):
    """The named workload shapes: 'c1' 256x192 gray, 'c2' 1024x436 RGB,
    'c3' 1242x375 RGB."""
    if name == "c1":
        return noise_affine_pair(seed)
    if name == "c2":
        return sintel_like_pair(seed)
    if name == "c3":
        return kitti_like_pair(seed)
    raise KeyError(name)


BATCH_SIZES = [(320, 240), (640, 480), (1024, 436), (1242, 375), (1920, 1080)]


def mixed_batch(seed, n=64, sizes=BATCH_SIZES):
    """n pairs of sizes drawn uniformly from ``sizes``, made as Sintel-like
    (odd draws) or noise-affine (even draws) pairs."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        w, h = sizes[int(rng.integers(len(sizes)))]
        s = int(rng.integers(1 << 30))
        if i % 2:
            out.append(sintel_like_pair(s, w, h, t_max=min(150.0, w / 8)))
        else:
            f1, f2, fl = noise_affine_pair(s, w, h)
            out.append((np.repeat(f1[..., None], 3, -1), np.repeat(f2[..., None], 3, -1), fl))
    return out
