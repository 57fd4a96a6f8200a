"""Pins of the CPU oracle's single steps against what the mathematics fixes:
published known-answer vectors, closed forms, floating-point definitions and
pure-Python brute force.  CPU only."""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
import brute

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLD, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


# ---- Philox4x32-10 (Salmon et al., SC'11) --------------------------------
def test_philox_known_answers():
    for r in _rows("philox4x32_10_kat.txt"):
        v = [int(x, 16) for x in r]
        assert O.philox4x32_10(v[0:4], v[4:6]).tolist() == v[6:10]


# ---- integer cube root (CIELab, reading R3) -------------------------------
def test_icbrt_exact():
    rng = np.random.default_rng(0)
    vals = [0, 1, 7, 8, 9, 26, 27, 28, 2 ** 48, 2 ** 48 - 1, 2 ** 48 + 1, 65536 ** 3 - 1]
    vals += [int(x) for x in rng.integers(0, 2 ** 48, size=2000, dtype=np.uint64)]
    for v in vals:
        c = O.icbrt(v)
        assert c ** 3 <= v < (c + 1) ** 3, v


# ---- colour spaces (readings R2, R3) -------------------------------------
def _all_colours():
    r, g, b = np.meshgrid(np.arange(256), np.arange(256), np.arange(256), indexing="ij")
    return np.stack([r, g, b], -1).reshape(-1, 3).astype(np.uint8)


def test_gray_and_ycrcb_vs_float_definition():
    rgb = _all_colours()
    f = rgb.astype(np.float64)
    y = 0.299 * f[:, 0] + 0.587 * f[:, 1] + 0.114 * f[:, 2]
    g = O.convert(O.SP_GRAY, rgb).astype(np.float64)
    assert np.abs(g - y).max() <= 0.51
    ycc = O.convert(O.SP_YCRCB, rgb).astype(np.float64)
    assert np.abs(ycc[:, 0] - y).max() <= 0.51
    yi = ycc[:, 0]                               # Cr, Cb are defined on the integer Y
    cr = np.clip((f[:, 0] - yi) * 0.713 + 128, 0, 255)
    cb = np.clip((f[:, 2] - yi) * 0.564 + 128, 0, 255)
    assert np.abs(ycc[:, 1] - cr).max() <= 0.52
    assert np.abs(ycc[:, 2] - cb).max() <= 0.52


def test_lab_vs_double_definition():
    rgb = _all_colours()
    f = rgb.astype(np.float64) / 255.0           # linear RGB (no companding, R3)
    M = np.array([[0.412453, 0.357580, 0.180423],
                  [0.212671, 0.715160, 0.072169],
                  [0.019334, 0.119193, 0.950227]])
    xyz = f @ M.T / M.sum(1)
    e = (6.0 / 29.0) ** 3
    ff = np.where(xyz > e, np.cbrt(xyz), xyz * (841.0 / 108.0) + 4.0 / 29.0)
    L = (116 * ff[:, 1] - 16) * 255 / 100
    a = 500 * (ff[:, 0] - ff[:, 1]) + 128
    b = 200 * (ff[:, 1] - ff[:, 2]) + 128
    ref = np.clip(np.stack([L, a, b], -1), 0, 255)
    lab = O.convert(O.SP_LAB, rgb).astype(np.float64)
    err = np.abs(lab - ref)
    assert err.max() <= 1.0, err.max()
    assert O.convert(O.SP_LAB, np.array([[255, 255, 255]], np.uint8)).tolist() == [[255, 128, 128]]
    assert O.convert(O.SP_LAB, np.array([[0, 0, 0]], np.uint8)).tolist() == [[0, 128, 128]]


# ---- image pyramid (reading R1) ------------------------------------------
def test_pyr_down_constant_and_bias():
    for w, h in [(1, 1), (7, 5), (16, 9)]:
        for v in (0, 37, 255):
            out = O.pyr_down(np.full((h, w), v, np.uint8))
            assert out.shape == ((h + 1) // 2, (w + 1) // 2) and (out == v).all()
    rng = np.random.default_rng(1)
    img = rng.integers(0, 200, size=(23, 31), dtype=np.uint8)
    assert (O.pyr_down(img + 55).astype(int) == O.pyr_down(img).astype(int) + 55).all()


def test_pyr_down_brute():
    rng = np.random.default_rng(2)
    k = [1, 4, 6, 4, 1]
    for h, w in [(9, 13), (4, 3), (1, 6)]:
        img = rng.integers(0, 256, size=(h, w), dtype=np.uint8)
        out = O.pyr_down(img)
        for y in range(out.shape[0]):
            for x in range(out.shape[1]):
                s = sum(k[i + 2] * k[j + 2] * int(img[brute.clamp(2 * y + j, 0, h - 1),
                                                    brute.clamp(2 * x + i, 0, w - 1)])
                        for i in range(-2, 3) for j in range(-2, 3))
                assert out[y, x] == (s + 128) >> 8


# ---- Sobel, Eq. 1 (reading R4) --------------------------------------------
def test_sobel_closed_forms():
    h, w = 12, 20
    for a in (1, 3, 12):
        ramp = np.tile((np.arange(w) * a).astype(np.uint8), (h, 1))
        for S, gain in ((5, 128), (3, 8)):
            gx, gy = O.sobel(ramp, S)
            R = S // 2
            assert (gx[:, R:w - R] == gain * a).all()
            assert (gy == 0).all()
            gx2, gy2 = O.sobel(np.ascontiguousarray(ramp.T), S)
            assert (gy2[R:w - R, :] == gain * a).all() and (gx2 == 0).all()
    gx, gy = O.sobel(np.full((7, 9), 200, np.uint8), 5)
    assert not gx.any() and not gy.any()
    step = np.zeros((10, 10), np.uint8); step[:, 5:] = 255
    gx, _ = O.sobel(step, 5)
    assert gx.max() == 255 * 3 * 16 and gx.min() == 0          # |G| <= 12240


def test_sobel_brute():
    rng = np.random.default_rng(3)
    img = rng.integers(0, 256, size=(8, 11), dtype=np.uint8)
    for S, d, s in ((5, [-1, -2, 0, 2, 1], [1, 4, 6, 4, 1]), (3, [-1, 0, 1], [1, 2, 1])):
        gx, gy = O.sobel(img, S)
        R = S // 2
        for y in range(8):
            for x in range(11):
                px = lambda i, j: int(img[brute.clamp(y + j, 0, 7), brute.clamp(x + i, 0, 10)])
                ex = sum(s[j + R] * d[i + R] * px(i, j) for i in range(-R, R + 1) for j in range(-R, R + 1))
                ey = sum(d[j + R] * s[i + R] * px(i, j) for i in range(-R, R + 1) for j in range(-R, R + 1))
                assert gx[y, x] == ex and gy[y, x] == ey


# ---- patch distance, Eq. 3 (readings R6, R7) ------------------------------
def test_patch_dist_brute():
    rng = np.random.default_rng(4)
    A = rng.integers(-12240, 12241, size=(6, 9, 12)).astype(np.int16)
    B = rng.integers(-12240, 12241, size=(6, 10, 11)).astype(np.int16)
    for P in (1, 2, 3, 5, 8):
        for norm in (0, 1):
            for a, b in [((0, 0), (10, 9)), ((4, 4), (5, 5)), ((11, 8), (0, 3)), ((6, 2), (9, 0))]:
                assert O.patch_dist(A, B, a, b, P, norm) == brute.patch_dist(A, B, a, b, P, norm)


def test_patch_dist_extremes_need_64_bits():
    A = np.full((6, 16, 16), 12240, np.int16)
    B = np.full((6, 16, 16), -12240, np.int16)
    assert O.patch_dist(A, B, (8, 8), (8, 8), 16, 0) == 16 * 16 * 6 * 24480 ** 2
    assert O.patch_dist(A, B, (8, 8), (8, 8), 16, 1) == 16 * 16 * 6 * 24480
    assert O.patch_dist(A, A, (3, 3), (3, 3), 7, 0) == 0


# ---- random-search offsets, Eq. 5 (reading R11) ---------------------------
def test_rs_offset_symmetric():
    for W in (1, 2, 3, 8):
        for k in range(4):
            rho = max(1, W >> k)
            assert O.rs_offset(0, k, W, 0) == -rho
            assert O.rs_offset(2 ** 32 - 1, k, W, 0) == rho
            rng = np.random.default_rng(W * 10 + k)
            rs = rng.integers(0, 2 ** 32, size=500, dtype=np.uint64)
            vals = [O.rs_offset(int(r), k, W, 0) for r in rs]
            assert min(vals) >= -rho and max(vals) <= rho
            assert vals == [brute.rs_offset(int(r), k, W, 0) for r in rs]


def test_rs_offset_literal_floor():
    rng = np.random.default_rng(5)
    for W in (1, 2, 5):
        for k in range(3):
            for r in [0, 1, 2 ** 31, 2 ** 32 - 1] + [int(x) for x in rng.integers(0, 2 ** 32, 300)]:
                R = Fraction(2 * r - (2 ** 32 - 1), 2 ** 32)       # R in (-1, 1)
                want = (R * W / 2 ** k).__floor__()
                assert O.rs_offset(r, k, W, 1) == want


# ---- inter-level transfer, Eq. 7-8 (hand-computed) ------------------------
def test_transfer_hand_cases():
    import ctypes as C
    for r in _rows("eq7_eq8_cases.txt"):
        kind, cells = r[0], r[1]
        want = [int(x) for x in r[3:7]]
        cs = [[int(v) for v in c.split(",")] for c in cells.split(";")]
        n = len(cs)
        ux = (C.c_int32 * n)(*[c[0] for c in cs]); uy = (C.c_int32 * n)(*[c[1] for c in cs])
        va = (C.c_uint8 * n)(*([1] * n)); ol = (C.c_uint8 * n)(*[c[2] for c in cs])
        out = (C.c_int32 * 4)()
        O.lib().orc_xfer_cell(1 if kind == "up" else 0, n, ux, uy, va, ol, 0, out)
        got = list(out)
        assert got[2:] == want[2:], (r, got)
        if want[2]:
            assert got[:2] == want[:2], (r, got)


# ---- uniform 8-sector angle descriptor (an extension) ---------------------
def test_sector_rule_against_angles():
    """The integer rule equals round(angle / 45 deg) mod 8 away from the sector
    boundaries (22.5 deg + k 45 deg; its tan(22.5) ~ 169/408 is within 1e-6);
    codes are 64 (cos, sin) of the sector centre, 45 on the diagonals."""
    import math
    code = {0: (64, 0), 1: (45, 45), 2: (0, 64), 3: (-45, 45), 4: (-64, 0), 5: (-45, -45),
            6: (0, -64), 7: (45, -45)}
    rng = np.random.default_rng(8)
    for gx, gy in rng.integers(-12240, 12241, size=(3000, 2)):
        gx, gy = int(gx), int(gy)
        if gx == 0 and gy == 0:
            continue
        ang = math.degrees(math.atan2(gy, gx)) % 360.0
        if abs(((ang - 22.5) % 45.0) - 22.5) > 22.49:          # within 0.01 deg of a boundary
            continue
        assert O.sector(gx, gy) == code[int(round(ang / 45.0)) % 8], (gx, gy)
    assert O.sector(0, 0) == (0, 0)
    assert O.sector(408, 169) == (64, 0) and O.sector(408, 170) == (45, 45)   # ties to the axis
    assert O.sector(-169, 408) == (0, 64) and O.sector(-170, 408) == (-45, 45)


def test_sector_pyramid_codes():
    """The descriptor mode 2 writes sector codes of the Sobel gradients."""
    rng = np.random.default_rng(9)
    img = rng.integers(0, 256, size=(12, 17), dtype=np.uint8)
    P0 = O.Pyramid(dict(levels=1, color=0, descriptor=0), img)
    P2 = O.Pyramid(dict(levels=1, color=0, descriptor=2), img)
    g, s = P0.desc(0, 0), P2.desc(0, 0)
    for y in range(12):
        for x in range(17):
            assert (s[0, y, x], s[1, y, x]) == O.sector(int(g[0, y, x]), int(g[1, y, x]))


# ---- Table 2 colour-space schedule and the level assembly (reading R1) ----
# Table 2 of the paper, written out here independently of the oracle: the
# colour space of each level (0, 1, 2) of the forward and the backward
# gradient pyramid; reading R1 repeats the three columns for L > 3.
TABLE2 = {0: (O.SP_RGB, O.SP_LAB, O.SP_YCRCB),       # forward pyramid
          1: (O.SP_LAB, O.SP_YCRCB, O.SP_RGB)}       # backward pyramid


def _brute_down(img):
    """One pyramid step by the definition (5-tap binomial, +128 >> 8,
    replicated border, even samples), vectorised over the output grid."""
    h, w = img.shape
    k = np.array([1, 4, 6, 4, 1], np.int64)
    ys = np.arange((h + 1) // 2)[:, None]
    xs = np.arange((w + 1) // 2)[None, :]
    s = np.zeros((ys.shape[0], xs.shape[1]), np.int64)
    for j in range(-2, 3):
        for i in range(-2, 3):
            yy = np.clip(2 * ys + j, 0, h - 1)
            xx = np.clip(2 * xs + i, 0, w - 1)
            s += k[j + 2] * k[i + 2] * img[yy, xx].astype(np.int64)
    return ((s + 128) >> 8).astype(np.uint8)


def test_brute_down_matches_loop_definition():
    rng = np.random.default_rng(12)
    img = rng.integers(0, 256, size=(7, 10), dtype=np.uint8)
    k = [1, 4, 6, 4, 1]
    out = _brute_down(img)
    for y in range(out.shape[0]):
        for x in range(out.shape[1]):
            s = sum(k[i + 2] * k[j + 2] * int(img[brute.clamp(2 * y + j, 0, 6), brute.clamp(2 * x + i, 0, 9)])
                    for i in range(-2, 3) for j in range(-2, 3))
            assert out[y, x] == (s + 128) >> 8


@pytest.mark.parametrize("L", [3, 6])
def test_table2_schedule_and_level_assembly(L):
    """Each level image of a colour pyramid is the RGB image pyramided by the
    binomial step (in RGB), then converted to the Table 2 space of its level
    and pyramid; the descriptor is the Sobel of that image, channels ordered
    Gx of each colour channel then Gy of each.  A swapped row, a level off by
    one or a conversion before the pyramid fails here."""
    rng = np.random.default_rng(20 + L)
    rgb = rng.integers(0, 256, size=(70, 83, 3), dtype=np.uint8)
    planes = [[rgb[..., c] for c in range(3)]]
    for _ in range(1, L):
        planes.append([_brute_down(p) for p in planes[-1]])
    prm = dict(levels=L, color=1, cs_sched=0, sobel=5)
    P = O.Pyramid(prm, rgb)
    assert P.schemes == 2 and P.channels == 3
    for scheme in (0, 1):
        for level in range(L):
            lv = np.stack(planes[level], -1)
            want = O.convert(TABLE2[scheme][level % 3], lv)
            got = np.moveaxis(P.cimage(scheme, level), 0, -1)
            assert got.shape == want.shape
            assert (got == want).all(), (scheme, level)
            d = P.desc(scheme, level)
            for c in range(3):
                gx, gy = O.sobel(np.ascontiguousarray(want[..., c]), 5)
                assert (d[c] == gx).all() and (d[3 + c] == gy).all(), (scheme, level, c)
    # the two properties the paper states for Table 2: within a pyramid any
    # two of the three levels differ in space, and per level the forward and
    # backward spaces differ
    for s in (0, 1):
        assert len(set(TABLE2[s])) == 3
    assert all(TABLE2[0][l] != TABLE2[1][l] for l in range(3))


def test_gray_and_plain_schedules():
    """PGM-G/GD: the image is converted to gray first and one gray pyramid
    serves both directions (reading R19); the plain schedule keeps RGB at every
    level."""
    rng = np.random.default_rng(31)
    rgb = rng.integers(0, 256, size=(41, 29, 3), dtype=np.uint8)
    g = O.convert(O.SP_GRAY, rgb)
    want = [g]
    for _ in range(2):
        want.append(_brute_down(want[-1]))
    P = O.Pyramid(dict(levels=3, color=0), rgb)
    assert P.schemes == 1 and P.channels == 1
    for l in range(3):
        assert (P.cimage(0, l)[0] == want[l]).all()
    Pp = O.Pyramid(dict(levels=3, color=1, cs_sched=1), rgb)
    assert Pp.schemes == 1
    lv = [rgb[..., c] for c in range(3)]
    for l in range(3):
        assert (np.moveaxis(Pp.cimage(0, l), 0, -1) == np.stack(lv, -1)).all()
        lv = [_brute_down(p) for p in lv]


# ---- direction-only descriptor G ./ |G| (reading R5) ----------------------
def test_direction_sign_closed_forms():
    """A ramp increasing along x has Gx > 0 and Gy = 0 everywhere (also at the
    replicated border), so its direction code is (+1, 0); a decreasing ramp
    gives (-1, 0); a ramp along y gives (0, +1); a constant gives 0 (0/0 := 0)."""
    h, w = 9, 14
    ramp = np.tile((np.arange(w) * 7).astype(np.uint8), (h, 1))
    for S in (3, 5):
        prm = dict(levels=1, color=0, descriptor=1, sobel=S)
        d = O.Pyramid(prm, ramp).desc(0, 0)
        assert (d[0] == 1).all() and (d[1] == 0).all()
        d = O.Pyramid(prm, ramp[:, ::-1].copy()).desc(0, 0)
        assert (d[0] == -1).all() and (d[1] == 0).all()
        d = O.Pyramid(prm, np.ascontiguousarray(ramp.T)).desc(0, 0)
        assert (d[0] == 0).all() and (d[1] == 1).all()
        d = O.Pyramid(prm, np.full((h, w), 77, np.uint8)).desc(0, 0)
        assert not d.any()


@pytest.mark.parametrize("color", [0, 1])
def test_direction_equals_sign_of_full_descriptor(color):
    """descriptor = 1 is exactly the elementwise sign of descriptor = 0, channel
    by channel, at every level and in both colour schemes."""
    rng = np.random.default_rng(40 + color)
    shape = (37, 52, 3) if color else (37, 52)
    img = rng.integers(0, 256, size=shape, dtype=np.uint8)
    full = O.Pyramid(dict(levels=3, color=color, descriptor=0), img)
    dirn = O.Pyramid(dict(levels=3, color=color, descriptor=1), img)
    for s in range(full.schemes):
        for l in range(3):
            f, d = full.desc(s, l), dirn.desc(s, l)
            assert set(np.unique(d)) <= {-1, 0, 1}
            assert (d == np.sign(f)).all(), (s, l)


# ---- region removal on given arrays (Sec. III-E, reading R16) -------------
def test_filter_arrays_vs_union_find():
    """The oracle's region removal on caller-supplied arrays agrees with the
    brute-force union-find, and its rows are (x, y, x + ux, y + uy) of the
    kept seeds in raster order."""
    class F:
        pass
    rng = np.random.default_rng(50)
    for ny, nx, dmax2, mreg in [(17, 23, 4, 3), (9, 40, 144, 9), (30, 30, 1, 2)]:
        blocks = rng.integers(-6, 7, size=(ny // 3 + 1, nx // 3 + 1, 2))
        u = np.repeat(np.repeat(blocks, 3, 0), 3, 1)[:ny, :nx]
        u = u + (rng.random((ny, nx, 2)) < 0.15) * rng.integers(-3, 4, size=(ny, nx, 2))
        ux, uy = u[..., 0].astype(np.int32), u[..., 1].astype(np.int32)
        va = (rng.random((ny, nx)) > 0.05).astype(np.uint8)
        ol = (rng.random((ny, nx)) < 0.1).astype(np.uint8)
        rows, keep = O.filter_arrays(dict(seed_stride=3, min_region=mreg, region_dmax2=dmax2),
                                     ux, uy, va, ol)
        f = F()
        f.nx, f.ny = nx, ny
        f.ux, f.uy = ux.ravel().tolist(), uy.ravel().tolist()
        f.valid, f.outl = va.ravel().tolist(), ol.ravel().tolist()
        want = brute.region_keep(f, dmax2, mreg)
        assert (keep == want).all()
        jj, ii = np.nonzero(want)
        x, y = 1 + 3 * ii, 1 + 3 * jj
        exp = np.stack([x, y, x + ux[jj, ii], y + uy[jj, ii]], -1)
        assert rows.shape == exp.shape and (rows == exp).all()
