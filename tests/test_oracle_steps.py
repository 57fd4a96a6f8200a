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
