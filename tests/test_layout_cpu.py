"""The buffer layouts the C ABI reports (pgm_pyramid_bytes,
pgm_pyramid_desc_layout, pgm_pyramid_image_layout, pgm_match_workspace_bytes,
pgm_field_layout) over a seeded sweep of image sizes and parameters, far
beyond the sizes the GPU tests run: every reported array lies inside its
buffer, arrays of different levels, directions and schemes never overlap
(except the documented aliases), alignments hold, and the level sizes and
seed lattices follow the pyramid (W_{l+1} = ceil(W_l / 2)) and lattice
(stride sigma, offset sigma // 2) definitions.  Host-only queries: no GPU."""
import ctypes as C

import numpy as np
import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_1704_03217_gb300 import build, _lib
    build.build()
    return _lib.load()


def _desc(L, cp, w, h, s, l):
    off, lw, lh, nch, row, px, bord = (C.c_size_t(), C.c_int(), C.c_int(), C.c_int(), C.c_int(),
                                       C.c_int(), C.c_int())
    assert L.pgm_pyramid_desc_layout(C.byref(cp), w, h, s, l, C.byref(off), C.byref(lw),
                                     C.byref(lh), C.byref(nch), C.byref(row), C.byref(px),
                                     C.byref(bord)) == 0
    return off.value, lw.value, lh.value, nch.value, row.value, px.value, bord.value


def _image(L, cp, w, h, s, l):
    off, lw, lh, ch, row, plane = (C.c_size_t(), C.c_int(), C.c_int(), C.c_int(), C.c_int(),
                                   C.c_size_t())
    assert L.pgm_pyramid_image_layout(C.byref(cp), w, h, s, l, C.byref(off), C.byref(lw),
                                      C.byref(lh), C.byref(ch), C.byref(row), C.byref(plane)) == 0
    return off.value, lw.value, lh.value, ch.value, row.value, plane.value


def _disjoint(spans, what):
    spans = sorted(set(spans))
    for (a0, a1), (b0, b1) in zip(spans, spans[1:]):
        assert a1 <= b0, (what, (a0, a1), (b0, b1))


def _configs(n=120):
    rng = np.random.default_rng(20260)
    for k in range(n):
        w = int(rng.integers(1, 5000)) if k % 3 else int(rng.integers(1, 80))
        h = int(rng.integers(1, 3000)) if k % 3 else int(rng.integers(1, 80))
        yield w, h, dict(levels=int(rng.integers(1, 7)), color=int(rng.integers(0, 2)),
                         descriptor=int(rng.integers(0, 3)), cs_sched=int(rng.integers(0, 2)),
                         seed_stride=int(rng.integers(1, 6)))


@pytest.mark.parametrize("w,h,prm", list(_configs()))
def test_pyramid_layout(lib, w, h, prm):
    from paper_1704_03217_gb300.api import Params
    cp = Params(**prm).cstruct()
    total = lib.pgm_pyramid_bytes(C.byref(cp), w, h)
    assert total > 0 and total % 256 == 0
    C_ = 3 if prm["color"] == 1 else 1
    two_schemes = prm["color"] == 1 and prm["cs_sched"] == 0
    descs, images = [], []
    W, H = w, h
    for l in range(prm["levels"]):
        for s in (0, 1):
            off, lw, lh, nch, row, px, bord = _desc(lib, cp, w, h, s, l)
            assert (lw, lh, nch) == (W, H, 2 * C_)
            assert px == (8 if C_ == 3 else 2) and row % 8 == 0 and row >= (lw + 2 * bord) * px
            start = off - 2 * (bord * row + bord * px)
            end = start + 2 * row * (lh + 2 * bord)
            assert start >= 0 and start % 256 == 0 and end <= total, (l, s)
            ioff, iw, ih, ch, irow, plane = _image(lib, cp, w, h, s, l)
            assert (iw, ih, ch) == (W, H, C_) and irow >= iw and irow % 16 == 0
            assert plane == irow * ih and ioff % 256 == 0 and ioff + ch * plane <= total
            if s == 1 and not two_schemes:          # one scheme serves both directions
                assert (off, ioff) == (descs[-1][0] + 2 * (bord * row + bord * px), images[-1][0])
                continue
            descs.append((start, end))
            images.append((ioff, ioff + ch * plane))
        W, H = (W + 1) // 2, (H + 1) // 2
    _disjoint(descs, "descriptors")
    # an image span is either a level's RGB / gray planes or a converted copy;
    # two schemes may share a level's planes (RGB in both), which set() merges
    _disjoint(images, "images")
    _disjoint(descs + images, "descriptors and images")


@pytest.mark.parametrize("w,h,prm", list(_configs(60)))
def test_workspace_layout(lib, w, h, prm):
    from paper_1704_03217_gb300.api import Params
    cp = Params(**prm).cstruct()
    w2, h2 = max(1, h * 3 // 4), max(1, w * 2 // 3)     # a pair of different sizes
    total = lib.pgm_match_workspace_bytes(C.byref(cp), w, h, w2, h2)
    assert total > 0
    sig = prm["seed_stride"]
    c = sig // 2
    spans = [(0, 72)]                                   # status word and counters
    dims = [(w, h), (w2, h2)]
    for l in range(prm["levels"]):
        for d in (0, 1):
            lw, lh = dims[d]
            nx, ny = C.c_int(), C.c_int()
            ou, oc, of = C.c_size_t(), C.c_size_t(), C.c_size_t()
            assert lib.pgm_field_layout(C.byref(cp), w, h, w2, h2, l, d, C.byref(nx), C.byref(ny),
                                        C.byref(ou), C.byref(oc), C.byref(of)) == 0
            want_nx = (lw - 1 - c) // sig + 1 if lw - 1 - c >= 0 else 0
            want_ny = (lh - 1 - c) // sig + 1 if lh - 1 - c >= 0 else 0
            assert (nx.value, ny.value) == (want_nx, want_ny), (l, d)
            n = nx.value * ny.value
            for off, size in ((ou.value, 4 * n), (oc.value, 8 * n), (of.value, n)):
                assert off % 256 == 0 and off + size <= total
                if size:
                    spans.append((off, off + size))
        dims = [((x + 1) // 2, (y + 1) // 2) for x, y in dims]
    _disjoint(spans, "fields")


def test_size_limits(lib):
    """Images up to 32767 pixels a side are accepted (the largest PGM-C
    pyramid is tens of GB, still addressed in 64 bits), one pixel more is
    refused; the layout at the limit stays inside its buffer."""
    from paper_1704_03217_gb300.api import Params
    cp = Params(levels=5, color=1).cstruct()
    big = lib.pgm_pyramid_bytes(C.byref(cp), 32767, 32767)
    assert big > 2 * 2 * 32767 * 32767 * 16                # descriptor + split copy, 2 schemes
    assert lib.pgm_pyramid_bytes(C.byref(cp), 32768, 64) == 0
    assert lib.pgm_pyramid_bytes(C.byref(cp), 64, 32768) == 0
    off, lw, lh, nch, row, px, bord = _desc(lib, cp, 32767, 32767, 1, 0)
    assert off + 2 * row * (lh + bord) <= big
    ws = lib.pgm_match_workspace_bytes(C.byref(cp), 32767, 32767, 32767, 32767)
    assert ws > 2 * 13 * ((32767 - 2) // 3 + 1) ** 2      # u, cost, flags per seed, 2 directions
    assert lib.pgm_match_workspace_bytes(C.byref(cp), 32768, 8, 8, 8) == 0
