"""Host logic of bench.py's stage accounting (CPU only): the visit order it
assumes is the oracle's schedule (Fig. 5 as read in R15), and the pyramid
stage's compulsory bytes equal the descriptor and split-copy sizes the C ABI
reports through its layout queries, plus the input images."""
import ctypes as C
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench
import oracle as O


@pytest.mark.parametrize("levels,rounds", [(1, 2), (2, 0), (3, 2), (4, 1), (5, 2), (5, 3)])
def test_visit_levels_follow_the_oracle_schedule(levels, rounds):
    rng = np.random.default_rng(levels * 10 + rounds)
    img = rng.integers(0, 256, size=(40, 56), dtype=np.uint8)
    prm = dict(levels=levels, color=0, refine_rounds=rounds, patch_fwd=3, patch_bwd=3,
               iters_coarse=1, iters_fine=1)
    p = O.make_params(prm)
    M = O.Match(p, O.Pyramid(p, img), O.Pyramid(p, img))
    assert bench.visit_levels(levels, rounds) == M.visits


def test_pyramid_bytes_match_the_abi_layout():
    from paper_1704_03217_gb300 import api, build, _lib
    build.build()
    L = _lib.load()
    prm = api.Params(**bench.PARAMS)
    cp = prm.cstruct()
    w, h, pairs = bench.W_IMG, bench.H_IMG, 3
    desc = 0
    for scheme in (0, 1):
        for level in range(bench.PARAMS["levels"]):
            off, lw, lh, nch, row = C.c_size_t(), C.c_int(), C.c_int(), C.c_int(), C.c_int()
            pxe, bord = C.c_int(), C.c_int()
            assert L.pgm_pyramid_desc_layout(C.byref(cp), w, h, scheme, level, C.byref(off),
                                             C.byref(lw), C.byref(lh), C.byref(nch),
                                             C.byref(row), C.byref(pxe), C.byref(bord)) == 0
            desc += lw.value * lh.value * nch.value * 2      # int16 descriptor
    want = 2 * pairs * (3 * w * h + 2 * desc)              # + the split copy, + the input
    got = bench.hbm_stage_bytes(bench.PARAMS, w, h, pairs, 0)["pyramid"]
    assert got == want


def test_lattice_sizes_match_the_abi_field_layout():
    """The seed counts bench.py scales the traffic record with are the
    lattice sizes of the C ABI's field layout at every level."""
    from paper_1704_03217_gb300 import api, build, _lib
    build.build()
    L = _lib.load()
    for w, h in ((1024, 436), (1242, 375), (257, 193)):
        prm = api.Params(**bench.PARAMS)
        cp = prm.cstruct()
        n = bench.lattice_sizes(bench.PARAMS, w, h)
        for level in range(bench.PARAMS["levels"]):
            nx, ny = C.c_int(), C.c_int()
            o1, o2, o3 = C.c_size_t(), C.c_size_t(), C.c_size_t()
            assert L.pgm_field_layout(C.byref(cp), w, h, w, h, level, 0, C.byref(nx), C.byref(ny),
                                      C.byref(o1), C.byref(o2), C.byref(o3)) == 0
            assert n[level] == nx.value * ny.value


def test_paper_timings_are_the_table_3_figures():
    """The paper's per-pair times quoted beside the measurements: each variant
    on both datasets, the direction-only variants faster than their
    full-gradient twins as Table 3 has them."""
    t = bench.PAPER_TIMINGS["s_per_pair"]
    assert set(t) == {"PGM-C", "PGM-G", "PGM-CD", "PGM-GD", "PGM-C3", "PGM-G3"}
    assert t["PGM-C"] == {"sintel": 3.49, "kitti2012": 4.55}
    for full, fast in (("PGM-C", "PGM-CD"), ("PGM-G", "PGM-GD"), ("PGM-C", "PGM-C3"),
                       ("PGM-G", "PGM-G3")):
        assert all(t[fast][d] < t[full][d] for d in ("sintel", "kitti2012"))
    import json
    json.dumps(bench.PAPER_TIMINGS)


def test_optional_section_reports_failures_in_place(capsys):
    """A supplementary measurement that raises is reported in its place in the
    line (and on stderr) instead of ending the run; one that works returns
    its value."""
    assert bench.optional_section("ok", lambda: {"x": 1}) == {"x": 1}

    def broken():
        raise RuntimeError("CUDA out of memory")
    r = bench.optional_section("serving", broken)
    assert r == {"error": "serving: RuntimeError: CUDA out of memory"}
    assert "CUDA out of memory" in capsys.readouterr().err
