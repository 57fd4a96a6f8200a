"""The C-ABI library loads and exports every symbol include/pgm.h declares;
host-only queries and argument checks behave as documented.  No kernel is
launched (CPU only)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1704_03217_gb300 import build, _lib
    build.build()
    return _lib.load()


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"\b(pgm_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_exports_every_declared_symbol(lib):
    from paper_1704_03217_gb300 import _lib
    declared = _declared()
    assert len(declared) >= 13
    assert set(declared) == set(_lib.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name


def test_default_params_are_the_papers(lib):
    from paper_1704_03217_gb300 import _lib
    from paper_1704_03217_gb300.api import Params
    p = _lib.CParams()
    lib.pgm_default_params(C.byref(p))
    d = Params()
    for n, _ in _lib.PARAM_FIELDS:
        assert getattr(p, n) == getattr(d, n), n
    assert (p.levels, p.rs_W, p.sobel, p.refine_rounds, p.iters_coarse, p.iters_fine) == (3, 2, 5, 2, 4, 6)
    assert (p.patch_fwd, p.patch_bwd, p.min_region, p.region_dmax2) == (15, 11, 9, 144)
    assert p.philox_key == d.philox_key
    assert list(p.iters_level) == [-1] * 12 == list(d.cstruct().iters_level)


def test_status_strings(lib):
    for code in range(8):
        assert lib.pgm_status_string(code)
    assert lib.pgm_status_string(99) == b"unknown status"


def test_size_queries_and_argument_checks(lib):
    from paper_1704_03217_gb300.api import Params
    p = Params(levels=5, color=1).cstruct()
    assert lib.pgm_pyramid_bytes(C.byref(p), 1024, 436) > 2 * 1024 * 436 * 12
    assert lib.pgm_pyramid_bytes(C.byref(p), 0, 436) == 0
    ws = lib.pgm_match_workspace_bytes(C.byref(p), 1024, 436, 1024, 436)
    assert ws > 49445 * 13
    bad = Params(levels=13).cstruct()
    assert lib.pgm_pyramid_bytes(C.byref(bad), 64, 64) == 0
    assert lib.pgm_build_pyramid(C.byref(p), None, 64, 64, 3, 192, None, 0, None) == 1
    big = Params(patch_fwd=17).cstruct()
    assert lib.pgm_match(C.byref(big), C.c_void_p(256), C.c_void_p(512), 64, 64, 64, 64, 0,
                         C.c_void_p(1024), 1 << 30, None) == 7
    for lv in ((2, -2), (32768,)):              # per-level counts: -1 .. 32767
        bad_it = Params(iters_level=lv).cstruct()
        assert lib.pgm_match(C.byref(bad_it), C.c_void_p(256), C.c_void_p(512), 64, 64, 64, 64, 0,
                             C.c_void_p(1024), 1 << 30, None) == 1
    # workspace too small is reported before any launch
    assert lib.pgm_match(C.byref(p), C.c_void_p(256), C.c_void_p(512), 1024, 436, 1024, 436, 0,
                         C.c_void_p(1024), 16, None) == 3
    # a level without seeds
    tiny = Params(levels=5, seed_stride=3).cstruct()
    assert lib.pgm_match(C.byref(tiny), C.c_void_p(256), C.c_void_p(512), 4, 4, 4, 4, 0,
                         C.c_void_p(1024), 1 << 30, None) == 2
    # misaligned buffers
    assert lib.pgm_match(C.byref(p), C.c_void_p(257), C.c_void_p(512), 64, 64, 64, 64, 0,
                         C.c_void_p(1024), 1 << 30, None) == 1
    assert lib.pgm_filter(C.byref(p), 64, 64, 64, 64, None, 1 << 20, None, 0, None, None, None) == 1


def test_fault_injection_arguments(lib):
    """pgm_inject_launch_failure arms and disarms without touching the device;
    a negative step count is refused."""
    assert lib.pgm_inject_launch_failure(-1) == 1
    assert lib.pgm_inject_launch_failure(5) == 0
    assert lib.pgm_inject_launch_failure(0) == 0


def test_nominal_evals_match_hand_count(lib):
    """Hand count for 256x192, L = 3, stride 3, 6 iterations everywhere:
    lattices 85x64, 43x32, 21x16; visits 2,1,2,1,2,1,0; per seed and
    iteration 2 propagation + 2 search candidates, plus one cost per visit."""
    from paper_1704_03217_gb300.api import Params, nominal_evals
    p = Params(levels=3, color=0, patch_fwd=8, patch_bwd=8, iters_coarse=6, iters_fine=6)
    per_visit = {0: 85 * 64, 1: 43 * 32, 2: 21 * 16}
    want = sum(2 * per_visit[l] * (1 + 6 * 4) for l in [2, 1, 2, 1, 2, 1, 0])
    assert nominal_evals(p, 256, 192, 256, 192) == want


def test_noalloc_rejects_misaligned_pointers():
    """pgm_filter_noalloc checks its pointers before it touches the device: a
    displacement or count pointer that is not 4-byte aligned, or a match
    buffer that is not 16-byte aligned, gives PGM_ERR_ARG without a GPU."""
    from paper_1704_03217_gb300 import build, _lib
    build.build()
    L = _lib.load()
    cp = _lib.CParams()
    L.pgm_default_params(C.byref(cp))
    good = dict(u=4096, f=8192, m=16384, c=32768)
    for bad in (dict(u=4097), dict(u=4098), dict(c=32769), dict(m=16388)):
        a = dict(good, **bad)
        code = L.pgm_filter_noalloc(C.byref(cp), 8, 8, C.c_void_p(a["u"]), C.c_void_p(a["f"]),
                                    C.c_void_p(a["m"]), 64, C.c_void_p(a["c"]), None)
        assert code == 1, (bad, code)


def test_binding_refuses_pyramids_of_another_layout():
    """pgm_match and pgm_interpolate take pyramid buffers without their sizes,
    so the binding refuses, before calling the library, a pyramid built under
    other layout parameters or a buffer smaller than the layout (buffers in
    host memory here: nothing reaches the library's compute calls)."""
    import torch
    from paper_1704_03217_gb300 import api, build
    build.build()
    p = api.Params(levels=4, color=1)
    P1 = api.Pyramid(p, 64, 48, device="cpu")
    P2 = api.Pyramid(p, 64, 48, device="cpu")
    for other in (dict(levels=3), dict(color=0), dict(descriptor=1), dict(sobel=3),
                  dict(cs_sched=1)):
        q = p.replace(**other)
        with pytest.raises(ValueError, match=next(iter(other))):
            api.match(q, P1, P2)
        with pytest.raises(ValueError):
            api.match_batch(q, [P1], [P2], [0], [None])
        with pytest.raises(ValueError):
            api.interpolate(q, P1, torch.zeros((1, 4), dtype=torch.int32),
                            torch.zeros(1, dtype=torch.int32))
    # parameters that do not change the pyramid pass the check
    api.check_pyramids(p.replace(iters_fine=2, philox_key=7, patch_fwd=9, seed_stride=2), P1, P2)
    short = api.Pyramid(p, 64, 48, device="cpu")
    short.buf = short.buf[:-1]
    with pytest.raises(ValueError, match="needs"):
        api.match(p, P1, short)
    with pytest.raises(ValueError, match="length"):
        api.match_batch(p, [P1, P1], [P2], [0, 1], [None, None])
