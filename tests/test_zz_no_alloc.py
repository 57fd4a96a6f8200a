"""pgm_filter_noalloc -- the final filter for callers that cannot allocate
device memory (for example code running inside another framework's launch
callback, or under a memory budget fixed in advance) -- must give exactly what
pgm_filter gives on the same level-0 forward field.

Collected last on purpose: it runs after every other test, and it also passes
alone in a fresh process.  Two calls in a row, the second on a smaller field
than the first, check that the shared scratch array left by one call does not
leak into the next."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_03217_gb300 import build
    build.build()
    from paper_1704_03217_gb300 import api as A
    return A


def _field_ptrs(ws):
    nx, ny, off_u, _, off_flags = ws.layout(0, 0)
    base = ws.buf.data_ptr()
    return nx, ny, base + off_u, base + off_flags


def test_noalloc_filter_matches_pgm_filter(api):
    from paper_1704_03217_gb300 import _lib, synth
    L = _lib.load()
    prm = api.Params(levels=4, color=1)
    cp = prm.cstruct()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for seed, (w, h) in [(21, (512, 300)), (22, (256, 150))]:   # larger field first
        f1, f2, _ = synth.sintel_like_pair(seed, w, h, t_max=40.0)
        P1 = api.build_pyramid(prm, torch.from_numpy(f1).cuda())
        P2 = api.build_pyramid(prm, torch.from_numpy(f2).cuda())
        ws = api.match(prm, P1, P2, stream_id=seed)
        want, _ = api.filter_matches(prm, ws)
        nx, ny, pu, pf = _field_ptrs(ws)
        rows = torch.full((nx * ny, 4), -7, dtype=torch.int32, device="cuda")
        cnt = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        code = L.pgm_filter_noalloc(C.byref(cp), nx, ny, C.c_void_p(pu), C.c_void_p(pf),
                                    C.c_void_p(rows.data_ptr()), rows.shape[0],
                                    C.c_void_p(cnt.data_ptr()), stream)
        assert code == 0, _lib.STATUS.get(code)
        torch.cuda.synchronize()
        n = int(cnt.item())
        assert n == want.shape[0] and n > 0
        assert torch.equal(rows[:n], want)


def test_noalloc_filter_rejects_oversized_field(api):
    from paper_1704_03217_gb300 import _lib
    L = _lib.load()
    cp = api.Params().cstruct()
    side = 1025                                  # 1025 * 1025 > 2^20 seeds
    assert side * side > _lib.NOALLOC_MAX_SEEDS
    code = L.pgm_filter_noalloc(C.byref(cp), side, side, C.c_void_p(256), C.c_void_p(512),
                                C.c_void_p(1024), 16, C.c_void_p(2048), None)
    assert code == 7                             # PGM_ERR_UNSUPPORTED, nothing launched
