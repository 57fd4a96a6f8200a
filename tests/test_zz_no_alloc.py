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


def _field(seed, ny, nx):
    """A piecewise-constant displacement field with noise, small regions and
    outliers: (ux, uy, valid, outlier) as numpy arrays, and the packed device
    form (int32 u = ux | uy << 16, uint8 flags = valid | outlier << 1)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    blocks = rng.integers(-40, 41, size=(ny // 5 + 1, nx // 5 + 1, 2))
    u = np.repeat(np.repeat(blocks, 5, 0), 5, 1)[:ny, :nx]
    u = u + (rng.random((ny, nx, 2)) < 0.1) * rng.integers(-20, 21, size=(ny, nx, 2))
    ux, uy = u[..., 0].astype(np.int32), u[..., 1].astype(np.int32)
    valid = (rng.random((ny, nx)) > 0.03).astype(np.uint8)
    outl = (rng.random((ny, nx)) < 0.08).astype(np.uint8)
    packed = ((ux & 0xffff) | (uy.astype(np.int64) << 16)).astype(np.int64).astype(np.uint32)
    return ux, uy, valid, outl, packed.view(np.int32), (valid | (outl << 1)).astype(np.uint8)


def _noalloc(api, prm, ny, nx, du, dflags, rows, cnt):
    from paper_1704_03217_gb300 import _lib
    L = _lib.load()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return L.pgm_filter_noalloc(C.byref(prm.cstruct()), nx, ny, C.c_void_p(du.data_ptr()),
                                C.c_void_p(dflags.data_ptr()), C.c_void_p(rows.data_ptr()),
                                rows.shape[0], C.c_void_p(cnt.data_ptr()), stream)


def test_noalloc_filter_at_capacity(api):
    """A field of exactly PGM_NOALLOC_MAX_SEEDS seeds (1024 x 1024) fills the
    fixed scratch array (region labels, region sizes, scan block sums); its
    matches equal the oracle's region removal (Sec. III-E) and export (Sec.
    III-G) on the same arrays.  A smaller field follows in the next call."""
    import oracle as O
    from paper_1704_03217_gb300 import _lib
    prm = api.Params(seed_stride=3, min_region=9, region_dmax2=144)
    for seed, (ny, nx) in [(31, (1024, 1024)), (32, (301, 517))]:
        assert ny * nx <= _lib.NOALLOC_MAX_SEEDS
        ux, uy, va, ol, packed, flags = _field(seed, ny, nx)
        want, _ = O.filter_arrays(dict(seed_stride=3, min_region=9, region_dmax2=144),
                                  ux, uy, va, ol)
        du = torch.from_numpy(packed.copy()).cuda()
        df = torch.from_numpy(flags).cuda()
        rows = torch.full((nx * ny, 4), -7, dtype=torch.int32, device="cuda")
        cnt = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        assert _noalloc(api, prm, ny, nx, du, df, rows, cnt) == 0
        torch.cuda.synchronize()
        n = int(cnt.item())
        assert n == want.shape[0] and n > 1000
        assert (rows[:n].cpu().numpy() == want).all()


def test_noalloc_filter_allocates_nothing(api):
    """After a first call (which loads the library's module on the device and
    finds the array), further calls leave the device's free memory and the
    caching allocator's total unchanged."""
    prm = api.Params(seed_stride=3, min_region=9, region_dmax2=144)
    ux, uy, va, ol, packed, flags = _field(33, 600, 700)
    du = torch.from_numpy(packed.copy()).cuda()
    df = torch.from_numpy(flags).cuda()
    rows = torch.empty((600 * 700, 4), dtype=torch.int32, device="cuda")
    cnt = torch.zeros((1,), dtype=torch.int32, device="cuda")
    assert _noalloc(api, prm, 600, 700, du, df, rows, cnt) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(3):
        assert _noalloc(api, prm, 600, 700, du, df, rows, cnt) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0
