"""Python face of the plain CPU oracle (oracle/pgm_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / ``--impl reference`` leg may import this module;
the product package never does.  It shares no code with the CUDA library.

Parameters are passed as a plain ``dict`` with the field names of
``pgm_oracle.h``; missing fields take the paper's defaults (Sec. IV: W=2, S=5,
L=3, N=2, r=7 forward / r=5 backward, 4 iterations per level and 6 at full
resolution; region removal below 9 cells, Sec. III-E).
"""
import ctypes as C
import numpy as np

from . import build as _build

SCHED_CHECKERBOARD = 0
SCHED_SEQUENTIAL = 1
SP_GRAY, SP_RGB, SP_LAB, SP_YCRCB = 0, 1, 2, 3

FIELDS = [
    ("levels", 3), ("seed_stride", 3), ("patch_fwd", 15), ("patch_bwd", 11),
    ("sobel", 5), ("color", 0), ("descriptor", 0), ("cs_sched", 0), ("norm", 0),
    ("iters_coarse", 4), ("iters_fine", 6), ("refine_rounds", 2), ("rs_W", 2),
    ("rs_mode", 0), ("tau2", 1), ("min_region", 9), ("region_dmax2", 144),
    ("max_visits", 0), ("ablation", 0), ("rs_grid", 0),
]


class _Params(C.Structure):
    _fields_ = ([(n, C.c_int32) for n, _ in FIELDS] + [("philox_key", C.c_uint64)]
                + [("iters_level", C.c_int32 * 12)])


def make_params(d=None) -> _Params:
    d = dict(d or {})
    p = _Params()
    for n, default in FIELDS:
        setattr(p, n, int(d.pop(n, default)))
    p.philox_key = int(d.pop("philox_key", 0x5EED5EED1234ABCD))
    lv = list(d.pop("iters_level", ()))
    if len(lv) > 12:
        raise ValueError("iters_level: at most 12 levels")
    for l in range(12):
        p.iters_level[l] = int(lv[l]) if l < len(lv) else -1
    if d:
        raise KeyError("unknown oracle parameters: %s" % sorted(d))
    return p


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(_build.build())
        u8p, i16p, i32p, u32p, u64p = (C.POINTER(C.c_uint8), C.POINTER(C.c_int16),
                                       C.POINTER(C.c_int32), C.POINTER(C.c_uint32),
                                       C.POINTER(C.c_uint64))
        P = C.POINTER(_Params)
        L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.orc_icbrt.argtypes = [C.c_uint64]; L.orc_icbrt.restype = C.c_uint32
        L.orc_convert.argtypes = [C.c_int, u8p, C.c_int64, u8p]
        L.orc_pyr_down.argtypes = [u8p, C.c_int, C.c_int, u8p]
        L.orc_sobel.argtypes = [u8p, C.c_int, C.c_int, C.c_int, i16p, i16p]
        L.orc_patch_dist.argtypes = [i16p, C.c_int, C.c_int, i16p, C.c_int, C.c_int, C.c_int,
                                     C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]
        L.orc_patch_dist.restype = C.c_uint64
        L.orc_rs_offset.argtypes = [C.c_uint32, C.c_int, C.c_int, C.c_int]
        L.orc_rs_offset.restype = C.c_int32
        L.orc_sector.argtypes = [C.c_int, C.c_int, i16p]
        L.orc_pyr_build.argtypes = [P, u8p, C.c_int, C.c_int, C.c_int]
        L.orc_pyr_build.restype = C.c_void_p
        L.orc_pyr_free.argtypes = [C.c_void_p]
        for f in ("orc_pyr_levels", "orc_pyr_schemes", "orc_pyr_channels"):
            getattr(L, f).argtypes = [C.c_void_p]
        L.orc_pyr_dims.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.orc_pyr_image.argtypes = [C.c_void_p, C.c_int]; L.orc_pyr_image.restype = u8p
        L.orc_pyr_cimage.argtypes = [C.c_void_p, C.c_int, C.c_int]; L.orc_pyr_cimage.restype = u8p
        L.orc_pyr_desc.argtypes = [C.c_void_p, C.c_int, C.c_int]; L.orc_pyr_desc.restype = i16p
        L.orc_match_run.argtypes = [P, C.c_void_p, C.c_void_p, C.c_int, C.c_uint64]
        L.orc_match_run.restype = C.c_void_p
        L.orc_match_free.argtypes = [C.c_void_p]
        L.orc_match_visits.argtypes = [C.c_void_p]
        L.orc_match_visit_level.argtypes = [C.c_void_p, C.c_int]
        L.orc_match_evals.argtypes = [C.c_void_p]; L.orc_match_evals.restype = C.c_int64
        L.orc_field_dims.argtypes = [C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_int),
                                     C.POINTER(C.c_int)]
        L.orc_field_get.argtypes = [C.c_void_p, C.c_int, C.c_int, i32p, i32p, u8p, u64p, u8p, u8p]
        L.orc_filter.argtypes = [P, C.c_void_p, i32p, C.c_int64, u8p]
        L.orc_filter.restype = C.c_int64
        L.orc_filter_arrays.argtypes = [P, C.c_int, C.c_int, i32p, i32p, u8p, u8p, i32p,
                                        C.c_int64, u8p]
        L.orc_filter_arrays.restype = C.c_int64
        L.orc_interp_cost.argtypes = [i16p, C.c_int, C.c_int, C.c_int, C.c_int, u32p]
        L.orc_interp_knn.argtypes = [C.c_int, C.c_int, u32p, i32p, i32p, C.c_int64, C.c_int, u64p]
        L.orc_interp_knn.restype = C.c_int
        L.orc_interp_flow.argtypes = [C.c_int, C.c_int, C.c_int, u64p, i32p, i32p, i32p, i32p,
                                      C.c_double, C.c_int, C.POINTER(C.c_double)]
        _lib = L
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


# ---- single steps --------------------------------------------------------
def philox4x32_10(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    o = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_ptr(c, C.c_uint32), _ptr(k, C.c_uint32), _ptr(o, C.c_uint32))
    return o


def icbrt(v: int) -> int:
    return int(lib().orc_icbrt(int(v)))


def convert(space: int, rgb: np.ndarray) -> np.ndarray:
    rgb = np.ascontiguousarray(rgb, dtype=np.uint8)
    n = rgb.size // 3
    out = np.zeros(n * (1 if space == SP_GRAY else 3), np.uint8)
    lib().orc_convert(space, _ptr(rgb, C.c_uint8), n, _ptr(out, C.c_uint8))
    shp = rgb.shape[:-1]
    return out.reshape(shp if space == SP_GRAY else shp + (3,))


def pyr_down(img: np.ndarray) -> np.ndarray:
    img = np.ascontiguousarray(img, dtype=np.uint8)
    h, w = img.shape
    out = np.zeros(((h + 1) // 2, (w + 1) // 2), np.uint8)
    lib().orc_pyr_down(_ptr(img, C.c_uint8), w, h, _ptr(out, C.c_uint8))
    return out


def sobel(img: np.ndarray, S: int = 5):
    img = np.ascontiguousarray(img, dtype=np.uint8)
    h, w = img.shape
    gx = np.zeros((h, w), np.int16)
    gy = np.zeros((h, w), np.int16)
    lib().orc_sobel(_ptr(img, C.c_uint8), w, h, S, _ptr(gx, C.c_int16), _ptr(gy, C.c_int16))
    return gx, gy


def patch_dist(A, B, a, b, P, norm=0):
    """A, B: planar descriptors [nch][h][w] int16; a, b: (x, y) centres."""
    A = np.ascontiguousarray(A, dtype=np.int16)
    B = np.ascontiguousarray(B, dtype=np.int16)
    return int(lib().orc_patch_dist(_ptr(A, C.c_int16), A.shape[2], A.shape[1],
                                    _ptr(B, C.c_int16), B.shape[2], B.shape[1], A.shape[0],
                                    a[0], a[1], b[0], b[1], P, norm))


def sector(gx: int, gy: int):
    o = np.zeros(2, np.int16)
    lib().orc_sector(gx, gy, _ptr(o, C.c_int16))
    return int(o[0]), int(o[1])


def rs_offset(r: int, k: int, W: int, mode: int) -> int:
    return int(lib().orc_rs_offset(r, k, W, mode))


# ---- pyramid / match / filter --------------------------------------------
class Pyramid:
    """Gradient pyramid of one image (Sec. III-A, III-D, Table 2)."""

    def __init__(self, params, img: np.ndarray):
        self.params = params if isinstance(params, _Params) else make_params(params)
        img = np.ascontiguousarray(img, dtype=np.uint8)
        h, w = img.shape[:2]
        c = 1 if img.ndim == 2 else img.shape[2]
        self._img = img
        self.h = lib().orc_pyr_build(C.byref(self.params), _ptr(img, C.c_uint8), w, h, c)
        if not self.h:
            raise ValueError("oracle rejected the image/parameters")
        L = lib()
        self.levels = L.orc_pyr_levels(self.h)
        self.schemes = L.orc_pyr_schemes(self.h)
        self.channels = L.orc_pyr_channels(self.h)

    def dims(self, level):
        w, h = C.c_int(), C.c_int()
        lib().orc_pyr_dims(self.h, level, C.byref(w), C.byref(h))
        return w.value, h.value

    def image(self, level):
        w, h = self.dims(level)
        p = lib().orc_pyr_image(self.h, level)
        return np.ctypeslib.as_array(p, (self.channels, h, w)).copy()

    def cimage(self, scheme, level):
        w, h = self.dims(level)
        p = lib().orc_pyr_cimage(self.h, scheme, level)
        return np.ctypeslib.as_array(p, (self.channels, h, w)).copy()

    def desc(self, scheme, level):
        """[2C][h][w] int16: Gx of each channel, then Gy of each channel."""
        w, h = self.dims(level)
        p = lib().orc_pyr_desc(self.h, scheme, level)
        return np.ctypeslib.as_array(p, (2 * self.channels, h, w)).copy()

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_pyr_free(self.h)
            self.h = None


class Match:
    """Pyramidal matching of two pyramids (Sec. III-B, III-D)."""

    def __init__(self, params, p1: Pyramid, p2: Pyramid, schedule=SCHED_CHECKERBOARD,
                 stream_id=0):
        self.params = params if isinstance(params, _Params) else make_params(params)
        self._p1, self._p2 = p1, p2
        self.h = lib().orc_match_run(C.byref(self.params), p1.h, p2.h, schedule, stream_id)
        if not self.h:
            raise ValueError("oracle rejected the pyramids/parameters")

    @property
    def visits(self):
        L = lib()
        return [L.orc_match_visit_level(self.h, v) for v in range(L.orc_match_visits(self.h))]

    @property
    def evals(self):
        return int(lib().orc_match_evals(self.h))

    def dims(self, level, d):
        nx, ny = C.c_int(), C.c_int()
        lib().orc_field_dims(self.h, level, d, C.byref(nx), C.byref(ny))
        return nx.value, ny.value

    def field(self, level, d):
        """dict of (ny, nx) arrays: ux, uy, valid, cost, outlier, oinit."""
        nx, ny = self.dims(level, d)
        n = nx * ny
        ux = np.zeros(n, np.int32); uy = np.zeros(n, np.int32)
        va = np.zeros(n, np.uint8); co = np.zeros(n, np.uint64)
        ol = np.zeros(n, np.uint8); oi = np.zeros(n, np.uint8)
        lib().orc_field_get(self.h, level, d, _ptr(ux, C.c_int32), _ptr(uy, C.c_int32),
                            _ptr(va, C.c_uint8), _ptr(co, C.c_uint64), _ptr(ol, C.c_uint8),
                            _ptr(oi, C.c_uint8))
        r = lambda a: a.reshape(ny, nx)
        return {"ux": r(ux), "uy": r(uy), "valid": r(va), "cost": r(co),
                "outlier": r(ol), "oinit": r(oi)}

    def filter(self):
        """(rows [n][4] int32, keep mask (ny, nx) uint8) of the final filter."""
        nx, ny = self.dims(0, 0)
        keep = np.zeros(nx * ny, np.uint8)
        rows = np.zeros((max(nx * ny, 1), 4), np.int32)
        n = lib().orc_filter(C.byref(self.params), self.h, _ptr(rows, C.c_int32), nx * ny,
                             _ptr(keep, C.c_uint8))
        return rows[:n].copy(), keep.reshape(ny, nx)

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_match_free(self.h)
            self.h = None


def filter_arrays(params, ux, uy, valid, outlier):
    """Region removal and export (Sec. III-E, III-G) on a level-0 forward
    field given as (ny, nx) arrays: (rows [n][4] int32, keep (ny, nx) uint8)."""
    p = params if isinstance(params, _Params) else make_params(params)
    ny, nx = ux.shape
    ux = np.ascontiguousarray(ux, np.int32); uy = np.ascontiguousarray(uy, np.int32)
    va = np.ascontiguousarray(valid, np.uint8); ol = np.ascontiguousarray(outlier, np.uint8)
    rows = np.zeros((max(nx * ny, 1), 4), np.int32)
    keep = np.zeros(nx * ny, np.uint8)
    n = lib().orc_filter_arrays(C.byref(p), nx, ny, _ptr(ux, C.c_int32), _ptr(uy, C.c_int32),
                                _ptr(va, C.c_uint8), _ptr(ol, C.c_uint8), _ptr(rows, C.c_int32),
                                nx * ny, _ptr(keep, C.c_uint8))
    return rows[:n].copy(), keep.reshape(ny, nx)


def run_pair(params, img1, img2, schedule=SCHED_CHECKERBOARD, stream_id=0):
    """Whole path on one pair: (Pyramid1, Pyramid2, Match, rows)."""
    p = params if isinstance(params, _Params) else make_params(params)
    P1, P2 = Pyramid(p, img1), Pyramid(p, img2)
    M = Match(p, P1, P2, schedule, stream_id)
    rows, _ = M.filter()
    return P1, P2, M, rows


# ---- sparse-to-dense interpolation (Sec. III-G, readings R23-R25) ----------
EMPTY_KEY = np.uint64(0xFFFFFFFFFFFFFFFF)


def interp_cost(desc, shift=10):
    """desc: (nch, h, w) int16 -> (h, w) uint32 step costs (R23)."""
    d = np.ascontiguousarray(desc, dtype=np.int16)
    nch, h, w = d.shape
    out = np.zeros((h, w), np.uint32)
    lib().orc_interp_cost(_ptr(d, C.c_int16), nch, w, h, shift, _ptr(out, C.c_uint32))
    return out


def interp_knn(cost, sx, sy, K):
    """(h, w, K) uint64 keys d << 32 | match index of the K geodesically
    nearest matches (R24)."""
    c = np.ascontiguousarray(cost, dtype=np.uint32)
    h, w = c.shape
    sx = np.ascontiguousarray(sx, dtype=np.int32)
    sy = np.ascontiguousarray(sy, dtype=np.int32)
    keys = np.zeros((h, w, K), np.uint64)
    if lib().orc_interp_knn(w, h, _ptr(c, C.c_uint32), _ptr(sx, C.c_int32), _ptr(sy, C.c_int32),
                            len(sx), K, _ptr(keys, C.c_uint64)) != 0:
        raise MemoryError("orc_interp_knn")
    return keys


def interp_flow(keys, sx, sy, fx, fy, lam, use_la):
    """(h, w, 2) float64 flow from the K nearest matches (R25)."""
    k = np.ascontiguousarray(keys, dtype=np.uint64)
    h, w, K = k.shape
    a = [np.ascontiguousarray(v, dtype=np.int32) for v in (sx, sy, fx, fy)]
    out = np.zeros((h, w, 2), np.float64)
    lib().orc_interp_flow(w, h, K, _ptr(k, C.c_uint64), *[_ptr(v, C.c_int32) for v in a],
                          float(lam), int(use_la), _ptr(out, C.c_double))
    return out


def interpolate(desc, rows, K=16, lam=32.0, shift=10, mode=0, la_permyriad=220):
    """The whole interpolation of exported rows (x1, y1, x2, y2) over the
    reference image of desc (nch, h, w): (keys, flow, use_la).  mode 0
    chooses LA when the matches exceed la_permyriad / 10^4 of the pixels
    (the paper's rule: 2.2 %), 1 forces NW, 2 forces LA."""
    rows = np.asarray(rows, dtype=np.int32).reshape(-1, 4)
    nch, h, w = np.asarray(desc).shape
    use_la = (len(rows) * 10000 > la_permyriad * w * h) if mode == 0 else (mode == 2)
    cost = interp_cost(desc, shift)
    sx, sy = rows[:, 0], rows[:, 1]
    keys = interp_knn(cost, sx, sy, K)
    flow = interp_flow(keys, sx, sy, rows[:, 2] - rows[:, 0], rows[:, 3] - rows[:, 1], lam, use_la)
    return keys, flow, bool(use_la)
