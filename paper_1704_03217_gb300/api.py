"""Python face of libpgm: argument marshalling only.

PyTorch provides device memory and streams; every step of the method runs in
the library's CUDA kernels (include/pgm.h).  There is no CPU path.
"""
import ctypes as C
from dataclasses import dataclass, fields, asdict

import torch

from . import _lib
from ._lib import check


@dataclass
class Params:
    """Method parameters (field meaning: include/pgm.h, pgm_params).

    Defaults are the paper's (Sec. IV: W=2, S=5, L=3, N=2, 4 iterations per
    level and 6 at full resolution; Sec. III-E: r=7 / r=5 patches, regions
    under 9 removed, motion difference under 12 px) on a stride-3 lattice."""
    levels: int = 3
    seed_stride: int = 3
    patch_fwd: int = 15
    patch_bwd: int = 11
    sobel: int = 5
    color: int = 1
    descriptor: int = 0
    cs_sched: int = 0
    norm: int = 0
    iters_coarse: int = 4
    iters_fine: int = 6
    refine_rounds: int = 2
    rs_W: int = 2
    rs_mode: int = 0
    tau2: int = 1
    min_region: int = 9
    region_dmax2: int = 144
    max_visits: int = 0
    ablation: int = 0
    rs_grid: int = 0
    philox_key: int = 0x5EED5EED1234ABCD
    iters_level: tuple = ()       # per-level iteration counts (level 0 first); () keeps
                                  # iters_coarse / iters_fine, -1 keeps them at one level

    def cstruct(self) -> _lib.CParams:
        p = _lib.CParams()
        for f in fields(self):
            if f.name == "iters_level":
                lv = tuple(self.iters_level)
                if len(lv) > 12:
                    raise ValueError("iters_level: at most 12 levels")
                for l in range(12):
                    p.iters_level[l] = int(lv[l]) if l < len(lv) else -1
            else:
                setattr(p, f.name, int(getattr(self, f.name)))
        return p

    def replace(self, **kw) -> "Params":
        d = asdict(self)
        d.update(kw)
        return Params(**d)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class Pyramid:
    """Gradient pyramid of one w x h image in one device buffer."""

    def __init__(self, params: Params, w: int, h: int, device="cuda"):
        L = _lib.load()
        self.params, self.w, self.h = params, int(w), int(h)
        self._cp = params.cstruct()
        nbytes = L.pgm_pyramid_bytes(C.byref(self._cp), self.w, self.h)
        if nbytes == 0:
            raise ValueError("invalid parameters or image size")
        self.buf = torch.empty(nbytes, dtype=torch.uint8, device=device)

    def build(self, img: torch.Tensor, stream=None) -> "Pyramid":
        """img: uint8 (h, w) or (h, w, 3) on the device, rows contiguous."""
        if img.dtype != torch.uint8 or not img.is_cuda:
            raise TypeError("img must be a uint8 CUDA tensor")
        c = 1 if img.dim() == 2 else img.shape[2]
        if img.shape[0] != self.h or img.shape[1] != self.w:
            raise ValueError("image size differs from the pyramid's")
        if img.stride(-1) != 1 or (img.dim() == 3 and img.stride(1) != c):
            raise ValueError("pixels must be contiguous within a row")
        check(_lib.load().pgm_build_pyramid(
            C.byref(self._cp), C.c_void_p(img.data_ptr()), self.w, self.h, c,
            img.stride(0), C.c_void_p(self.buf.data_ptr()), self.buf.numel(), _stream(stream)),
            "pgm_build_pyramid")
        return self

    def desc_layout(self, scheme: int, level: int) -> dict:
        off, lw, lh, nch, row = C.c_size_t(), C.c_int(), C.c_int(), C.c_int(), C.c_int()
        pxe, bord = C.c_int(), C.c_int()
        check(_lib.load().pgm_pyramid_desc_layout(C.byref(self._cp), self.w, self.h, scheme,
                                                  level, C.byref(off), C.byref(lw), C.byref(lh),
                                                  C.byref(nch), C.byref(row), C.byref(pxe),
                                                  C.byref(bord)),
              "pgm_pyramid_desc_layout")
        return dict(offset=off.value, w=lw.value, h=lh.value, nch=nch.value, row=row.value,
                    px=pxe.value, border=bord.value)

    def desc_padded(self, scheme: int, level: int) -> torch.Tensor:
        """(lh + 2 B, lw + 2 B, 2C) int16 view of the descriptor with its
        replicated border of B pixels."""
        d = self.desc_layout(scheme, level)
        B, row, px = d["border"], d["row"], d["px"]
        start = d["offset"] - 2 * (B * row + B * px)
        v = self.buf[start:start + 2 * row * (d["h"] + 2 * B)].view(torch.int16)
        v = v.view(d["h"] + 2 * B, row)[:, :(d["w"] + 2 * B) * px]
        return v.reshape(d["h"] + 2 * B, d["w"] + 2 * B, px)[..., :d["nch"]]

    def desc(self, scheme: int, level: int) -> torch.Tensor:
        """(lh, lw, 2C) int16 view: Gx of each channel, then Gy of each."""
        d = self.desc_layout(scheme, level)
        B = d["border"]
        return self.desc_padded(scheme, level)[B:B + d["h"], B:B + d["w"]]

    def cimage(self, scheme: int, level: int) -> torch.Tensor:
        """(C, lh, lw) uint8 view of the colour-converted level image."""
        off, lw, lh, ch = C.c_size_t(), C.c_int(), C.c_int(), C.c_int()
        row, plane = C.c_int(), C.c_size_t()
        check(_lib.load().pgm_pyramid_image_layout(C.byref(self._cp), self.w, self.h, scheme,
                                                   level, C.byref(off), C.byref(lw), C.byref(lh),
                                                   C.byref(ch), C.byref(row), C.byref(plane)),
              "pgm_pyramid_image_layout")
        v = self.buf[off.value:off.value + plane.value * ch.value]
        return v.view(ch.value, lh.value, row.value)[:, :, :lw.value]


class Workspace:
    """Match workspace of one (w1 x h1) -> (w2 x h2) pair."""

    def __init__(self, params: Params, w1, h1, w2, h2, device="cuda"):
        L = _lib.load()
        self.params = params
        self.dims = (int(w1), int(h1), int(w2), int(h2))
        self._cp = params.cstruct()
        nbytes = L.pgm_match_workspace_bytes(C.byref(self._cp), *self.dims)
        if nbytes == 0:
            raise ValueError("invalid parameters or image size")
        self.buf = torch.zeros(nbytes, dtype=torch.uint8, device=device)

    def layout(self, level: int, d: int):
        nx, ny = C.c_int(), C.c_int()
        ou, oc, of = C.c_size_t(), C.c_size_t(), C.c_size_t()
        check(_lib.load().pgm_field_layout(C.byref(self._cp), *self.dims, level, d,
                                           C.byref(nx), C.byref(ny), C.byref(ou), C.byref(oc),
                                           C.byref(of)), "pgm_field_layout")
        return nx.value, ny.value, ou.value, oc.value, of.value

    def field(self, level: int, d: int) -> dict:
        """Views of one level and direction (0 forward, 1 backward): ux, uy
        (int16), cost (int64 bits of the uint64 cost), and the flag bits."""
        nx, ny, ou, oc, of = self.layout(level, d)
        n = nx * ny
        u = self.buf[ou:ou + 4 * n].view(torch.int16).view(ny, nx, 2)
        cost = self.buf[oc:oc + 8 * n].view(torch.int64).view(ny, nx)
        flags = self.buf[of:of + n].view(ny, nx)
        return {"ux": u[..., 0], "uy": u[..., 1], "cost": cost,
                "valid": flags & 1, "outlier": (flags >> 1) & 1, "oinit": (flags >> 2) & 1}

    def evals(self) -> dict:
        """Patch distances evaluated by the last match (device counters)."""
        o = _lib.WS_EVALS_OFFSET
        v = self.buf[o:o + 8 * _lib.WS_EVALS_COUNT].view(torch.int64).tolist()
        return {"pm": v[0:2], "cost": v[2:4], "init": v[4:6], "pm_global": v[6:8]}

    def sync_status(self, stream=None):
        check(_lib.load().pgm_sync_status(C.byref(self._cp), *self.dims,
                                          C.c_void_p(self.buf.data_ptr()), self.buf.numel(),
                                          _stream(stream)), "device status")

    def dump(self, path):
        """Write the fields of every level and direction to an .npz file, for
        debugging: arrays ``l<level>_d<dir>_ux / _uy`` (int16), ``_cost``
        (uint64) and ``_flags`` (uint8: bit 0 initialised, bit 1 outlier, bit 2
        outlier record initialised), the pair's dims and the parameters as
        JSON.  Reads the buffer (a device synchronisation on CUDA)."""
        import json
        import numpy as np
        out = {"dims": np.array(self.dims, dtype=np.int32),
               "params": np.array(json.dumps(asdict(self.params)))}
        for level in range(self.params.levels):
            for d in (0, 1):
                nx, ny, ou, oc, of = self.layout(level, d)
                n = nx * ny
                u = self.buf[ou:ou + 4 * n].view(torch.int16).view(ny, nx, 2).cpu().numpy()
                k = "l%d_d%d_" % (level, d)
                out[k + "ux"], out[k + "uy"] = u[..., 0].copy(), u[..., 1].copy()
                out[k + "cost"] = self.buf[oc:oc + 8 * n].view(torch.int64).view(ny, nx) \
                    .cpu().numpy().view(np.uint64)
                out[k + "flags"] = self.buf[of:of + n].view(ny, nx).cpu().numpy()
        np.savez_compressed(path, **out)


def load_fields(path):
    """Read a ``Workspace.dump`` file: (params dict, dims tuple, {(level, dir):
    {"ux", "uy", "cost", "flags"}})."""
    import json
    import numpy as np
    with np.load(path) as z:
        params = json.loads(str(z["params"]))
        dims = tuple(int(v) for v in z["dims"])
        fields_ = {}
        for key in z.files:
            if key.startswith("l") and "_d" in key:
                lv, d, name = key[1:].split("_", 2)
                fields_.setdefault((int(lv), int(d[1:])), {})[name] = z[key]
    return params, dims, fields_


# the pgm_params fields that fix a pyramid buffer's layout and contents
PYRAMID_FIELDS = ("levels", "sobel", "color", "descriptor", "cs_sched")


def check_pyramids(params: Params, *pyrs) -> None:
    """pgm_match and pgm_interpolate take pyramid buffers without their sizes
    and read them with the layout `params` implies.  Refuse, before the call,
    a pyramid built under other layout parameters (it would be read with the
    wrong layout, possibly past its end) or a buffer smaller than the layout."""
    L = _lib.load()
    cp = params.cstruct()
    for p in pyrs:
        diff = [f for f in PYRAMID_FIELDS if getattr(p.params, f) != getattr(params, f)]
        if diff:
            raise ValueError("pyramid built with other %s than the call's parameters"
                             % ", ".join(diff))
        need = L.pgm_pyramid_bytes(C.byref(cp), p.w, p.h)
        if need == 0 or p.buf.numel() < need:
            raise ValueError("pyramid buffer of %d bytes, the layout needs %d"
                             % (p.buf.numel(), need))


def nominal_evals(params: Params, w1, h1, w2, h2) -> int:
    return int(_lib.load().pgm_nominal_evals(C.byref(params.cstruct()), w1, h1, w2, h2))


def build_pyramid(params: Params, img: torch.Tensor, stream=None) -> Pyramid:
    return Pyramid(params, img.shape[1], img.shape[0], img.device).build(img, stream)


def match(params: Params, pyr1: Pyramid, pyr2: Pyramid, stream_id: int = 0,
          ws: Workspace = None, stream=None) -> Workspace:
    check_pyramids(params, pyr1, pyr2)
    if ws is None:
        ws = Workspace(params, pyr1.w, pyr1.h, pyr2.w, pyr2.h, pyr1.buf.device)
    cp = params.cstruct()
    check(_lib.load().pgm_match(C.byref(cp), C.c_void_p(pyr1.buf.data_ptr()),
                                C.c_void_p(pyr2.buf.data_ptr()), pyr1.w, pyr1.h, pyr2.w, pyr2.h,
                                int(stream_id), C.c_void_p(ws.buf.data_ptr()), ws.buf.numel(),
                                _stream(stream)), "pgm_match")
    return ws


def match_batch(params: Params, pyrs1, pyrs2, stream_ids, wss, stream=None):
    n = len(pyrs1)
    if not (len(pyrs2) == len(stream_ids) == len(wss) == n):
        raise ValueError("match_batch: pyrs1, pyrs2, stream_ids and wss differ in length")
    check_pyramids(params, *pyrs1, *pyrs2)
    cp = params.cstruct()
    P1 = (C.c_void_p * n)(*[p.buf.data_ptr() for p in pyrs1])
    P2 = (C.c_void_p * n)(*[p.buf.data_ptr() for p in pyrs2])
    dims = (C.c_int32 * (4 * n))(*[v for a, b in zip(pyrs1, pyrs2) for v in (a.w, a.h, b.w, b.h)])
    sids = (C.c_uint64 * n)(*[int(s) for s in stream_ids])
    W = (C.c_void_p * n)(*[w.buf.data_ptr() for w in wss])
    WB = (C.c_size_t * n)(*[w.buf.numel() for w in wss])
    check(_lib.load().pgm_match_batch(C.byref(cp), n, P1, P2, dims, sids, W, WB, _stream(stream)),
          "pgm_match_batch")
    return wss


def build_pyramids(params: Params, imgs, pyrs, stream=None):
    """Build many pyramids in shared launches (pgm_build_pyramid_batch)."""
    n = len(imgs)
    cp = params.cstruct()
    for img, p in zip(imgs, pyrs):
        if img.dtype != torch.uint8 or not img.is_cuda or img.shape[0] != p.h or img.shape[1] != p.w:
            raise ValueError("image/pyramid mismatch")
    I = (C.c_void_p * n)(*[x.data_ptr() for x in imgs])
    dims = (C.c_int32 * (3 * n))(*[v for x in imgs
                                     for v in (x.shape[1], x.shape[0], 1 if x.dim() == 2 else x.shape[2])])
    pit = (C.c_size_t * n)(*[x.stride(0) for x in imgs])
    P = (C.c_void_p * n)(*[p.buf.data_ptr() for p in pyrs])
    PB = (C.c_size_t * n)(*[p.buf.numel() for p in pyrs])
    check(_lib.load().pgm_build_pyramid_batch(C.byref(cp), n, I, dims, pit, P, PB, _stream(stream)),
          "pgm_build_pyramid_batch")
    return pyrs


def filter_batch(params: Params, wss, rows, counts, stream=None):
    """pgm_filter on many workspaces in shared launches.  rows[k]: [max, 4]
    int32, counts[k]: [1] int32 (device)."""
    n = len(wss)
    cp = params.cstruct()
    dims = (C.c_int32 * (4 * n))(*[v for w in wss for v in w.dims])
    W = (C.c_void_p * n)(*[w.buf.data_ptr() for w in wss])
    WB = (C.c_size_t * n)(*[w.buf.numel() for w in wss])
    R = (C.c_void_p * n)(*[r.data_ptr() for r in rows])
    RM = (C.c_int64 * n)(*[r.shape[0] for r in rows])
    CN = (C.c_void_p * n)(*[c.data_ptr() for c in counts])
    check(_lib.load().pgm_filter_batch(C.byref(cp), n, dims, W, WB, R, RM, CN, _stream(stream)),
          "pgm_filter_batch")


def filter_into(params: Params, ws: Workspace, matches: torch.Tensor, count: torch.Tensor,
                keep: torch.Tensor = None, stream=None):
    """Enqueue the final filter into preallocated matches [max, 4] int32 and
    count [1] int32 (device)."""
    cp = params.cstruct()
    check(_lib.load().pgm_filter(C.byref(cp), *ws.dims, C.c_void_p(ws.buf.data_ptr()),
                                 ws.buf.numel(), C.c_void_p(matches.data_ptr()),
                                 matches.shape[0], C.c_void_p(count.data_ptr()),
                                 C.c_void_p(keep.data_ptr() if keep is not None else 0),
                                 _stream(stream)), "pgm_filter")


def filter_matches(params: Params, ws: Workspace, max_matches: int = None, stream=None):
    """(matches [n, 4] int32 (x1, y1, x2, y2), keep mask (ny, nx) uint8)."""
    nx, ny, *_ = ws.layout(0, 0)
    cap = nx * ny if max_matches is None else max_matches
    dev = ws.buf.device
    rows = torch.empty((max(cap, 1), 4), dtype=torch.int32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    keep = torch.empty((ny, nx), dtype=torch.uint8, device=dev)
    filter_into(params, ws, rows, cnt, keep, stream)
    n = int(cnt.item())
    return rows[:min(n, cap)], keep


class PairMatcher:
    """Preallocated buffers for repeated matching of `batch` pairs of one size:
    pyramids, workspaces and match rows stay resident in HBM."""

    def __init__(self, params: Params, w: int, h: int, batch: int = 1, device="cuda"):
        self.params, self.w, self.h, self.batch = params, w, h, batch
        self.p1 = [Pyramid(params, w, h, device) for _ in range(batch)]
        self.p2 = [Pyramid(params, w, h, device) for _ in range(batch)]
        self.ws = [Workspace(params, w, h, w, h, device) for _ in range(batch)]
        nx, ny, *_ = self.ws[0].layout(0, 0)
        self.cap = nx * ny
        self.rows = torch.empty((batch, self.cap, 4), dtype=torch.int32, device=device)
        self.count = torch.zeros((batch, 1), dtype=torch.int32, device=device)

    def enqueue(self, imgs1, imgs2, stream_ids=None, stream=None):
        """Whole hot path on the device for the batch: pyramids, matching,
        filter (three C-ABI calls).  imgs*: lists of uint8 CUDA tensors."""
        build_pyramids(self.params, list(imgs1) + list(imgs2), self.p1 + self.p2, stream)
        sids = list(range(self.batch)) if stream_ids is None else stream_ids
        match_batch(self.params, self.p1, self.p2, sids, self.ws, stream)
        filter_batch(self.params, self.ws, [self.rows[k] for k in range(self.batch)],
                     [self.count[k] for k in range(self.batch)], stream)

    def capture(self, imgs1, imgs2, stream_ids=None):
        """Record one whole step on these (fixed) device image tensors as a CUDA
        graph; ``replay()`` then reruns it with whatever the tensors hold.
        Returns the number of library kernels one replay launches."""
        L = _lib.load()
        self.enqueue(imgs1, imgs2, stream_ids)          # first call sets kernel attributes
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        n0 = L.pgm_launch_count()
        with torch.cuda.graph(self.graph):
            self.enqueue(imgs1, imgs2, stream_ids)
        self.graph_launches = int(L.pgm_launch_count() - n0)
        return self.graph_launches

    def replay(self):
        self.graph.replay()

    def results(self):
        counts = self.count[:, 0].tolist()
        return [self.rows[k, :min(c, self.cap)] for k, c in enumerate(counts)]


@dataclass
class InterpParams:
    """Sparse-to-dense interpolation parameters (include/pgm.h,
    pgm_interp_params): k nearest matches, mode 0 auto (LA above
    la_permyriad / 10^4 matches per pixel, the paper's 2.2 %), 1 NW, 2 LA."""
    k: int = 16
    mode: int = 0
    cost_shift: int = 10
    la_permyriad: int = 220
    lam: float = 32.0

    def cstruct(self) -> _lib.CInterp:
        return _lib.CInterp(int(self.k), int(self.mode), int(self.cost_shift),
                            int(self.la_permyriad), float(self.lam))


def interpolate(params: Params, pyr1: Pyramid, matches: torch.Tensor, count: torch.Tensor,
                ip: InterpParams = None, ws: torch.Tensor = None, stream=None):
    """Dense flow (h, w, 2) float32 of image 1 from exported matches
    (n, 4) int32 and their device count (pgm_interpolate).  Returns (flow,
    workspace); the workspace starts with the (h, w, k) uint64 neighbour keys."""
    check_pyramids(params, pyr1)
    ip = ip or InterpParams()
    cip = ip.cstruct()
    L = _lib.load()
    nbytes = L.pgm_interp_workspace_bytes(pyr1.w, pyr1.h, C.byref(cip))
    if nbytes == 0:
        raise ValueError("invalid interpolation parameters or image size")
    if ws is None or ws.numel() < nbytes:
        ws = torch.empty(nbytes, dtype=torch.uint8, device=pyr1.buf.device)
    flow = torch.empty((pyr1.h, pyr1.w, 2), dtype=torch.float32, device=pyr1.buf.device)
    m = matches.contiguous()
    check(L.pgm_interpolate(C.byref(params.cstruct()), C.c_void_p(pyr1.buf.data_ptr()), pyr1.w,
                            pyr1.h, C.c_void_p(m.data_ptr()), C.c_void_p(count.data_ptr()),
                            int(m.shape[0]), C.byref(cip), C.c_void_p(ws.data_ptr()), ws.numel(),
                            C.c_void_p(flow.data_ptr()), _stream(stream)), "pgm_interpolate")
    return flow, ws


def interp_keys(ws: torch.Tensor, w: int, h: int, k: int) -> torch.Tensor:
    """(h, w, k) int64 view of the neighbour keys at the start of an
    interpolation workspace (uint64 bits)."""
    return ws[:8 * w * h * k].view(torch.int64).view(h, w, k)
