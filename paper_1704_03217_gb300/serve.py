"""Serving: continuous batching of image pairs under a device-memory budget.

Requests (pairs of images, any size) arrive over time.  Every scheduler tick
admits the waiting requests, oldest first, while the device-memory budget and
the batch limit allow; the admitted batch is launched on its own CUDA stream
(host->device copies, batched pyramids, batched matching, batched filter,
device->host copy of the matches) while earlier batches are still running,
so their work overlaps on the GPU.  A finished batch releases its memory,
which lets the next waiting requests in.  Latency is measured from arrival to
the moment the matches are on the host.

The admission policy (``Scheduler``) is plain Python with no GPU dependency,
so it is tested on the CPU with a fake clock; ``GpuExecutor`` runs batches
through the library's batched entry points.
"""
import collections
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    arrival: float                  # seconds, on the server clock
    img1: np.ndarray                # uint8 (h, w) or (h, w, 3)
    img2: np.ndarray
    stream_id: int = 0
    admitted: float = None
    done: float = None
    matches: np.ndarray = None
    nbytes: int = 0

    @property
    def latency(self):
        return None if self.done is None else self.done - self.arrival


class Scheduler:
    """FIFO admission under a byte budget.  ``bytes_of(req)`` is the device
    memory a request holds while it is in flight."""

    def __init__(self, budget_bytes, max_batch, bytes_of):
        self.budget, self.max_batch, self.bytes_of = int(budget_bytes), int(max_batch), bytes_of
        self.waiting = collections.deque()
        self.in_use = 0
        self.peak = 0

    def arrive(self, req):
        req.nbytes = int(self.bytes_of(req))
        if req.nbytes > self.budget:
            raise ValueError("request %d needs %d bytes, over the whole budget" % (req.rid, req.nbytes))
        self.waiting.append(req)

    def admit(self, now):
        """Requests to launch now: oldest first, stopping at the first that does
        not fit (no overtaking), at most max_batch."""
        batch = []
        while self.waiting and len(batch) < self.max_batch:
            r = self.waiting[0]
            if r.arrival > now or self.in_use + r.nbytes > self.budget:
                break
            self.waiting.popleft()
            self.in_use += r.nbytes
            r.admitted = now
            batch.append(r)
        self.peak = max(self.peak, self.in_use)
        return batch

    def complete(self, batch, now):
        for r in batch:
            self.in_use -= r.nbytes
            r.done = now


def serve(requests, scheduler, executor, clock=time.perf_counter, idle_sleep=0.0002):
    """Run the continuous-batching loop until every request is done.  Request
    arrival times are relative to the start of the loop."""
    pending = sorted(requests, key=lambda r: r.arrival)
    t0 = clock()
    i, finished = 0, 0
    while finished < len(pending):
        now = clock() - t0
        while i < len(pending) and pending[i].arrival <= now:
            scheduler.arrive(pending[i])
            i += 1
        for batch in executor.poll():
            scheduler.complete(batch, clock() - t0)
            finished += len(batch)
        batch = scheduler.admit(clock() - t0)
        if batch:
            executor.launch(batch)
        elif idle_sleep:
            time.sleep(idle_sleep)
    return pending


def summary(done, wall=None):
    lat = np.array([r.latency for r in done]) * 1e3
    first = min(r.arrival for r in done)
    last = max(r.done for r in done)
    span = wall if wall is not None else (last - first)
    return {"requests": len(done), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "pairs_per_s": len(done) / span}


class GpuExecutor:
    """Runs admitted batches through the library: one CUDA stream per batch in
    flight (a small pool), completion detected with events."""

    def __init__(self, params, streams=3, device="cuda"):
        import torch
        from . import api
        self.torch, self.api = torch, api
        self.params, self.device = params, device
        self.streams = [torch.cuda.Stream(device=device) for _ in range(streams)]
        self.next = 0
        self.inflight = []            # (event, batch, buffers)

    def bytes_of(self, req):
        from . import _lib
        import ctypes as C
        L = _lib.load()
        cp = self.params.cstruct()
        h1, w1 = req.img1.shape[:2]
        h2, w2 = req.img2.shape[:2]
        nx = (w1 - 1 - self.params.seed_stride // 2) // self.params.seed_stride + 1
        ny = (h1 - 1 - self.params.seed_stride // 2) // self.params.seed_stride + 1
        return (L.pgm_pyramid_bytes(C.byref(cp), w1, h1) + L.pgm_pyramid_bytes(C.byref(cp), w2, h2)
                + L.pgm_match_workspace_bytes(C.byref(cp), w1, h1, w2, h2)
                + req.img1.nbytes + req.img2.nbytes + 16 * nx * ny + 4)

    def launch(self, batch):
        torch, api = self.torch, self.api
        st = self.streams[self.next % len(self.streams)]
        self.next += 1
        with torch.cuda.stream(st):
            i1 = [torch.from_numpy(r.img1).to(self.device, non_blocking=True) for r in batch]
            i2 = [torch.from_numpy(r.img2).to(self.device, non_blocking=True) for r in batch]
            p1 = [api.Pyramid(self.params, x.shape[1], x.shape[0], self.device) for x in i1]
            p2 = [api.Pyramid(self.params, x.shape[1], x.shape[0], self.device) for x in i2]
            api.build_pyramids(self.params, i1 + i2, p1 + p2, st)
            ws = [api.Workspace(self.params, a.w, a.h, b.w, b.h, self.device) for a, b in zip(p1, p2)]
            api.match_batch(self.params, p1, p2, [r.stream_id for r in batch], ws, st)
            caps = [w.layout(0, 0)[0] * w.layout(0, 0)[1] for w in ws]
            rows = [torch.empty((max(c, 1), 4), dtype=torch.int32, device=self.device) for c in caps]
            cnt = [torch.zeros(1, dtype=torch.int32, device=self.device) for _ in batch]
            api.filter_batch(self.params, ws, rows, cnt, st)
            rows_h = [r.to("cpu", non_blocking=True) for r in rows]
            cnt_h = [c.to("cpu", non_blocking=True) for c in cnt]
            ev = torch.cuda.Event()
            ev.record(st)
        self.inflight.append((ev, batch, (i1, i2, p1, p2, ws, rows, cnt, rows_h, cnt_h)))

    def poll(self):
        done, keep = [], []
        for ev, batch, bufs in self.inflight:
            if ev.query():
                rows_h, cnt_h = bufs[7], bufs[8]
                for r, rh, ch in zip(batch, rows_h, cnt_h):
                    n = int(ch.item())
                    r.matches = rh[:min(n, rh.shape[0])].numpy()
                done.append(batch)
            else:
                keep.append((ev, batch, bufs))
        self.inflight = keep
        return done


def poisson_requests(seed, rate_hz, n, sizes=((640, 480), (1280, 720), (1920, 1080), (1024, 436)),
                     pool=8):
    """n requests with exponential inter-arrival times (mean 1/rate_hz); each
    carries a Sintel-like pair of a size drawn uniformly from ``sizes``.  A
    pool of `pool` distinct pairs per size is generated and reused."""
    from . import synth
    rng = np.random.default_rng(seed)
    cache = {}
    t, out = 0.0, []
    for k in range(n):
        t += rng.exponential(1.0 / rate_hz)
        w, h = sizes[int(rng.integers(len(sizes)))]
        key = (w, h, int(rng.integers(pool)))
        if key not in cache:
            sd = (seed * 7919 + w * 1009 + h * 101 + key[2]) & 0xFFFFFF
            f1, f2, _ = synth.sintel_like_pair(sd, w, h, t_max=min(150.0, w / 8))
            cache[key] = (f1, f2)
        f1, f2 = cache[key]
        out.append(Request(k, t, f1, f2, stream_id=k))
    return out
