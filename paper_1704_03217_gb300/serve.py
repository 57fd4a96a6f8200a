"""Serving: continuous batching of image pairs under a device-memory budget.

Requests (pairs of images, any size) arrive over time.  Every scheduler tick
admits the waiting requests, oldest first, while the device-memory budget and
the batch limit allow; the admitted batch is launched on its own CUDA stream
(host->device copies, batched pyramids, batched matching, batched filter,
device->host copy of the matches) while earlier batches are still running,
so their work overlaps on the GPU.  A finished batch releases its memory,
which lets the next waiting requests in.  Latency is measured from arrival to
the moment the matches are on the host.

Failures are contained to the request that caused them:
  - a request larger than the whole budget is rejected on arrival (its
    ``error`` says why) and the loop goes on;
  - a batch whose launch fails (an allocation failure, an argument error)
    is put back at the head of the queue and its requests are retried one at
    a time, so only the failing request is evicted;
  - a request whose device-side status reports an error (a bounded wait that
    ran out, a failed bounds check) is evicted when its batch completes,
    without its matches; the others of the batch deliver theirs.
``Faults`` injects failures of each kind on the host, for tests: from code,
or from the environment as ``PGM_FAULT=alloc@5,admit@7,timeout@9`` (a failed
slot allocation for request 5, request 7 refused at admission, request 9
reported as if a bounded device wait had run out).  No injected fault touches
the GPU: each one is decided on the host, between launches.

The admission policy (``Scheduler``) is plain Python with no GPU dependency,
so it is tested on the CPU with a fake clock; ``GpuExecutor`` runs batches
through the library's batched entry points, on buffers kept resident in a
pool of slots (pyramids, workspace, match rows) reused across batches.
"""
import collections
import os
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
    error: str = None               # why the request was rejected or evicted

    @property
    def latency(self):
        return None if self.done is None else self.done - self.arrival


@dataclass
class Faults:
    """Host-side fault injection, by request id:
      alloc_fail:   the launch of the request's batch fails as if a slot
                    allocation failed (the batch is retried singly, the
                    request evicted);
      device_error: the request completes with a device-side error reported;
      admit_reject: the request is refused when it arrives;
      timeout:      the request completes as if a bounded wait of the search
                    kernel had run out (PGM_ERR_TIMEOUT in its status word)."""
    alloc_fail: set = field(default_factory=set)
    device_error: set = field(default_factory=set)
    admit_reject: set = field(default_factory=set)
    timeout: set = field(default_factory=set)

    KINDS = {"alloc": "alloc_fail", "admit": "admit_reject", "timeout": "timeout",
             "device": "device_error"}

    @classmethod
    def parse(cls, spec):
        """Faults from a spec such as ``alloc@5,admit@7,timeout@9+12``: comma-
        separated ``kind@ids`` items, ids joined by ``+``; kinds alloc, admit,
        timeout and device.  An empty spec injects nothing; anything else
        malformed raises ValueError."""
        f = cls()
        for item in (spec or "").replace(" ", "").split(","):
            if not item:
                continue
            kind, sep, ids = item.partition("@")
            if not sep or kind not in cls.KINDS or not ids:
                raise ValueError("PGM_FAULT item %r: expected kind@id with kind in %s"
                                 % (item, "/".join(sorted(cls.KINDS))))
            try:
                rids = {int(x) for x in ids.split("+")}
            except ValueError:
                raise ValueError("PGM_FAULT item %r: request ids must be integers" % item) from None
            getattr(f, cls.KINDS[kind]).update(rids)
        return f

    @classmethod
    def from_env(cls, environ=None):
        """Faults named by the PGM_FAULT environment variable (none if unset)."""
        env = os.environ if environ is None else environ
        return cls.parse(env.get("PGM_FAULT", ""))

    def device_failure(self, rid):
        """The device-side failure injected for request `rid`, or None."""
        if rid in self.timeout:
            return "PGM_ERR_TIMEOUT (injected: a bounded device wait ran out)"
        if rid in self.device_error:
            return "injected device error"
        return None


class LaunchError(RuntimeError):
    """A batch could not be launched; ``rids`` names the requests involved."""

    def __init__(self, msg, rids):
        super().__init__(msg)
        self.rids = list(rids)


class Scheduler:
    """FIFO admission under a byte budget.  ``bytes_of(req)`` is the device
    memory a request holds while it is in flight.  ``faults.admit_reject``
    (default: from PGM_FAULT) names requests refused on arrival."""

    def __init__(self, budget_bytes, max_batch, bytes_of, faults=None):
        self.budget, self.max_batch, self.bytes_of = int(budget_bytes), int(max_batch), bytes_of
        self.faults = faults if faults is not None else Faults.from_env()
        self.waiting = collections.deque()
        self.in_use = 0
        self.peak = 0
        self.rejected = []
        self.single = 0              # requests to admit one at a time (retries)

    def arrive(self, req, now=0.0):
        """Queue a request; one larger than the whole budget, or named by
        faults.admit_reject, is rejected (returns False, req.error set)."""
        req.nbytes = int(self.bytes_of(req))
        err = None
        if req.rid in self.faults.admit_reject:
            err = "rejected: injected admission failure"
        elif req.nbytes > self.budget:
            err = "rejected: needs %d bytes, over the %d-byte budget" % (req.nbytes, self.budget)
        if err is not None:
            req.error = err
            req.done = now
            self.rejected.append(req)
            return False
        self.waiting.append(req)
        return True

    def admit(self, now):
        """Requests to launch now: oldest first, stopping at the first that does
        not fit (no overtaking), at most max_batch (1 while retrying)."""
        batch = []
        limit = 1 if self.single > 0 else self.max_batch
        while self.waiting and len(batch) < limit:
            r = self.waiting[0]
            if r.arrival > now or self.in_use + r.nbytes > self.budget:
                break
            self.waiting.popleft()
            self.in_use += r.nbytes
            r.admitted = now
            batch.append(r)
        if batch and self.single > 0:
            self.single -= 1
        self.peak = max(self.peak, self.in_use)
        return batch

    def requeue_front(self, batch):
        """A batch whose launch failed: release it and put its requests back at
        the head of the queue, in order, to be retried one at a time."""
        for r in reversed(batch):
            self.in_use -= r.nbytes
            r.admitted = None
            self.waiting.appendleft(r)
        self.single += len(batch)

    def complete(self, batch, now):
        for r in batch:
            self.in_use -= r.nbytes
            r.done = now


def serve(requests, scheduler, executor, clock=time.perf_counter, idle_sleep=0.0002):
    """Run the continuous-batching loop until every request is done, matched or
    failed (req.error).  Request arrival times are relative to the start of
    the loop."""
    pending = sorted(requests, key=lambda r: r.arrival)
    t0 = clock()
    i, finished = 0, 0
    while finished < len(pending):
        now = clock() - t0
        while i < len(pending) and pending[i].arrival <= now:
            if not scheduler.arrive(pending[i], now):
                finished += 1                      # rejected on arrival
            i += 1
        for batch in executor.poll():
            scheduler.complete(batch, clock() - t0)
            finished += len(batch)
        batch = scheduler.admit(clock() - t0)
        if batch:
            try:
                executor.launch(batch)
            except (LaunchError, MemoryError, RuntimeError) as e:
                if len(batch) > 1:
                    scheduler.requeue_front(batch)   # retry singly: find the culprit
                else:
                    batch[0].error = "evicted: %s" % e
                    scheduler.complete(batch, clock() - t0)
                    finished += 1
        elif idle_sleep:
            time.sleep(idle_sleep)
    return pending


def summary(done, wall=None):
    """Latency and throughput of the matched requests; failed ones counted
    (latencies are NaN when no request was matched)."""
    if not done:
        nan = float("nan")
        return {"requests": 0, "failed": 0, "p50_ms": nan, "p99_ms": nan, "mean_ms": nan,
                "pairs_per_s": 0.0}
    ok = [r for r in done if r.error is None]
    lat = np.array([r.latency for r in ok], dtype=np.float64) * 1e3
    first = min(r.arrival for r in done)
    last = max(r.done for r in done)
    span = wall if wall is not None else (last - first)
    pct = (lambda q: float(np.percentile(lat, q))) if ok else (lambda q: float("nan"))
    return {"requests": len(done), "failed": len(done) - len(ok),
            "p50_ms": pct(50), "p99_ms": pct(99),
            "mean_ms": float(lat.mean()) if ok else float("nan"),
            "pairs_per_s": len(ok) / span if span > 0 else float("nan")}


class GpuExecutor:
    """Runs admitted batches through the library: one CUDA stream per batch in
    flight (a small pool), completion detected with events.  The device
    buffers of a request (two pyramids, a workspace, its match rows and count,
    and pinned host copies of these) form a slot; slots are kept in a pool
    keyed by the pair's sizes and reused, up to ``pool_bytes`` of idle slots."""

    def __init__(self, params, streams=3, device="cuda", faults=None, pool_bytes=8 << 30):
        import torch
        from . import api
        self.torch, self.api = torch, api
        self.params, self.device = params, device
        self.faults = faults if faults is not None else Faults.from_env()
        self.streams = [torch.cuda.Stream(device=device) for _ in range(streams)]
        self.next = 0
        self.inflight = []            # (event, batch, slots)
        self.pool = collections.defaultdict(list)
        self.pool_bytes, self.idle_bytes = int(pool_bytes), 0
        self.slots_made = 0

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

    def _key(self, r):
        return r.img1.shape + r.img2.shape

    def _take(self, r):
        torch, api = self.torch, self.api
        key = self._key(r)
        if self.pool[key]:
            slot = self.pool[key].pop()
            self.idle_bytes -= slot["bytes"]
            return slot
        h1, w1 = r.img1.shape[:2]
        h2, w2 = r.img2.shape[:2]
        p1 = api.Pyramid(self.params, w1, h1, self.device)
        p2 = api.Pyramid(self.params, w2, h2, self.device)
        ws = api.Workspace(self.params, w1, h1, w2, h2, self.device)
        nx, ny = ws.layout(0, 0)[:2]
        cap = max(nx * ny, 1)
        self.slots_made += 1
        return {"key": key, "p1": p1, "p2": p2, "ws": ws,
                "i1": torch.empty(r.img1.shape, dtype=torch.uint8, device=self.device),
                "i2": torch.empty(r.img2.shape, dtype=torch.uint8, device=self.device),
                "rows": torch.empty((cap, 4), dtype=torch.int32, device=self.device),
                "cnt": torch.zeros(1, dtype=torch.int32, device=self.device),
                "rows_h": torch.empty((cap, 4), dtype=torch.int32).pin_memory(),
                "cnt_h": torch.empty(1, dtype=torch.int32).pin_memory(),
                "bytes": self.bytes_of(r)}

    def _give(self, slot):
        if self.idle_bytes + slot["bytes"] <= self.pool_bytes:
            self.pool[slot["key"]].append(slot)
            self.idle_bytes += slot["bytes"]

    def launch(self, batch):
        torch, api = self.torch, self.api
        bad = [r.rid for r in batch if r.rid in self.faults.alloc_fail]
        if bad:
            raise LaunchError("injected allocation failure (request %s)" % bad, bad)
        slots = [self._take(r) for r in batch]
        st = self.streams[self.next % len(self.streams)]
        self.next += 1
        with torch.cuda.stream(st):
            for r, sl in zip(batch, slots):
                sl["i1"].copy_(torch.from_numpy(r.img1), non_blocking=True)
                sl["i2"].copy_(torch.from_numpy(r.img2), non_blocking=True)
            p1 = [sl["p1"] for sl in slots]
            p2 = [sl["p2"] for sl in slots]
            api.build_pyramids(self.params, [sl["i1"] for sl in slots] + [sl["i2"] for sl in slots],
                               p1 + p2, st)
            ws = [sl["ws"] for sl in slots]
            api.match_batch(self.params, p1, p2, [r.stream_id for r in batch], ws, st)
            api.filter_batch(self.params, ws, [sl["rows"] for sl in slots],
                             [sl["cnt"] for sl in slots], st)
            for sl in slots:
                sl["rows_h"].copy_(sl["rows"], non_blocking=True)
                sl["cnt_h"].copy_(sl["cnt"], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(st)
        self.inflight.append((ev, batch, slots))

    def poll(self):
        done, keep = [], []
        for ev, batch, slots in self.inflight:
            if ev.query():
                for r, sl in zip(batch, slots):
                    try:
                        sl["ws"].sync_status()          # device-side status word of the pair
                        failed = self.faults.device_failure(r.rid)
                    except RuntimeError as e:
                        failed = str(e)
                    if failed:
                        r.error = "evicted: %s" % failed
                        r.matches = None
                    else:
                        n = int(sl["cnt_h"][0])
                        r.matches = sl["rows_h"][:min(n, sl["rows_h"].shape[0])].numpy().copy()
                    self._give(sl)
                done.append(batch)
            else:
                keep.append((ev, batch, slots))
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
