"""The serving scheduler on the CPU: a fake clock and a fake executor stand in
for the GPU (a batch takes a fixed time), so the admission policy can be
checked exactly: FIFO without overtaking, the memory budget never exceeded,
and continuous batching (requests that arrive while a batch runs start before
it finishes)."""
import numpy as np
import pytest

from paper_1704_03217_gb300.serve import Faults, LaunchError, Request, Scheduler, serve, summary


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 0.001            # every look at the clock advances it by 1 ms
        return self.t


class FakeExecutor:
    """A batch of n requests finishes `base + per * n` seconds after launch.
    Faults as in the GPU executor: a launch containing a request of
    faults.alloc_fail raises; a request of faults.device_error or
    faults.timeout completes without matches."""

    def __init__(self, clock, base=0.02, per=0.005, faults=None):
        self.clock, self.base, self.per = clock, base, per
        self.faults = faults or Faults()
        self.inflight, self.launched, self.max_inflight = [], [], 0

    def launch(self, batch):
        bad = [r.rid for r in batch if r.rid in self.faults.alloc_fail]
        if bad:
            raise LaunchError("injected allocation failure", bad)
        self.inflight.append((self.clock.t + self.base + self.per * len(batch), batch))
        self.launched.append([r.rid for r in batch])
        self.max_inflight = max(self.max_inflight, len(self.inflight))

    def poll(self):
        done = [b for t, b in self.inflight if t <= self.clock.t]
        self.inflight = [(t, b) for t, b in self.inflight if t > self.clock.t]
        for b in done:
            for r in b:
                failed = self.faults.device_failure(r.rid)
                if failed:
                    r.error, r.matches = "evicted: %s" % failed, None
                else:
                    r.matches = np.array([[r.rid]])
        return done


def _reqs(n, gap, size=1):
    return [Request(k, k * gap, np.zeros((size, size), np.uint8), np.zeros((size, size), np.uint8),
                    stream_id=k) for k in range(n)]


def test_fifo_budget_and_continuous_batching():
    clock = FakeClock()
    ex = FakeExecutor(clock)
    sch = Scheduler(budget_bytes=10, max_batch=4, bytes_of=lambda r: 3)   # at most 3 in flight
    reqs = serve(_reqs(40, 0.004), sch, ex, clock=clock, idle_sleep=0)
    order = [rid for b in ex.launched for rid in b]
    assert order == list(range(40))                      # oldest first, nobody overtakes
    assert sch.peak <= 10 and sch.in_use == 0
    assert ex.max_inflight >= 2                          # batches overlap
    assert all(len(b) <= 4 for b in ex.launched)
    assert all(r.done >= r.arrival and r.matches[0, 0] == r.rid for r in reqs)
    s = summary(reqs)
    assert s["requests"] == 40 and s["p99_ms"] >= s["p50_ms"] > 0


def test_large_request_waits_for_memory():
    clock = FakeClock()
    ex = FakeExecutor(clock)
    sizes = {0: 6, 1: 6, 2: 2}
    sch = Scheduler(budget_bytes=10, max_batch=8, bytes_of=lambda r: sizes[r.rid])
    reqs = serve(_reqs(3, 0.0), sch, ex, clock=clock, idle_sleep=0)
    # request 1 does not fit beside 0; request 2 would, but must not overtake 1
    assert ex.launched[0] == [0] and ex.launched[1] == [1, 2]
    assert reqs[1].admitted >= reqs[0].done


def test_request_over_budget_is_rejected_and_the_loop_goes_on():
    clock = FakeClock()
    ex = FakeExecutor(clock)
    sizes = {k: 3 for k in range(8)}
    sizes[2] = 6                                          # over the whole budget
    sch = Scheduler(budget_bytes=5, max_batch=2, bytes_of=lambda r: sizes[r.rid])
    reqs = serve(_reqs(8, 0.003), sch, ex, clock=clock, idle_sleep=0)
    assert reqs[2].error.startswith("rejected") and reqs[2].matches is None
    assert [r.rid for r in sch.rejected] == [2]
    assert all(r.error is None and r.matches[0, 0] == r.rid for r in reqs if r.rid != 2)
    assert sch.in_use == 0 and sch.peak <= 5
    assert summary(reqs)["failed"] == 1


def _run(faults, n=30, max_batch=4):
    clock = FakeClock()
    ex = FakeExecutor(clock, faults=faults)
    sch = Scheduler(budget_bytes=12, max_batch=max_batch, bytes_of=lambda r: 3, faults=faults)
    return serve(_reqs(n, 0.002), sch, ex, clock=clock, idle_sleep=0), sch, ex


def test_failed_launch_evicts_only_the_culprit():
    """An allocation failure fails the whole batch's launch; its requests are
    retried one at a time, so only the failing request is evicted and
    reported, and every other request gets exactly the matches it gets in a
    run without faults."""
    clean, _, _ = _run(Faults())
    reqs, sch, ex = _run(Faults(alloc_fail={5, 17}))
    assert [r.rid for r in reqs if r.error] == [5, 17]
    assert all("allocation" in reqs[k].error and reqs[k].matches is None for k in (5, 17))
    for a, b in zip(clean, reqs):
        if b.rid not in (5, 17):
            assert b.error is None and (a.matches == b.matches).all()
    assert sch.in_use == 0 and sch.peak <= 12
    order = [rid for b in ex.launched for rid in b]
    assert order == [k for k in range(30) if k not in (5, 17)]     # still first come, first served


def test_device_error_evicts_only_that_request():
    clean, _, _ = _run(Faults())
    reqs, sch, _ = _run(Faults(device_error={3, 4, 29}))
    assert [r.rid for r in reqs if r.error] == [3, 4, 29]
    for a, b in zip(clean, reqs):
        if b.rid not in (3, 4, 29):
            assert b.error is None and (a.matches == b.matches).all()
    s = summary(reqs)
    assert s["failed"] == 3 and s["requests"] == 30 and sch.in_use == 0


def test_fault_spec():
    f = Faults.parse("alloc@5,admit@7, timeout@9+12,device@3")
    assert (f.alloc_fail, f.admit_reject, f.timeout, f.device_error) == ({5}, {7}, {9, 12}, {3})
    assert Faults.parse("") == Faults() == Faults.from_env({})
    assert Faults.from_env({"PGM_FAULT": "admit@1+2"}).admit_reject == {1, 2}
    assert "PGM_ERR_TIMEOUT" in f.device_failure(9) and f.device_failure(4) is None
    for bad in ("alloc", "alloc@", "oom@3", "alloc@x", "@4"):
        with pytest.raises(ValueError):
            Faults.parse(bad)


def test_admission_fault_rejects_only_that_request():
    clean, _, _ = _run(Faults())
    reqs, sch, ex = _run(Faults(admit_reject={7, 8}))
    assert [r.rid for r in sch.rejected] == [7, 8]
    assert all(reqs[k].error == "rejected: injected admission failure" for k in (7, 8))
    assert all(rid not in (7, 8) for b in ex.launched for rid in b)
    for a, b in zip(clean, reqs):
        if b.rid not in (7, 8):
            assert b.error is None and (a.matches == b.matches).all()
    assert sch.in_use == 0 and summary(reqs)["failed"] == 2


def test_pgm_fault_environment_drives_every_kind(monkeypatch):
    """PGM_FAULT alone (no Faults passed) injects all three host-side kinds
    into one run: the named requests fail with their own reasons, the others
    get exactly the matches of a run without faults."""
    clean, _, _ = _run(Faults())
    monkeypatch.setenv("PGM_FAULT", "alloc@5,admit@11,timeout@20")
    clock = FakeClock()
    ex = FakeExecutor(clock, faults=Faults.from_env())
    sch = Scheduler(budget_bytes=12, max_batch=4, bytes_of=lambda r: 3)     # reads PGM_FAULT
    reqs = serve(_reqs(30, 0.002), sch, ex, clock=clock, idle_sleep=0)
    err = {r.rid: r.error for r in reqs if r.error}
    assert sorted(err) == [5, 11, 20]
    assert "allocation" in err[5] and err[11].startswith("rejected") and "PGM_ERR_TIMEOUT" in err[20]
    for a, b in zip(clean, reqs):
        if b.rid not in err:
            assert b.error is None and (a.matches == b.matches).all()
    assert sch.in_use == 0 and sch.peak <= 12


def test_summary_when_every_request_failed():
    reqs = _reqs(3, 0.01)
    for r in reqs:
        r.error, r.done = "evicted: x", r.arrival + 0.5
    s = summary(reqs)
    assert s["failed"] == 3 and s["pairs_per_s"] == 0.0
    assert np.isnan(s["p50_ms"]) and np.isnan(s["p99_ms"]) and np.isnan(s["mean_ms"])


def test_no_requests():
    clock = FakeClock()
    ex = FakeExecutor(clock)
    sch = Scheduler(budget_bytes=10, max_batch=4, bytes_of=lambda r: 3, faults=Faults())
    assert serve([], sch, ex, clock=clock, idle_sleep=0) == []
    s = summary([])
    assert s["requests"] == 0 and s["pairs_per_s"] == 0.0 and np.isnan(s["p50_ms"])
