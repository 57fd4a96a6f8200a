"""The serving scheduler on the CPU: a fake clock and a fake executor stand in
for the GPU (a batch takes a fixed time), so the admission policy can be
checked exactly: FIFO without overtaking, the memory budget never exceeded,
and continuous batching (requests that arrive while a batch runs start before
it finishes)."""
import numpy as np
import pytest

from paper_1704_03217_gb300.serve import Request, Scheduler, serve, summary


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 0.001            # every look at the clock advances it by 1 ms
        return self.t


class FakeExecutor:
    """A batch of n requests finishes `base + per * n` seconds after launch."""

    def __init__(self, clock, base=0.02, per=0.005):
        self.clock, self.base, self.per = clock, base, per
        self.inflight, self.launched, self.max_inflight = [], [], 0

    def launch(self, batch):
        self.inflight.append((self.clock.t + self.base + self.per * len(batch), batch))
        self.launched.append([r.rid for r in batch])
        self.max_inflight = max(self.max_inflight, len(self.inflight))

    def poll(self):
        done = [b for t, b in self.inflight if t <= self.clock.t]
        self.inflight = [(t, b) for t, b in self.inflight if t > self.clock.t]
        for b in done:
            for r in b:
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


def test_request_over_budget_is_rejected():
    sch = Scheduler(budget_bytes=5, max_batch=2, bytes_of=lambda r: 6)
    with pytest.raises(ValueError):
        sch.arrive(_reqs(1, 0.0)[0])
