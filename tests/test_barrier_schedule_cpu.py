"""The tile pipeline of the search kernels on a model of parity-waited
mbarriers (CPU only).  Producers stage tiles n = p (mod NPROD) into buffer
n mod nbuf; consumer agents (groups of warps) score tiles n = g (mod NG).  A
wait on parity P returns once the barrier's current phase has parity != P,
as `mbarrier.try_wait.parity` does.  Random interleavings, with the tensor
copies completing at random later times, check that a consumer only reads a
buffer that holds its own tile, fully copied, and that a producer only
refills a buffer nobody still reads.

Waiting on one barrier per buffer (phase n / nbuf) is safe when every
consumer takes every tile; once agents take every NG-th tile and the ring
does not divide evenly, a wait can skip a phase and return early.  One full
barrier per (buffer, agent) and one empty barrier per (buffer, producer),
each waited for its next phase, never does."""
import random

import pytest


class Bar:
    def __init__(self, count):
        self.count, self.pending, self.phase = count, count, 0

    def arrive(self):
        self.pending -= 1
        if self.pending == 0:
            self.phase += 1
            self.pending = self.count

    def passed(self, parity):
        return self.phase % 2 != parity


def run(tiles, nbuf, nprod, ng, warps_per_agent, per_agent, seed):
    """One random interleaving; returns a violation message or None."""
    rng = random.Random(seed)
    if per_agent:
        full = {(b, g): Bar(1) for b in range(nbuf) for g in range(ng)}
        empty = {(b, p): Bar(warps_per_agent) for b in range(nbuf) for p in range(nprod)}
    else:
        full = {b: Bar(1) for b in range(nbuf)}
        empty = {b: Bar(warps_per_agent) for b in range(nbuf)}
    content = [None] * nbuf            # (tile, copied) of each buffer
    readers = [0] * nbuf
    inflight = []                      # copies issued, not landed: (buffer, tile)
    prod = [dict(n=p, waits={}) for p in range(nprod)]
    cons = [dict(g=w // warps_per_agent, n=w // warps_per_agent, reading=False, seen={})
            for w in range(ng * warps_per_agent)]
    done_reads = 0
    need = sum(warps_per_agent for _ in range(tiles))
    for _ in range(200000):
        moves = []
        for i, p in enumerate(prod):
            if p["n"] < tiles:
                moves.append(("p", i))
        for i, c in enumerate(cons):
            if c["n"] < tiles:
                moves.append(("c", i))
        if inflight:
            moves.append(("t", 0))
        if not moves:
            break
        kind, i = rng.choice(moves)
        if kind == "t":                                    # a copy lands
            b, n = inflight.pop(rng.randrange(len(inflight)))
            content[b] = (n, True)
            (full[(b, n % ng)] if per_agent else full[b]).arrive()
        elif kind == "p":
            p = prod[i]
            n = p["n"]
            b = n % nbuf
            if n >= nbuf:
                if per_agent:
                    k = p["waits"].get(b, 0)
                    if not empty[(b, i)].passed(k & 1):
                        continue
                    p["waits"][b] = k + 1
                elif not empty[b].passed(((n // nbuf) - 1) & 1):
                    continue
            if readers[b]:
                return "producer %d refilled buffer %d under a reader (tile %d)" % (i, b, n)
            content[b] = (n, False)
            inflight.append((b, n))
            p["n"] += nprod
        else:
            c = cons[i]
            n = c["n"]
            b = n % nbuf
            if not c["reading"]:
                if per_agent:
                    k = c["seen"].get(b, 0)
                    if not full[(b, c["g"])].passed(k & 1):
                        continue
                    c["seen"][b] = k + 1
                elif not full[b].passed((n // nbuf) & 1):
                    continue
                if content[b] != (n, True):
                    return "consumer %d read tile %s from buffer %d, wanted %d" % (i, content[b], b, n)
                c["reading"] = True
                readers[b] += 1
            else:                                          # done with the tile
                c["reading"] = False
                readers[b] -= 1
                (empty[(b, (n + nbuf) % nprod)] if per_agent else empty[b]).arrive()
                done_reads += 1
                c["n"] += ng
    if done_reads != need:
        return "stalled after %d of %d tile reads" % (done_reads, need)
    return None


@pytest.mark.parametrize("nbuf,nprod,ng,wpa", [(16, 4, 12, 1), (3, 2, 2, 4), (5, 2, 3, 2),
                                               (8, 4, 20, 1)])
def test_per_agent_barriers_are_safe(nbuf, nprod, ng, wpa):
    """The one-seed-per-lane bit-plane kernel's ring (16 buffers, 4
    producers, 12 consumers) and other uneven rings."""
    for seed in range(300):
        assert run(60, nbuf, nprod, ng, wpa, True, seed) is None, seed


def test_one_barrier_per_buffer_is_safe_when_every_warp_takes_every_tile():
    """The warp-per-seed kernels: every consumer warp scores every tile."""
    for nbuf, nprod, warps in ((3, 2, 14), (8, 4, 20), (3, 2, 18)):
        for seed in range(200):
            assert run(40, nbuf, nprod, 1, warps, False, seed) is None, (nbuf, seed)


def test_one_barrier_per_buffer_fails_for_agents_that_skip_phases():
    """Two tile groups on a ring of three buffers: some interleaving makes a
    parity wait return a phase early."""
    bad = [run(60, 3, 2, 2, 4, False, seed) for seed in range(300)]
    assert any(m is not None for m in bad)
