"""The tensor-core initialisation's operand layout on a CPU model (no GPU).

The kernel never builds patch matrices: each MMA step reads two pixels of
every row through strided views of staged images (target centres as a
Toeplitz view of a bordered copy, seeds through sigma^2 phase images of the
reference), pairs pixels so that both second-pixel offsets are positive, and
gives an unpaired pixel a zero block.  This model restates the staging, the
pairing and the descriptor address arithmetic, then checks that
- every patch pixel is used exactly once, and every offset is positive and
  encodable (14 bits of 16-byte units);
- every read of a step (128 seed rows, 160 centre rows, both halves) stays
  inside its staged region;
- with worst-case magnitudes (|v| = 12240) the three accumulators' partial
  sums stay below 2^24 for patches up to 15 x 15, so fp32 holds them;
- the three accumulators give the exact cross terms of clamped patches,
  compared with a direct brute-force correlation.
"""
import numpy as np
import pytest

BORD, TC_M, TC_N, TC_NT = 8, 128, 160, 2


def lattice_n(W, s):
    c = s // 2
    return (W - 1 - c) // s + 1 if W - 1 - c >= 0 else 0


def pairs(P, s):
    """Raster order; the partner is the first later unpaired pixel that is
    also later in phase order (phase, r div s, p div s); else a zero block."""
    used = [False] * (P * P)
    key = lambda i: (((i // P) % s) * s + (i % P) % s, (i // P) // s, (i % P) // s)
    out = []
    for i in range(P * P):
        if used[i]:
            continue
        used[i] = True
        j = next((j for j in range(i + 1, P * P) if not used[j] and key(j) > key(i)), None)
        if j is None:
            out.append((i % P, i // P, None, None))
        else:
            used[j] = True
            out.append((i % P, i // P, j % P, j // P))
    return out


def geom(P, s, nx, ny, tw, th):
    e = (P - 1) // s
    Wu = nx + e
    g = dict(e=e, Wu=Wu, mtiles=-(-ny * Wu // TC_M), LA=Wu * (e + 1) + TC_M + e, Wt=tw + P - 1,
             ph=s * s)
    g["ntiles"] = -(-th * g["Wt"] // TC_N)
    g["bands"] = -(-g["ntiles"] // TC_NT)
    g["LB"] = TC_NT * TC_N + (P - 1) * (g["Wt"] + 1)
    return g


def split(v):
    lo = ((v + 64) & 127) - 64
    return (v - lo) >> 7, lo


def steps(P, s, g):
    """Offsets (16-byte units) of both pixels of every step: A relative to
    the tile's first seed in part 0, B relative to the tile's first centre."""
    out = []
    for p1, r1, p2, r2 in pairs(P, s):
        a1 = ((r1 % s) * s + p1 % s) * g["LA"] + (r1 // s) * g["Wu"] + p1 // s
        z = p2 is None
        a2 = a1 + 1 if z else ((r2 % s) * s + p2 % s) * g["LA"] + (r2 // s) * g["Wu"] + p2 // s
        b1 = r1 * g["Wt"] + p1
        b2 = None if z else r2 * g["Wt"] + p2
        out.append((a1, a2, b1, b2))
    return out


@pytest.mark.parametrize("P,s", [(15, 3), (11, 3), (15, 2), (13, 3), (9, 4), (7, 1), (6, 2),
                                 (4, 3), (3, 3), (1, 3), (15, 1)])
def test_pairing_covers_every_pixel_once(P, s):
    st = pairs(P, s)
    seen = [(p, r) for p, r, _, _ in st] + [(p, r) for _, _, p, r in st if p is not None]
    assert sorted(seen) == sorted((p, r) for r in range(P) for p in range(P))
    assert len(st) >= (P * P + 1) // 2 and len(st) <= 128
    if (P, s) == (15, 3):
        assert len(st) == 113 and sum(q is None for _, _, q, _ in st) == 1
    if (P, s) == (11, 3):
        assert len(st) == 61


@pytest.mark.parametrize("P,s,nx,ny,tw,th", [(15, 3, 21, 9, 64, 28), (11, 3, 21, 9, 64, 28),
                                             (15, 3, 40, 23, 120, 68), (15, 1, 30, 20, 30, 20),
                                             (9, 4, 19, 12, 75, 50), (4, 3, 7, 5, 18, 16)])
def test_reads_stay_in_their_regions(P, s, nx, ny, tw, th):
    g = geom(P, s, nx, ny, tw, th)
    LA, LB, ph = g["LA"], g["LB"], g["ph"]
    A0, B0 = 0, 2 * ph * LA
    Z0 = B0 + 2 * LB
    for a1, a2, b1, b2 in steps(P, s, g):
        alb = a2 - a1
        assert 0 < alb < 1 << 14
        for mt in range(g["mtiles"]):
            moff = mt * TC_M - (mt * TC_M // g["Wu"]) * g["Wu"]
            for pa in range(2):
                a = A0 + pa * ph * LA + moff + a1
                assert A0 + pa * ph * LA <= a and a + alb + TC_M <= A0 + (pa + 1) * ph * LA
        for k in range(TC_NT):
            for pb in range(2):
                b = B0 + pb * LB + k * TC_N + b1
                blb = Z0 - b if b2 is None else b2 - b1
                assert 0 < blb < 1 << 14
                assert B0 + pb * LB <= b and b + TC_N <= B0 + (pb + 1) * LB
                if b2 is None:
                    assert Z0 == b + blb                      # the zero block
                else:
                    assert b + blb + TC_N <= B0 + (pb + 1) * LB
    assert 16 * (Z0 + TC_N) < 1 << 18                         # 14-bit start addresses


@pytest.mark.parametrize("P", [15, 11, 7])
def test_accumulators_stay_below_2_24(P):
    """Worst case: every value 12240 (or -12240) in both operands."""
    hi, lo = split(np.array([12240, -12240]))
    mh, ml = np.abs(hi).max(), max(np.abs(lo).max(), 64)
    n = P * P * 6
    assert n * mh * mh < 2 ** 24                               # <a_h, b_h>
    assert n * 2 * mh * ml < 2 ** 24                           # <a_h, b_l> + <a_l, b_h>
    assert n * ml * ml < 2 ** 24                               # <a_l, b_l>
    v = np.arange(-12240, 12241)
    h, l = split(v)
    assert (128 * h + l == v).all() and l.min() >= -64 and l.max() <= 63
    assert np.abs(h).max() <= 96


def _model_cross(P, s, rw, rh, tw, th, rng):
    c, h = s // 2, P // 2
    nx, ny = lattice_n(rw, s), lattice_n(rh, s)
    R = rng.integers(-12240, 12241, size=(rh, rw, 8)); R[..., 6:] = 0
    T = rng.integers(-12240, 12241, size=(th, tw, 8)); T[..., 6:] = 0
    Rp = np.pad(R, ((BORD, BORD), (BORD, BORD), (0, 0)), mode="edge")
    Tp = np.pad(T, ((BORD, BORD), (BORD, BORD), (0, 0)), mode="edge")
    g = geom(P, s, nx, ny, tw, th)
    LA, LB, Wu, Wt, ph = g["LA"], g["LB"], g["Wu"], g["Wt"], g["ph"]
    st = steps(P, s, g)
    o = c - h
    got = np.zeros((ny * nx, th * tw), np.int64)
    for mt in range(g["mtiles"]):
        m0 = mt * TC_M
        v0 = m0 // Wu
        moff = m0 - v0 * Wu
        e = np.arange(ph * LA)
        phase, k = e // LA, e % LA
        f = v0 * Wu + k
        X = np.clip(s * (f % Wu) + phase % s + o, -BORD, rw + BORD - 1)
        Y = np.clip(s * (f // Wu) + phase // s + o, -BORD, rh + BORD - 1)
        Ah, Al = split(Rp[Y + BORD, X + BORD])
        A = np.concatenate([Ah, Al])                          # [part][phase][LA] flattened
        for band in range(g["bands"]):
            nb = band * TC_NT * TC_N
            f = nb + np.arange(LB)
            Xb = np.clip(f % Wt - h, -BORD, tw + BORD - 1)
            Yb = np.clip(f // Wt - h, -BORD, th + BORD - 1)
            Bh, Bl = split(Tp[Yb + BORD, Xb + BORD])
            Bm = np.concatenate([Bh, Bl, np.zeros((TC_N, 8), np.int64)])
            Z0 = 2 * LB
            for kt in range(min(TC_NT, g["ntiles"] - band * TC_NT)):
                acc = np.zeros((3, TC_M, TC_N), np.int64)
                rows_a, rows_b = np.arange(TC_M), np.arange(TC_N)
                for a1, a2, b1, b2 in st:
                    for pa in range(2):
                        a = pa * ph * LA + moff + a1
                        Am = np.concatenate([A[a + rows_a], A[a + (a2 - a1) + rows_a]], 1)
                        for pb in range(2):
                            b = pb * LB + kt * TC_N + b1
                            b_2 = Z0 if b2 is None else b + (b2 - b1)
                            Bt = np.concatenate([Bm[b + rows_b], Bm[b_2 + rows_b]], 1)
                            acc[pa + pb] += Am @ Bt.T
                assert np.abs(acc).max() < 2 ** 24
                cross = (acc[0] << 14) + (acc[1] << 7) + acc[2]
                mm = m0 + rows_a
                n = nb + kt * TC_N + rows_b
                sm = (mm % Wu < nx) & (mm // Wu < ny)
                sn = (n % Wt < tw) & (n // Wt < th)
                si = (mm // Wu * nx + mm % Wu)[sm]
                qi = (n // Wt * tw + n % Wt)[sn]
                got[np.ix_(si, qi)] = cross[np.ix_(sm, sn)]
    # brute force: clamped patches, plain correlation
    idx = lambda c0, n: np.clip(np.arange(c0, c0 + P), 0, n - 1)
    sp = np.stack([R[np.ix_(idx(c + s * j - h, rh), idx(c + s * i - h, rw))].reshape(-1)
                   for j in range(ny) for i in range(nx)])
    tp = np.stack([T[np.ix_(idx(y - h, th), idx(x - h, tw))].reshape(-1)
                   for y in range(th) for x in range(tw)])
    return got, sp @ tp.T


@pytest.mark.parametrize("P,s,rw,rh,tw,th", [(15, 3, 64, 28, 64, 28), (11, 3, 40, 20, 33, 17),
                                             (7, 1, 30, 18, 26, 14), (6, 2, 25, 13, 22, 15),
                                             (9, 4, 50, 19, 47, 23), (1, 3, 9, 9, 9, 9)])
def test_accumulators_give_the_exact_cross_terms(P, s, rw, rh, tw, th):
    got, want = _model_cross(P, s, rw, rh, tw, th, np.random.default_rng(P * 31 + s))
    assert (got == want).all()
