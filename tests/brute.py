"""Pure-Python brute force for tiny inputs -- a second, independent statement of
the method used to pin the C oracle (it imports nothing from it except the
Philox generator, which is itself pinned by the published known-answer vectors).

Everything here is plain loops over small images: the patch distance of Eq. 3,
the exhaustive initialisation, propagation (Eq. 4) and limited random search
(Eq. 5) in both schedules, the consistency check, the outlier-record update of
Eq. 6, the transfers of Eq. 7-8, and region removal by union-find.
"""
import numpy as np


def clamp(v, lo, hi):
    return lo if v < lo else (hi if v > hi else v)


def patch_dist(A, B, a, b, P, norm=0):
    """Eq. 3 with replicated borders; A, B planar [nch][h][w]."""
    nch, ha, wa = A.shape
    _, hb, wb = B.shape
    lo, hi = -(P // 2), P - 1 - P // 2
    s = 0
    for oy in range(lo, hi + 1):
        for ox in range(lo, hi + 1):
            xa, ya = clamp(a[0] + ox, 0, wa - 1), clamp(a[1] + oy, 0, ha - 1)
            xb, yb = clamp(b[0] + ox, 0, wb - 1), clamp(b[1] + oy, 0, hb - 1)
            for c in range(nch):
                d = int(A[c, ya, xa]) - int(B[c, yb, xb])
                s += d * d if norm == 0 else abs(d)
    return s


def lattice_n(W, sigma):
    c = sigma // 2
    return (W - 1 - c) // sigma + 1 if W - 1 - c >= 0 else 0


def rs_offset(r, k, W, mode):
    if mode == 0:
        rho = max(1, W >> k)
        return ((r * (2 * rho + 1)) >> 32) - rho
    return ((2 * r - (2 ** 32 - 1)) * W) // (2 ** (32 + k))   # Python // is floor


def schedule(L, N, ablation=0):
    if ablation & 1:
        N = 0
    m = L - 1
    lv, xo = [m], [0]
    if m > 0:
        for _ in range(N):
            lv += [m - 1, m]; xo += [1, 1]
        lv.append(m - 1); xo.append(0)
        for l in range(m - 2, -1, -1):
            lv.append(l); xo.append(1)
    if ablation & 4:
        xo = [0] * len(xo)
    return lv, xo


class Field:
    def __init__(self, nx, ny):
        self.nx, self.ny = nx, ny
        n = nx * ny
        self.ux = [0] * n; self.uy = [0] * n; self.valid = [0] * n
        self.cost = [None] * n; self.outl = [0] * n; self.oinit = [0] * n


def run_pipeline(prm, D1, D2, philox, schedule_kind=0, stream_id=0):
    """The whole matching schedule on tiny inputs.

    D1[s][l], D2[s][l]: planar descriptors of images 1 and 2 (scheme s, level l).
    philox(ctr, key) -> 4 uint32.  Returns {(level, dir): Field}.
    """
    L, sig = prm["levels"], prm["seed_stride"]
    c = sig // 2
    ns = len(D1)
    K = 0
    w = prm["rs_W"]
    while w >= 1:
        K += 1; w >>= 1
    key = (prm["philox_key"] & 0xFFFFFFFF, prm["philox_key"] >> 32)

    def imgs(l, d):
        s = min(d, ns - 1)
        return (D1[s][l], D2[s][l]) if d == 0 else (D2[s][l], D1[s][l])

    def P_of(d):
        return prm["patch_fwd"] if d == 0 else prm["patch_bwd"]

    fields = {}
    for l in range(L):
        for d in range(2):
            R, _ = imgs(l, d)
            fields[(l, d)] = Field(lattice_n(R.shape[2], sig), lattice_n(R.shape[1], sig))

    def inside(l, d, qx, qy):
        _, T = imgs(l, d)
        return 0 <= qx < T.shape[2] and 0 <= qy < T.shape[1]

    def cost(l, d, px, py, qx, qy):
        R, T = imgs(l, d)
        return patch_dist(R, T, (px, py), (qx, qy), P_of(d), prm["norm"])

    SX, SY = [1, -1, -1, 1], [1, -1, 1, -1]

    def update(l, d, v, t, i, j):
        F = fields[(l, d)]
        s = j * F.nx + i
        px, py = c + sig * i, c + sig * j
        have = F.valid[s]
        bu = (F.ux[s], F.uy[s])
        bc = F.cost[s] if have else None
        for ni, nj in ((i - SX[t % 4], j), (i, j - SY[t % 4])):
            if not (0 <= ni < F.nx and 0 <= nj < F.ny):
                continue
            n = nj * F.nx + ni
            if not F.valid[n]:
                continue
            cu = (F.ux[n], F.uy[n])
            if not inside(l, d, px + cu[0], py + cu[1]):
                continue
            cc = cost(l, d, px, py, px + cu[0], py + cu[1])
            if bc is None or cc < bc:
                bc, bu, have = cc, cu, 1
        g = prm.get("rs_grid", 0)
        if not have or (l == 0 and g > 0 and not (px % g == g // 2 and py % g == g // 2)):
            if have:
                F.ux[s], F.uy[s], F.valid[s], F.cost[s] = bu[0], bu[1], 1, bc
            return
        u0 = bu
        r = None
        for k in range(K):
            if k % 2 == 0:
                ctr = (s, (v << 16) | (d << 15) | t, (l << 16) | (k // 2), stream_id & 0xFFFFFFFF)
                r = philox(ctr, key)
            dx = rs_offset(int(r[2 * (k % 2)]), k, prm["rs_W"], prm["rs_mode"])
            dy = rs_offset(int(r[2 * (k % 2) + 1]), k, prm["rs_W"], prm["rs_mode"])
            cu = (u0[0] + dx, u0[1] + dy)
            if not inside(l, d, px + cu[0], py + cu[1]):
                continue
            cc = cost(l, d, px, py, px + cu[0], py + cu[1])
            if cc < bc:
                bc, bu = cc, cu
        F.ux[s], F.uy[s], F.valid[s], F.cost[s] = bu[0], bu[1], 1, bc

    lv, xo = schedule(L, prm["refine_rounds"], prm.get("ablation", 0))
    if prm.get("max_visits", 0) > 0:
        lv = lv[:prm["max_visits"]]
    prop_all = (prm.get("ablation", 0) >> 1) & 1
    for v, l in enumerate(lv):
        if v == 0:
            for d in range(2):
                F = fields[(l, d)]
                _, T = imgs(l, d)
                for j in range(F.ny):
                    for i in range(F.nx):
                        px, py = c + sig * i, c + sig * j
                        best = None
                        for qy in range(T.shape[1]):
                            for qx in range(T.shape[2]):
                                cc = cost(l, d, px, py, qx, qy)
                                if best is None or cc < best[0]:
                                    best = (cc, qx, qy)
                        s = j * F.nx + i
                        F.ux[s], F.uy[s] = best[1] - px, best[2] - py
                        F.valid[s], F.cost[s], F.outl[s], F.oinit[s] = 1, best[0], 0, 0
        else:
            src = lv[v - 1]
            for d in range(2):
                S, Dd = fields[(src, d)], fields[(l, d)]
                for y in range(Dd.ny):
                    for x in range(Dd.nx):
                        if l == src + 1:
                            al = [(2 * x + a, 2 * y + b) for b in (0, 1) for a in (0, 1)
                                  if 2 * x + a < S.nx and 2 * y + b < S.ny]
                        else:
                            al = [(min(x // 2, S.nx - 1), min(y // 2, S.ny - 1))]
                        al = [q[1] * S.nx + q[0] for q in al]
                        inl = [q for q in al if not S.outl[q]]
                        use = [q for q in al if (not S.outl[q]) or (prop_all and S.valid[q])]
                        t = y * Dd.nx + x
                        Dd.valid[t] = 1 if use else 0
                        Dd.ux[t] = Dd.uy[t] = 0
                        Dd.cost[t] = None
                        if use:
                            sx = sum(S.ux[q] for q in use); sy = sum(S.uy[q] for q in use)
                            if l == src + 1:
                                n = len(use)
                                Dd.ux[t] = (1 if sx >= 0 else -1) * ((abs(sx) + n) // (2 * n))
                                Dd.uy[t] = (1 if sy >= 0 else -1) * ((abs(sy) + n) // (2 * n))
                            else:
                                Dd.ux[t], Dd.uy[t] = 2 * sx, 2 * sy
                        if xo[v]:
                            Dd.outl[t], Dd.oinit[t] = (0 if inl else 1), 1
                        else:
                            Dd.outl[t], Dd.oinit[t] = 0, 0
        for d in range(2):                       # cost of the current u
            F = fields[(l, d)]
            for j in range(F.ny):
                for i in range(F.nx):
                    s = j * F.nx + i
                    if not F.valid[s]:
                        continue
                    px, py = c + sig * i, c + sig * j
                    qx, qy = px + F.ux[s], py + F.uy[s]
                    if not inside(l, d, qx, qy):
                        F.valid[s] = 0
                        continue
                    F.cost[s] = cost(l, d, px, py, qx, qy)
        T = prm["iters_fine"] if l == 0 else prm["iters_coarse"]
        for t in range(T):
            if schedule_kind == 0:
                for colour in (0, 1):
                    for d in (0, 1):
                        F = fields[(l, d)]
                        for j in range(F.ny):
                            for i in range(F.nx):
                                if (i + j) % 2 == colour:
                                    update(l, d, v, t, i, j)
            else:
                for d in (0, 1):
                    F = fields[(l, d)]
                    js = range(F.ny) if SY[t % 4] > 0 else range(F.ny - 1, -1, -1)
                    for j in js:
                        is_ = range(F.nx) if SX[t % 4] > 0 else range(F.nx - 1, -1, -1)
                        for i in is_:
                            update(l, d, v, t, i, j)
        C = {}
        for d in (0, 1):                         # consistency (both first)
            F, G = fields[(l, d)], fields[(l, 1 - d)]
            C[d] = []
            for j in range(F.ny):
                for i in range(F.nx):
                    s = j * F.nx + i
                    out = 1
                    if F.valid[s] and G.nx > 0 and G.ny > 0:
                        qx, qy = c + sig * i + F.ux[s], c + sig * j + F.uy[s]
                        gi = clamp((qx - c + sig // 2) // sig, 0, G.nx - 1)
                        gj = clamp((qy - c + sig // 2) // sig, 0, G.ny - 1)
                        g = gj * G.nx + gi
                        if G.valid[g]:
                            ex, ey = F.ux[s] + G.ux[g], F.uy[s] + G.uy[g]
                            out = 1 if ex * ex + ey * ey > prm["tau2"] else 0
                    C[d].append(out)
        for d in (0, 1):
            F = fields[(l, d)]
            for s in range(F.nx * F.ny):
                F.outl[s] = (F.outl[s] | C[d][s]) if F.oinit[s] else C[d][s]
    return fields


def region_keep(F, dmax2, min_region):
    """Region removal by union-find: inlier 4-neighbours join iff |du|^2 < dmax2."""
    n = F.nx * F.ny
    parent = list(range(n))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    inl = [F.valid[s] and not F.outl[s] for s in range(n)]
    for j in range(F.ny):
        for i in range(F.nx):
            s = j * F.nx + i
            if not inl[s]:
                continue
            for t in ([s + 1] if i + 1 < F.nx else []) + ([s + F.nx] if j + 1 < F.ny else []):
                if inl[t]:
                    dx, dy = F.ux[s] - F.ux[t], F.uy[s] - F.uy[t]
                    if dx * dx + dy * dy < dmax2:
                        a, b = find(s), find(t)
                        if a != b:
                            parent[max(a, b)] = min(a, b)
    size = {}
    for s in range(n):
        if inl[s]:
            r = find(s)
            size[r] = size.get(r, 0) + 1
    return np.array([1 if inl[s] and size[find(s)] >= min_region else 0 for s in range(n)],
                    np.uint8).reshape(F.ny, F.nx)
