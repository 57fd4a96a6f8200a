// pm_row.cu -- one checkerboard colour phase of propagation (Eq. 4) and
// limited random search (Eq. 5), and the cost refresh of a visit (the cost of
// every seed's current match), squared-L2 cost (Eq. 3), on seed tiles staged
// in shared memory.
//
// A tile is tw x th lattice seeds (tw th = 64; tw = 4, 8 or 16, a result-
// invariant tuning knob); its PR_NACT = 32 seeds of the current colour
// update.  A persistent CTA (one per SM) has PR_PROD producer warps and
// pr_cons consumer warps around a ring of tile buffers in shared memory, each
// with a "full" and an "empty" mbarrier:
//   - producer warp p stages the CTA's tiles p, p + PR_PROD, ...: it waits
//     until the tile's buffer is empty, reads the tile's seeds (one lane per
//     seed), drops the propagated candidates that cannot change the result,
//     draws the first Philox block of every seed, places the target window at
//     the per-component median of the current matches, and issues three 2D
//     tensor copies: the reference region of all the tile's patches
//     (split-byte words, a = 128 a_h + a_l), the target window (int16 words)
//     and the window's sums |b|^2;
//   - consumer warps take the tile's seeds from a shared counter, release the
//     buffer when the counter runs out and move on to the next tile.
// The descriptors carry a replicated border of BORD pixels in memory, so every
// patch whose centre lies in the image is read without clamping and every
// staged region is one tensor copy (coordinates outside the padded image read
// as zero and are never used).
//
// Consumer layout: a warp scores one seed at a time, up to two candidates per
// round.  Lane l owns the pixels k = l, l + 32, ... of the P x P patch in
// raster order and holds their reference words in registers (3 words per
// pixel for 6 channels, 1 for 2); a colour pixel of the target is one 16-byte
// load.  Reference region and window share one row pitch, congruent to P
// modulo 8 pixels, so pixel k of any patch lies in the 16-byte bank quad
// k + const (mod 8): the 8 lanes of a quarter-warp never collide.  The cross
// term <a, b> of a candidate is the warp sum (redux) of the lanes' dp2a
// partial sums over the low and the high bytes of a; then
//   D = sum |a|^2 + sum |b|^2 - 2 sum <a, b>,
// exact in integers, with sum |a|^2 per seed and sum |b|^2 per target pixel
// from the box filters of the same visit.  Over a patch of at most 16 x 16
// pixels and 6 values each the low and high sums stay below 2^31 in
// magnitude (1536 * 12240 * 96 < 1.9e9).  Candidates are compared in the
// paper's order (current match, the two propagated ones, then the random
// search around the match held after propagation) and replace the best only on
// a strictly lower cost, as in the sequential scan.  A candidate whose patch
// is not inside the window is read from the padded image in global memory.
#include <limits.h>
#include <mutex>

#include <cuda.h>

#include "match_common.cuh"

namespace pgm {

constexpr int PR_TILE = 64;                    // lattice seeds per tile (tw x th)
constexpr int PR_NACT = PR_TILE / 2;           // seeds of one colour per tile (one producer lane each)
constexpr int PR_PROD = 2;                     // producer warps
// consumer warps: 18 (20 warps of at most 96 registers), 14 for the colour
// layouts of 8 pixels per lane (P > 11), whose 24 reference words need more
__host__ __device__ constexpr int pr_cons(int nch, int PC) {
    return nch == 6 && (PC == 0 || PC > 11) ? 14 : 18;
}
constexpr int PR_NBUF = 3;                     // most tile buffers in the ring
constexpr int PR_MAPS = 32;                    // tensor-map slots of one launch
constexpr long long PR_DRAIN_CYCLES = 1ll << 31;   // final wait for issued copies (about 1 s)

struct RowGeom {
    int P, pxw;
    int tw, th;                       // tile shape in lattice seeds
    int ref_w, ref_h, win_w, win_h;   // staged regions (px)
    int sp;                           // words per shared row (reference region and window)
    int cw, ch, cwp;                  // window centres (cw x ch), row pitch of their sums (even)
    int off_win, off_sb, words;       // word offsets in a buffer, its size (multiples of 32)
    // bit-plane form (direction descriptor): words per staged bit row of the
    // reference region and of the window, offsets of their sign planes (the
    // nonzero planes start at 0 and off_win)
    int bwr, bww, off_rs, off_ws;
};

__host__ __device__ inline RowGeom rg_geom(int nch, int P, int sigma, int rs_W, int slack,
                                           int tw) {
    RowGeom g;
    g.P = P;
    g.pxw = px_words(nch);
    g.tw = tw;
    g.th = PR_TILE / tw;
    g.ref_w = sigma * (g.tw - 1) + P;
    g.ref_h = sigma * (g.th - 1) + P;
    const int rho = rs_W > 1 ? rs_W : 1;
    g.win_w = g.ref_w + 2 * (rho + slack);
    g.win_h = g.ref_h + 2 * (rho + slack);
    if (g.pxw == 4) {      // 16-byte pixels, pitch = P (mod 8) pixels
        int px = g.win_w;
        while ((px - P) % 8 != 0) ++px;
        g.sp = 4 * px;
    } else {               // words, + up to 3 of alignment shift, pitch = 16 (mod 32) words
        int w = g.win_w + 3;
        while (w % 32 != 16) ++w;
        g.sp = w;
    }
    g.cw = g.win_w - P + 1;
    g.ch = g.win_h - P + 1;
    g.cwp = (g.cw + 2) & ~1;                            // + 1 centre of alignment shift
    g.off_win = (g.sp * g.ref_h + 31) & ~31;            // regions start 128-byte aligned
    g.off_sb = (g.off_win + g.sp * g.win_h + 31) & ~31;
    g.words = (g.off_sb + 2 * g.cwp * g.ch + 31) & ~31;
    return g;
}

// The same staging for bit-planes (direction descriptor): a row of P pixels
// is P nch bits, read as NW aligned words from a staged row that starts at a
// 16-byte boundary (up to 127 bits before the first pixel); row pitches are 4
// (mod 8) words, so the 16 rows a half-warp reads meet at most 2 to a bank.
__host__ __device__ inline RowGeom rg_geom_bits(int nch, int P, int sigma, int rs_W, int slack,
                                                int tw) {
    RowGeom g = rg_geom(nch, P, sigma, rs_W, slack, tw);
    const int nw = nch == 6 ? 4 : 2;                      // words a lane reads per row
    auto pitch = [](int need) { while (need % 8 != 4) ++need; return need; };
    g.bwr = pitch((127 + sigma * (g.tw - 1) * nch) / 32 + nw);
    g.bww = pitch((127 + (g.win_w - P) * nch) / 32 + nw);
    g.off_rs = (g.bwr * g.ref_h + 31) & ~31;
    g.off_win = (g.off_rs + g.bwr * g.ref_h + 31) & ~31;
    g.off_ws = (g.off_win + g.bww * g.win_h + 31) & ~31;
    g.words = (g.off_ws + g.bww * g.win_h + 31) & ~31;
    g.off_sb = 0;
    return g;
}

namespace {

struct __align__(16) RowRec {       // one active seed of a staged tile
    int s, px, py, f;               // seed index (-1: none), centre, flags after the refresh
    int u, nb0, nb1, K;             // current match; propagated candidates to score; search count
    int r0, r1, f0, wr0;            // random-search offsets k = 0, 1 (packed like u); flags as read;
    int wu, w0, w1, wr1;            // window slots (row_slot) of u, nb0, nb1, and of the search
                                    // candidates k = 0, 1 around u (-2: not scored)
    unsigned long long cost, sa;    // current cost, sum |a|^2 of the reference patch
};

struct RowHdr { int pair, dir, rx0, ry0, wx0, wy0, use_win, shr, shw, shs, pad0, pad1; };

// The flattened tiles of one launch: slot k owns tiles [cum[k], cum[k + 1]);
// ndir = 1: slot k is pair k in direction dir; ndir = 2: slot k is pair k / 2
// in direction k % 2.
struct RowSched { int nk, total, dir, ndir; int cum[2 * MAXB + 1]; };

// Tensor maps of the staged arrays of every slot: [0] the padded reference
// split words, [1] the padded target descriptor, [2] the target sums |b|^2.
struct RowMaps { CUtensorMap m[PR_MAPS][3]; };

constexpr int NO_CAND = INT_MIN;             // no propagated candidate

__device__ __forceinline__ int lds32(unsigned addr) {
    int v;
    asm volatile("ld.shared.b32 %0, [%1];\n" : "=r"(v) : "r"(addr));
    return v;
}
__device__ __forceinline__ uint4 lds128(unsigned addr) {
    uint4 v;
    asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(addr));
    return v;
}
__device__ __forceinline__ unsigned long long lds64(unsigned addr) {
    unsigned long long v;
    asm volatile("ld.shared.b64 %0, [%1];\n" : "=l"(v) : "r"(addr));
    return v;
}
__device__ __forceinline__ void tma2d(unsigned dst, const CUtensorMap* map, int x, int y,
                                      unsigned bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];\n"
        ::"r"(dst), "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_test_wait(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    return ok != 0;
}
// Wait for phase `parity` of an mbarrier; give up after `limit` cycles or
// once another warp has flagged an abort.  The first look does not block
// (try_wait may suspend the thread for a while), so a limit of a few cycles
// runs out at once unless the phase is already complete.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, long long limit,
                                          const volatile int* abort) {
    const long long t0 = clock64();
    if (mbar_test_wait(bar, parity)) return true;
    for (;;) {
        if (abort && *abort) return false;
        if (clock64() - t0 > limit) return false;
        if (mbar_try_wait(bar, parity)) return true;
    }
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// Window slot of target centre (qx, qy): the word offset of its patch corner
// from the window start in the low 16 bits, the index of its sum |b|^2 above;
// -1 when the patch is not inside the staged window.
__device__ __forceinline__ int row_slot(const RowGeom& G, const RowHdr& H, int P, int qx, int qy) {
    const int x0 = qx - P / 2 - H.wx0, y0 = qy - P / 2 - H.wy0;
    if (!H.use_win || x0 < 0 || y0 < 0 || x0 + P > G.win_w || y0 + P > G.win_h) return -1;
    return (y0 * G.sp + H.shw + x0 * G.pxw) | ((y0 * G.cwp + H.shs + x0) << 16);
}

// The slot of a candidate for the producer: row_slot, or for the bit-plane
// form its patch corner (y0, x0) in the window as y0 << 16 | x0 (-1 outside).
template <bool BITS>
__device__ __forceinline__ int pr_slot(const RowGeom& G, const RowHdr& H, int P, int qx, int qy) {
    if constexpr (BITS) {
        const int x0 = qx - P / 2 - H.wx0, y0 = qy - P / 2 - H.wy0;
        if (!H.use_win || x0 < 0 || y0 < 0 || x0 + P > G.win_w || y0 + P > G.win_h) return -1;
        return (y0 << 16) | x0;
    } else {
        return row_slot(G, H, P, qx, qy);
    }
}

// Producer warp p: stage the CTA's tiles n = p, p + PR_PROD, ... (launch tiles
// blockIdx.x + n * gridDim.x) into buffer n mod nbuf.
// NG = 0: one full and one empty mbarrier per buffer; every consumer warp
// takes every tile, so waits see the phases of a buffer one after another.
// NG > 0: consumer agent g takes the tiles n = g (mod NG) and a buffer
// rotates among agents and producers, so a parity wait could otherwise
// skip a phase; buffer b then has a full barrier per agent (b NG + g, the
// phases of that agent's tiles in b) and an empty barrier per producer
// (b NPROD + p, released by the consumers of the tile before producer p's
// next tile in b), and every wait is for the next phase of its barrier.
template <int NCH, bool BITS, int NPROD, int NBUFMAX, int NG = 0>
__device__ void pr_produce(const LvlBatch& B, const MatchConst& mc, const RowSched& S,
                           const RowMaps& TM, int buf_words, int nbuf, unsigned a_sm,
                           RowRec (*rec)[PR_NACT], RowHdr* hdr, int* next, const RowGeom* geom,
                           unsigned full0, unsigned empty0, volatile int* abort, long long limit,
                           int pw, int lane) {
    constexpr int PXW = px_words(NCH);
    int lastn[NBUFMAX];                      // the tile this warp last armed in each buffer
    int waits[NBUFMAX];                      // NG > 0: waits so far on this warp's empty barrier of b
#pragma unroll
    for (int b = 0; b < NBUFMAX; ++b) { lastn[b] = -1; waits[b] = 0; }
    for (int n = pw;; n += NPROD) {
        const int t = blockIdx.x + n * gridDim.x;
        if (t >= S.total) break;
        const int b = n % nbuf;
        const unsigned full = full0 + 8u * (NG > 0 ? (unsigned)(b * NG + n % NG) : (unsigned)b);
        const unsigned empty = empty0 + 8u * (NG > 0 ? (unsigned)(b * NPROD + pw) : (unsigned)b);
        if (n >= nbuf) {            // the consumers released the buffer's last tile
            const unsigned par = NG > 0 ? (unsigned)(waits[b]++) & 1u : (unsigned)((n / nbuf) - 1) & 1u;
            const bool ok = __all_sync(FULL, mbar_wait(empty, par, limit, abort));
            if (!ok) {
                if (lane == 0 && !*abort) {
                    for (int k = 0; k < B.n; ++k) atomicOr(B.err[k], (unsigned)PGM_ERR_TIMEOUT);
                    *abort = 1;
                }
                break;
            }
        }
        if (*abort) break;
        int lo = 0, hi = S.nk - 1;                   // slot holding tile t:
        while (lo < hi) {                            // the last k with cum[k] <= t
            const int mid = (lo + hi + 1) >> 1;
            if (S.cum[mid] <= t) lo = mid; else hi = mid - 1;
        }
        const int k = lo, pair = S.ndir == 2 ? k >> 1 : k, dir = S.ndir == 2 ? (k & 1) : S.dir;
        const RowGeom& G = geom[dir];
        const DirLvl& D = B.d[pair][dir];
        const int tiles_x = (D.nx + G.tw - 1) / G.tw, tt = t - S.cum[k];
        const int i0 = (tt % tiles_x) * G.tw, j0 = (tt / tiles_x) * G.th;
        const int P = D.P, h = P / 2, sig = mc.sigma;
        const int rx0 = mc.c + sig * i0 - h, ry0 = mc.c + sig * j0 - h;
        // bit-plane form: first staged word (a multiple of 4) and bit shift
        const int rbit = (rx0 + BORD) * NCH, rws = (rbit >> 5) & ~3;
        const int shr = BITS ? rbit - 32 * rws : PXW == 4 ? 0 : ((rx0 + BORD) & 3);
        const unsigned buf = a_sm + 4u * (unsigned)(b * buf_words);
        fence_proxy_async();                         // the consumers' reads of this buffer come first
        if (lane == 0) {                             // the reference region does not depend on the seeds
            if constexpr (BITS) {                    // nonzero rows, then sign rows H + 2 BORD below
                mbar_expect_tx(full, 8u * (unsigned)(G.bwr * G.ref_h));
                tma2d(buf, &TM.m[k][0], rws, ry0 + BORD, full);
                tma2d(buf + 4u * (unsigned)G.off_rs, &TM.m[k][0], rws, D.rh + 2 * BORD + ry0 + BORD, full);
            } else {
                mbar_expect_tx(full, 4u * (unsigned)(G.sp * G.ref_h));
                tma2d(buf, &TM.m[k][0], PXW == 4 ? 2 * (rx0 + BORD) : rx0 + BORD - shr, ry0 + BORD, full);
            }
        }
        // the seed of this lane: active seed a = lane of the tile (Eq. 4 candidates, Eq. 5 draws)
        const int t4 = mc.t & 3;
        const int sx = (t4 == 0 || t4 == 3) ? 1 : -1, sy = (t4 == 0 || t4 == 2) ? 1 : -1;
        const int a = lane, j = j0 + a / (G.tw / 2);
        const int i = i0 + 2 * (a % (G.tw / 2)) + ((j + mc.colour) & 1);
        RowRec R;
        R.s = -1; R.px = 0; R.py = 0; R.f = 0; R.u = 0; R.nb0 = NO_CAND; R.nb1 = NO_CAND; R.K = 0;
        R.r0 = 0; R.r1 = 0; R.f0 = 0; R.wr0 = -2; R.wu = -1; R.w0 = -1; R.w1 = -1; R.wr1 = -2;
        R.cost = INF; R.sa = 0;
        if (i < D.nx && j < D.ny) {
            const int s = j * D.nx + i;
            const int px = mc.c + sig * i, py = mc.c + sig * j;
            const int f = D.flags[s], u = D.u[s];
            // (the bit-plane cost needs no sum |a|^2, and no box sums are made for it)
            const unsigned long long cst = D.cost[s], sa = BITS ? 0ull : D.sa2img[(size_t)py * D.rw + px];
            bool have = f & F_VALID;
            // the refresh (first iteration of a visit) drops a match whose centre
            // left the target, here and at the neighbours
            if (mc.refresh) have = have && inside(D, px + lo16((uint32_t)u), py + hi16((uint32_t)u));
            int c0 = NO_CAND, c1 = NO_CAND;
            if (!mc.cost_only) {
                const int ni = i - sx, nj = j - sy;
                const bool okx = ni >= 0 && ni < D.nx, oky = nj >= 0 && nj < D.ny;
                const int sn0 = okx ? j * D.nx + ni : s, sn1 = oky ? nj * D.nx + i : s;
                const int f0 = D.flags[sn0], f1 = D.flags[sn1], u0 = D.u[sn0], u1 = D.u[sn1];
                bool ok_n0 = okx && (f0 & F_VALID), ok_n1 = oky && (f1 & F_VALID);
                if (mc.refresh) {
                    ok_n0 = ok_n0 && inside(D, px - sx * sig + lo16((uint32_t)u0), py + hi16((uint32_t)u0));
                    ok_n1 = ok_n1 && inside(D, px + lo16((uint32_t)u1), py - sy * sig + hi16((uint32_t)u1));
                }
                // a candidate equal to the current match or to the other
                // candidate scores the same and cannot be strictly better
                if (ok_n0 && !(have && u0 == u) &&
                    inside(D, px + lo16((uint32_t)u0), py + hi16((uint32_t)u0)))
                    c0 = u0;
                if (ok_n1 && !(ok_n0 && u1 == u0) && !(have && u1 == u) &&
                    inside(D, px + lo16((uint32_t)u1), py + hi16((uint32_t)u1)))
                    c1 = u1;
            }
            R.s = s; R.px = px; R.py = py; R.u = u;
            R.f = have ? f : (f & ~F_VALID);
            R.f0 = f;
            R.nb0 = c0;
            R.nb1 = c1;
            R.cost = mc.refresh ? INF : cst;
            R.sa = sa;
            const int g = mc.rs_grid;                 // PGM-C3/G3: level-0 search on a grid only
            R.K = mc.cost_only ? 0
                  : (B.level == 0 && g > 0 && !(px % g == g / 2 && py % g == g / 2)) ? 0 : mc.K;
            if (R.K > 0) {
                const uint4 r = philox(
                    make_uint4((uint32_t)s,
                               ((uint32_t)B.visit << 16) | ((uint32_t)dir << 15) | (uint32_t)mc.t,
                               (uint32_t)B.level << 16, B.stream_id[pair]),
                    mc.key0, mc.key1);
                R.r0 = pack_u(rs_off(r.x, 0, mc.rs_W, mc.rs_mode), rs_off(r.y, 0, mc.rs_W, mc.rs_mode));
                R.r1 = pack_u(rs_off(r.z, 1, mc.rs_W, mc.rs_mode), rs_off(r.w, 1, mc.rs_W, mc.rs_mode));
            }
        }
        // window centre: per component, the median of the valid current
        // matches, the (nv / 2)-th smallest (0-based), found one bit at a time
        // over the offsets from the smallest value (only the bits in which the
        // tile's values differ)
        const bool v = R.s >= 0 && (R.f & F_VALID);
        const unsigned vm = __ballot_sync(FULL, v);
        const int nv = __popc(vm);
        const int ux = lo16((uint32_t)R.u), uy = hi16((uint32_t)R.u);
        const int lox = __reduce_min_sync(FULL, v ? ux : INT_MAX);
        const int loy = __reduce_min_sync(FULL, v ? uy : INT_MAX);
        const unsigned kx = v ? (unsigned)(ux - lox) : 0u, ky = v ? (unsigned)(uy - loy) : 0u;
        const unsigned span = __reduce_or_sync(FULL, kx | ky);
        unsigned cx = vm, cy = vm;
        int mx = nv / 2, my = nv / 2;
        for (int bit = span ? 31 - __clz(span) : -1; bit >= 0; --bit) {
            const unsigned zx = __ballot_sync(FULL, !((kx >> bit) & 1u)) & cx;
            const unsigned zy = __ballot_sync(FULL, !((ky >> bit) & 1u)) & cy;
            const int px_ = __popc(zx), py_ = __popc(zy);
            if (mx < px_) cx = zx; else { mx -= px_; cx &= ~zx; }
            if (my < py_) cy = zy; else { my -= py_; cy &= ~zy; }
        }
        const int rho = max(1, mc.rs_W);
        const int medx = __shfl_sync(FULL, ux, cx ? __ffs(cx) - 1 : 0);
        const int medy = __shfl_sync(FULL, uy, cy ? __ffs(cy) - 1 : 0);
        RowHdr H;
        H.pair = pair; H.dir = dir; H.rx0 = rx0; H.ry0 = ry0;
        H.use_win = nv > 0;
        H.wx0 = nv > 0 ? rx0 + medx - rho - mc.slack : 0;
        H.wy0 = nv > 0 ? ry0 + medy - rho - mc.slack : 0;
        H.shr = shr;
        const int wbit = (H.wx0 + BORD) * NCH, wws = (wbit >> 5) & ~3;
        H.shw = BITS ? wbit - 32 * wws : PXW == 4 ? 0 : ((H.wx0 + BORD) & 3);
        H.shs = (H.wx0 + h) & 1;
        H.pad0 = wws; H.pad1 = 0;
        // the window slots of the candidates known now
        R.wu = R.s >= 0 ? pr_slot<BITS>(G, H, P, R.px + lo16((uint32_t)R.u), R.py + hi16((uint32_t)R.u)) : -1;
        R.w0 = R.nb0 != NO_CAND ? pr_slot<BITS>(G, H, P, R.px + lo16((uint32_t)R.nb0), R.py + hi16((uint32_t)R.nb0)) : -1;
        R.w1 = R.nb1 != NO_CAND ? pr_slot<BITS>(G, H, P, R.px + lo16((uint32_t)R.nb1), R.py + hi16((uint32_t)R.nb1)) : -1;
        // the first two search candidates around the current match, the
        // centre of the search unless a propagated match wins
        if (R.s >= 0 && (R.f & F_VALID) && R.K > 0) {
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const uint32_t o = (uint32_t)(k ? R.r1 : R.r0);
                const int qx = R.px + ux + lo16(o), qy = R.py + uy + hi16(o);
                const bool ok = k < R.K && o != 0u && inside(D, qx, qy);
                const int w = ok ? pr_slot<BITS>(G, H, P, qx, qy) : -2;
                if (k) R.wr1 = w; else R.wr0 = w;
            }
        }
        rec[b][a] = R;
        if (lane == 0) {
            hdr[b] = H;
            next[b] = 0;
        }
        __syncwarp();
        if (lane == 0) {
            if (H.use_win) {
                if constexpr (BITS) {
                    mbar_arrive_tx(full, 8u * (unsigned)(G.bww * G.win_h));
                    tma2d(buf + 4u * (unsigned)G.off_win, &TM.m[k][1], wws, H.wy0 + BORD, full);
                    tma2d(buf + 4u * (unsigned)G.off_ws, &TM.m[k][1], wws,
                          D.th + 2 * BORD + H.wy0 + BORD, full);
                } else {
                    mbar_arrive_tx(full, 4u * (unsigned)(G.sp * G.win_h) + 8u * (unsigned)(G.cwp * G.ch));
                    tma2d(buf + 4u * (unsigned)G.off_win, &TM.m[k][1],
                          PXW == 4 ? 2 * (H.wx0 + BORD) : H.wx0 + BORD - H.shw, H.wy0 + BORD, full);
                    tma2d(buf + 4u * (unsigned)G.off_sb, &TM.m[k][2], H.wx0 + h - H.shs, H.wy0 + h, full);
                }
            } else {
                mbar_arrive(full);
            }
        }
        lastn[b] = n;
    }
    // after an abort: let the copies this warp issued land before the CTA exits
    if (*abort)
        for (int b = 0; b < nbuf; ++b)
            if (lastn[b] >= 0) {
                const int m = lastn[b];
                unsigned bar = (unsigned)b, ph = (unsigned)(m / nbuf);
                if (NG > 0) {             // the phase of tile m on its agent's barrier of b
                    bar = (unsigned)(b * NG + m % NG);
                    ph = 0;
                    for (int q = b; q < m; q += nbuf) ph += q % NG == m % NG;
                }
                (void)mbar_wait(full0 + 8u * bar, ph & 1u, PR_DRAIN_CYCLES, nullptr);
            }
}

// Partial cross products of one lane's pixels with the candidate patch whose
// corner is at shared byte address `base`: lane pixel m at base + off[m].
// Accumulators l[], h[] (low / high bytes of the reference).
template <int NCH, int M>
__device__ __forceinline__ void pr_acc_sh(const int (&ra)[M][NCH / 2], const unsigned (&off)[M],
                                          unsigned base, int (&l)[3], int (&h)[3]) {
#pragma unroll
    for (int m = 0; m < M; ++m) {
        if constexpr (NCH == 6) {
            const uint4 v = lds128(base + off[m]);
            l[0] = __dp2a_lo((int)v.x, ra[m][0], l[0]);
            h[0] = __dp2a_hi((int)v.x, ra[m][0], h[0]);
            l[1] = __dp2a_lo((int)v.y, ra[m][1], l[1]);
            h[1] = __dp2a_hi((int)v.y, ra[m][1], h[1]);
            l[2] = __dp2a_lo((int)v.z, ra[m][2], l[2]);
            h[2] = __dp2a_hi((int)v.z, ra[m][2], h[2]);
        } else {
            const int v = lds32(base + off[m]);
            l[m % 3] = __dp2a_lo(v, ra[m][0], l[m % 3]);
            h[m % 3] = __dp2a_hi(v, ra[m][0], h[m % 3]);
        }
    }
}
// The same from the padded target image in global memory (a patch outside
// the window): the patch corner is pixel (x0, y0) of an image with rows of
// `pitch` words; the lane's pixels are walked in raster order.
template <int NCH, int M>
__device__ __forceinline__ void pr_acc_glob(const int (&ra)[M][NCH / 2], const uint32_t* img,
                                            int pitch, int x0, int y0, int P, int lane,
                                            int (&l)[3], int (&h)[3]) {
    constexpr int PXW = px_words(NCH);
    int row = 0, col = lane;
    while (col >= P) { col -= P; ++row; }
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const bool in = row < P;
        const uint32_t* p = img + (ptrdiff_t)(y0 + (in ? row : 0)) * pitch +
                            (ptrdiff_t)(x0 + (in ? col : 0)) * PXW;
        if constexpr (NCH == 6) {
            const uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
            l[0] = __dp2a_lo((int)v.x, ra[m][0], l[0]);
            h[0] = __dp2a_hi((int)v.x, ra[m][0], h[0]);
            l[1] = __dp2a_lo((int)v.y, ra[m][1], l[1]);
            h[1] = __dp2a_hi((int)v.y, ra[m][1], h[1]);
            l[2] = __dp2a_lo((int)v.z, ra[m][2], l[2]);
            h[2] = __dp2a_hi((int)v.z, ra[m][2], h[2]);
        } else {
            const int v = (int)__ldg(p);
            l[m % 3] = __dp2a_lo(v, ra[m][0], l[m % 3]);
            h[m % 3] = __dp2a_hi(v, ra[m][0], h[m % 3]);
        }
        col += 32;
        while (col >= P) { col -= P; ++row; }
    }
}

// Six-channel pixels, P = 15, staged rows of a compile-time pitch SP words:
// lane l < 30 holds column l mod 15 of patch rows 2m + l div 15 (m = 0 .. 7,
// row 15 counting zero); lanes 30 and 31 read columns 15 and 16 of the odd
// rows and count zero.  Every load of pixel m then sits 8 SP m bytes from the
// lane's own base, an immediate offset.  The extra row and columns stay in
// the staged buffer: a region's last row is followed by the next region (the
// window after the reference rows, the sums after the window), and a row's
// pitch exceeds the window width by more than two pixels.
constexpr int PR_ROWS_SP = 188;                // the pitch of the default tiles (8 x 8, margin 2)
template <int OFF>
__device__ __forceinline__ uint4 lds128_at(unsigned addr) {
    uint4 v;
    asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4+%5];\n"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(addr), "n"(OFF));
    return v;
}
template <int SP, int m = 0>
__device__ __forceinline__ void pr_ref_rows(int (&ra)[8][3], unsigned base, unsigned vmask) {
    if constexpr (m < 8) {
        const uint4 v = lds128_at<8 * SP * m>(base);
        const int keep = ((vmask >> m) & 1u) ? -1 : 0;
        ra[m][0] = (int)v.x & keep;
        ra[m][1] = (int)v.y & keep;
        ra[m][2] = (int)v.z & keep;
        pr_ref_rows<SP, m + 1>(ra, base, vmask);
    }
}
template <int SP, int m = 0>
__device__ __forceinline__ void pr_acc_rows(const int (&ra)[8][3], unsigned base, int (&l)[3],
                                            int (&h)[3]) {
    if constexpr (m < 8) {
        const uint4 v = lds128_at<8 * SP * m>(base);
        l[0] = __dp2a_lo((int)v.x, ra[m][0], l[0]);
        h[0] = __dp2a_hi((int)v.x, ra[m][0], h[0]);
        l[1] = __dp2a_lo((int)v.y, ra[m][1], l[1]);
        h[1] = __dp2a_hi((int)v.y, ra[m][1], h[1]);
        l[2] = __dp2a_lo((int)v.z, ra[m][2], l[2]);
        h[2] = __dp2a_hi((int)v.z, ra[m][2], h[2]);
        pr_acc_rows<SP, m + 1>(ra, base, l, h);
    }
}
// the same lanes' pixels from the padded target image in global memory
// (pixels a lane does not hold read the patch corner)
__device__ __forceinline__ void pr_acc_glob_rows(const int (&ra)[8][3], const uint32_t* img,
                                                 int pitch, int x0, int y0, int r0, int col,
                                                 unsigned vmask, int (&l)[3], int (&h)[3]) {
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const bool in = (vmask >> m) & 1u;
        const uint32_t* p = img + (ptrdiff_t)(y0 + (in ? 2 * m + r0 : 0)) * pitch +
                            (ptrdiff_t)(x0 + (in ? col : 0)) * 4;
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
        l[0] = __dp2a_lo((int)v.x, ra[m][0], l[0]);
        h[0] = __dp2a_hi((int)v.x, ra[m][0], h[0]);
        l[1] = __dp2a_lo((int)v.y, ra[m][1], l[1]);
        h[1] = __dp2a_hi((int)v.y, ra[m][1], h[1]);
        l[2] = __dp2a_lo((int)v.z, ra[m][2], l[2]);
        h[2] = __dp2a_hi((int)v.z, ra[m][2], h[2]);
    }
}

// Consumer warps: for every tile of the CTA, the active seeds taken one at a
// time from the buffer's counter.  PC > 0: the patch side of every pair of the
// launch (compile time), else at most MAXP (run time).
template <int NCH, int PC, int SP = 0>
__device__ void pr_consume(const LvlBatch& B, const MatchConst& mc, const RowSched& S,
                           int buf_words, int nbuf, unsigned a_sm, const uint32_t* sm_gen,
                           RowRec (*rec)[PR_NACT], const RowHdr* hdr, int* next,
                           const RowGeom* geom, unsigned full0, unsigned empty0,
                           volatile int* abort, long long limit, int lane) {
    constexpr int PXW = px_words(NCH), WPP = NCH / 2;
    constexpr int M = PC > 0 ? (PC * PC + 31) / 32 : (MAXP * MAXP) / 32;   // pixels per lane
    static_assert(SP == 0 || (NCH == 6 && PC == 15), "fixed-pitch rows: six channels, P = 15");
    int cur_dir = -1, P = 0, h = 0;
    unsigned off[M];                 // byte offset of lane pixel m from a patch corner
    unsigned vmask = 0;              // bit m: lane pixel m lies in the patch
    unsigned lane_off = 0;           // SP > 0: byte offset of the lane's first pixel
    int r0 = 0, lcol = 0;            //         its patch row (0, 1) and column
    for (int n = 0;; ++n) {
        const int t = blockIdx.x + n * gridDim.x;
        if (t >= S.total) break;
        const int b = n % nbuf;
        if (!__all_sync(FULL, mbar_wait(full0 + 8u * b, (unsigned)(n / nbuf) & 1u, limit, abort))) {
            if (lane == 0 && !*abort) {
                for (int k = 0; k < B.n; ++k) atomicOr(B.err[k], (unsigned)PGM_ERR_TIMEOUT);
                *abort = 1;
            }
            break;
        }
        const RowHdr H = hdr[b];
        const RowGeom& G = geom[H.dir];
        const DirLvl& D = B.d[H.pair][H.dir];
        if (H.dir != cur_dir && SP > 0) {   // rows 2 m + r0 of column lcol
            cur_dir = H.dir;
            P = PC;
            h = P / 2;
            r0 = lane < 15 ? 0 : 1;
            lcol = lane < 30 ? lane % 15 : lane - 15;
            lane_off = 4u * (unsigned)(r0 * SP + lcol * 4);
            vmask = lane < 30 ? (lane < 15 ? 0xffu : 0x7fu) : 0u;
        }
        if (H.dir != cur_dir) {      // the lane's pixels k = lane + 32 m of a P x P patch
            cur_dir = H.dir;
            P = PC > 0 ? PC : G.P;
            h = P / 2;
            int row = 0, col = lane;
            while (col >= P) { col -= P; ++row; }
            vmask = 0;
#pragma unroll
            for (int m = 0; m < M; ++m) {
                const bool in = row < P;
                off[m] = in ? 4u * (unsigned)(row * G.sp + col * PXW) : 0u;
                vmask |= in ? 1u << m : 0u;
                col += 32;
                while (col >= P) { col -= P; ++row; }
            }
        }
        const unsigned buf = a_sm + 4u * (unsigned)(b * buf_words);
        const unsigned a_win = buf + 4u * (unsigned)G.off_win, a_sb = buf + 4u * (unsigned)G.off_sb;
        const uint32_t* t32 = reinterpret_cast<const uint32_t*>(D.tgt);
        const int tpw = D.tgt_pitch >> 1;                     // words per padded target row
        unsigned n_eval = 0, n_cost = 0, n_glob = 0;
        for (;;) {
            int a = 0;
            if (lane == 0) a = atomicAdd(next + b, 1);
            a = __shfl_sync(FULL, a, 0);
            if (a >= PR_NACT) break;
            const RowRec R = rec[b][a];
            const int s = R.s;
            if (s < 0) continue;
            const int Rf = R.f, Ru = R.u;
            bool have = Rf & F_VALID;
            if (!have && R.nb0 == NO_CAND && R.nb1 == NO_CAND) {     // nothing to score
                if (lane == 0 && Rf != R.f0) D.flags[s] = (uint8_t)Rf;   // the refresh dropped it
                continue;
            }
            const int px = R.px, py = R.py;
            const unsigned long long sa = R.sa;
            // this lane's reference words (zero for pixels past the patch)
            int ra[M][WPP];
            {
                const int roff = (py - h - H.ry0) * G.sp + H.shr + (px - h - H.rx0) * PXW;
                const bool rok = PGM_CHECK(py - h - H.ry0 >= 0 && px - h - H.rx0 >= 0 &&
                                           roff + (P - 1) * G.sp + P * PXW <= G.sp * G.ref_h,
                                           B.err[H.pair]);
                const unsigned rbase = buf + 4u * (unsigned)(rok ? roff : 0);
                if constexpr (SP > 0) pr_ref_rows<SP>(ra, rbase + lane_off, vmask);
                else
#pragma unroll
                for (int m = 0; m < M; ++m) {
                    // (pixel m of every lane lies in the patch for m < P^2 / 32)
                    const int keep = (PC > 0 && m < (PC * PC) / 32) || ((vmask >> m) & 1u) ? -1 : 0;
                    if constexpr (NCH == 6) {
                        const uint4 v = lds128(rbase + off[m]);
                        ra[m][0] = (int)v.x & keep;
                        ra[m][1] = (int)v.y & keep;
                        ra[m][2] = (int)v.z & keep;
                    } else {
                        ra[m][0] = lds32(rbase + off[m]) & keep;
                    }
                }
            }
            // the cost of one candidate (centre qx, qy; window slot, -1: read
            // from the padded image in global memory); uniform over the warp
            auto eval = [&](int slot, int qx, int qy) -> unsigned long long {
                int l[3] = {0, 0, 0}, hh[3] = {0, 0, 0};
                unsigned long long sb;
                if (slot >= 0) {
                    if (PGM_CHECK((slot & 0xffff) + (P - 1) * G.sp + P * PXW <= G.sp * G.win_h &&
                                  (slot >> 16) < G.cwp * G.ch, B.err[H.pair])) {
                        if constexpr (SP > 0)
                            pr_acc_rows<SP>(ra, a_win + 4u * (unsigned)(slot & 0xffff) + lane_off, l, hh);
                        else
                            pr_acc_sh<NCH, M>(ra, off, a_win + 4u * (unsigned)(slot & 0xffff), l, hh);
                        sb = lds64(a_sb + 8u * (unsigned)(slot >> 16));
                    } else {
                        sb = 0;
                    }
                } else {
                    if (PGM_CHECK(qx >= 0 && qy >= 0 && qx < D.tw && qy < D.th && h <= BORD,
                                  B.err[H.pair])) {
                        if constexpr (SP > 0)
                            pr_acc_glob_rows(ra, t32, tpw, qx - h, qy - h, r0, lcol, vmask, l, hh);
                        else
                            pr_acc_glob<NCH, M>(ra, t32, tpw, qx - h, qy - h, P, lane, l, hh);
                        sb = D.sb2[(size_t)qy * D.sbp + qx];
                    } else {
                        sb = 0;
                    }
                    if (lane == 0) ++n_glob;
                }
                const int sl = __reduce_add_sync(FULL, l[0] + l[1] + l[2]);
                const int sh = __reduce_add_sync(FULL, hh[0] + hh[1] + hh[2]);
                return xcost(sa, sb, (long long)sh * 128 + (long long)sl);
            };
            // the candidates in the paper's order, each scored by the whole
            // warp: the current match (cost refresh; R.cost is INF then), the
            // propagated matches (Eq. 4), then the limited random search (Eq.
            // 5) around the match held after propagation
            unsigned long long bc = have ? R.cost : INF;
            int32_t bu = Ru;
            if (mc.refresh && have) {
                bc = eval(R.wu, px + lo16((uint32_t)Ru), py + hi16((uint32_t)Ru));
                ++n_cost;
            }
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int cu = c ? R.nb1 : R.nb0;
                if (cu == NO_CAND) continue;
                const unsigned long long v = eval(c ? R.w1 : R.w0, px + lo16((uint32_t)cu),
                                                  py + hi16((uint32_t)cu));
                ++n_eval;
                if (v < bc) { bc = v; bu = cu; have = true; }
            }
            const int K = R.K;
            if (have && K > 0) {
                const int cx0 = lo16((uint32_t)bu), cy0 = hi16((uint32_t)bu);
                int k = 0;
                if (bu == Ru && (Rf & F_VALID)) {    // centre = current match: slots from the producer
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const int w = c ? R.wr1 : R.wr0;
                        if (w == -2) continue;
                        const uint32_t o = (uint32_t)(c ? R.r1 : R.r0);
                        const int dx = lo16(o), dy = hi16(o);
                        const unsigned long long v = eval(w, px + cx0 + dx, py + cy0 + dy);
                        ++n_eval;
                        if (v < bc) { bc = v; bu = pack_u(cx0 + dx, cy0 + dy); }
                    }
                    k = 2;
                }
                for (; k < K; ++k) {
                    int dx, dy;
                    if (k < 2) {
                        const uint32_t o = (uint32_t)(k ? R.r1 : R.r0);
                        dx = lo16(o);
                        dy = hi16(o);
                    } else {
                        const uint4 rq = philox(
                            make_uint4((uint32_t)s,
                                       ((uint32_t)B.visit << 16) | ((uint32_t)H.dir << 15) | (uint32_t)mc.t,
                                       ((uint32_t)B.level << 16) | (uint32_t)(k >> 1),
                                       B.stream_id[H.pair]),
                            mc.key0, mc.key1);
                        dx = rs_off((k & 1) ? rq.z : rq.x, k, mc.rs_W, mc.rs_mode);
                        dy = rs_off((k & 1) ? rq.w : rq.y, k, mc.rs_W, mc.rs_mode);
                    }
                    if (dx == 0 && dy == 0) continue;
                    const int qx = px + cx0 + dx, qy = py + cy0 + dy;   // tested before packing
                    if (!inside(D, qx, qy)) continue;
                    const unsigned long long v = eval(row_slot(G, H, P, qx, qy), qx, qy);
                    ++n_eval;
                    if (v < bc) { bc = v; bu = pack_u(cx0 + dx, cy0 + dy); }
                }
            }
            if (lane == 0) {
                if (have && (mc.refresh || bu != Ru || !(Rf & F_VALID))) {
                    D.u[s] = bu;
                    D.cost[s] = bc;
                    D.flags[s] = (uint8_t)(Rf | F_VALID);
                } else if (!have && Rf != R.f0) {
                    D.flags[s] = (uint8_t)Rf;
                }
            }
        }
        if (lane == 0) {
            if (n_eval) atomicAdd(B.evals[H.pair] + H.dir, (unsigned long long)n_eval);
            if (n_cost) atomicAdd(B.evals[H.pair] + 2 + H.dir, (unsigned long long)n_cost);
            if (n_glob) atomicAdd(B.evals[H.pair] + 6 + H.dir, (unsigned long long)n_glob);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(empty0 + 8u * b);         // this warp is done with the buffer
    }
}

// One colour phase (or the cost refresh alone, mc.cost_only) of one or both
// directions for all pairs of the launch.
template <int NCH, int PC, int SP = 0>
__global__ void __launch_bounds__(32 * (PR_PROD + pr_cons(NCH, PC)), 1)
k_pm_r(const __grid_constant__ LvlBatch B, const MatchConst mc, const __grid_constant__ RowSched S,
       const __grid_constant__ RowMaps TM, const int buf_words, const int nbuf,
       const long long limit) {
    extern __shared__ __align__(128) uint32_t sm[];
    __shared__ RowRec s_rec[PR_NBUF][PR_NACT];
    __shared__ RowHdr s_hdr[PR_NBUF];
    __shared__ RowGeom s_geom[2];
    __shared__ __align__(8) unsigned long long s_full[PR_NBUF], s_empty[PR_NBUF];
    __shared__ int s_next[PR_NBUF];
    __shared__ int s_abort;
    pdl_trigger();                  // the next phase may start its prologue
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned a_sm = (unsigned)__cvta_generic_to_shared(sm);
    const unsigned full0 = (unsigned)__cvta_generic_to_shared(&s_full[0]);
    const unsigned empty0 = (unsigned)__cvta_generic_to_shared(&s_empty[0]);
    if (threadIdx.x < 2)
        s_geom[threadIdx.x] = rg_geom(NCH, B.d[0][threadIdx.x].P, mc.sigma, mc.rs_W, mc.slack,
                                      mc.tile_w);
    if (threadIdx.x == 0) {
        for (int b = 0; b < nbuf; ++b) {
            mbar_init(full0 + 8u * b, 1);
            mbar_init(empty0 + 8u * b, pr_cons(NCH, PC));
        }
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    pdl_wait();                     // the previous phase is complete and visible
    volatile int* abort = &s_abort;
    if (warp >= pr_cons(NCH, PC))
        pr_produce<NCH, false, PR_PROD, PR_NBUF>(B, mc, S, TM, buf_words, nbuf, a_sm, s_rec, s_hdr, s_next, s_geom, full0,
                        empty0, abort, limit, warp - pr_cons(NCH, PC), lane);
    else
        pr_consume<NCH, PC, SP>(B, mc, S, buf_words, nbuf, a_sm, sm, s_rec, s_hdr, s_next, s_geom,
                            full0, empty0, abort, limit, lane);
}

// ------------------------------------------------------------------
// Bit-plane search (direction descriptor, Sec. III-F: every value a sign in
// {-1, 0, +1}).  With a nonzero plane nz and a sign plane s, a channel pair
// (a, b) gives (a - b)^2 = 1 when exactly one is zero and 4 when both are
// nonzero with opposite signs, else 0 (|a - b| = 1, 2 for the L1 cost), so a
// 32-bit word of 32 values costs popc(nzA ^ nzB) + 4 popc(nzA & nzB & (sA ^ sB)).
// A warp scores one seed at a time, two candidates per step: lane r of
// half-warp h works on patch row r of candidate h (rows past P count zero);
// it keeps the row's reference bits in registers (NR words per plane) and
// reads the candidate row as NW staged words per plane, aligned by funnel
// shifts.  The cost of a candidate is the half-warp sum; costs fit 32 bits.
template <int NCH, int PC>
__device__ void pr_consume_bits(const LvlBatch& B, const MatchConst& mc, const RowSched& S,
                                int buf_words, int nbuf, unsigned a_sm, RowRec (*rec)[PR_NACT],
                                const RowHdr* hdr, int* next, const RowGeom* geom, unsigned full0,
                                unsigned empty0, volatile int* abort, long long limit, int lane) {
    constexpr int NR = NCH == 6 ? 3 : 1;          // aligned words per row and plane
    constexpr int NW = NR + 1;                    // staged words read per row and plane
    constexpr unsigned INF32 = 0xffffffffu;
    const int hf = lane >> 4, r = lane & 15;
    const unsigned fac = mc.norm == PGM_L2SQ ? 2u : 1u;      // 4 = 1 << 2, 2 = 1 << 1
    for (int n = 0;; ++n) {
        const int t = blockIdx.x + n * gridDim.x;
        if (t >= S.total) break;
        const int b = n % nbuf;
        if (!__all_sync(FULL, mbar_wait(full0 + 8u * b, (unsigned)(n / nbuf) & 1u, limit, abort))) {
            if (lane == 0 && !*abort) {
                for (int k = 0; k < B.n; ++k) atomicOr(B.err[k], (unsigned)PGM_ERR_TIMEOUT);
                *abort = 1;
            }
            break;
        }
        const RowHdr H = hdr[b];
        const RowGeom& G = geom[H.dir];
        const DirLvl& D = B.d[H.pair][H.dir];
        const int P = PC > 0 ? PC : G.P, h = P / 2;
        const bool live = r < P;
        const int rr = live ? r : 0;
        unsigned msk[NR];                             // the row's bits in each aligned word
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            const int nb = P * NCH - 32 * k;
            msk[k] = !live || nb <= 0 ? 0u : nb >= 32 ? 0xffffffffu : (1u << nb) - 1u;
        }
        const unsigned buf = a_sm + 4u * (unsigned)(b * buf_words);
        const unsigned a_rn = buf, a_rs = buf + 4u * (unsigned)G.off_rs;
        const unsigned a_wn = buf + 4u * (unsigned)G.off_win, a_ws = buf + 4u * (unsigned)G.off_ws;
        const int tplane = D.tbit_row * (D.th + 2 * BORD);   // words from the nonzero to the sign plane
        unsigned n_eval = 0, n_cost = 0, n_glob = 0;
        for (;;) {
            int a = 0;
            if (lane == 0) a = atomicAdd(next + b, 1);
            a = __shfl_sync(FULL, a, 0);
            if (a >= PR_NACT) break;
            const RowRec R = rec[b][a];
            const int s = R.s;
            if (s < 0) continue;
            const int Rf = R.f, Ru = R.u;
            bool have = Rf & F_VALID;
            if (!have && R.nb0 == NO_CAND && R.nb1 == NO_CAND) {
                if (lane == 0 && Rf != R.f0) D.flags[s] = (uint8_t)Rf;
                continue;
            }
            const int px = R.px, py = R.py;
            // the reference bits of patch row rr
            unsigned an[NR], as[NR];
            {
                const int bit = H.shr + (px - h - H.rx0) * NCH, w = bit >> 5, sh = bit & 31;
                const unsigned rown = a_rn + 4u * (unsigned)((py - h - H.ry0 + rr) * G.bwr + w);
                const unsigned rows = a_rs + 4u * (unsigned)((py - h - H.ry0 + rr) * G.bwr + w);
                unsigned vn[NW], vs[NW];
#pragma unroll
                for (int k = 0; k < NW; ++k) {
                    vn[k] = (unsigned)lds32(rown + 4u * k);
                    vs[k] = (unsigned)lds32(rows + 4u * k);
                }
#pragma unroll
                for (int k = 0; k < NR; ++k) {
                    an[k] = __funnelshift_r(vn[k], vn[k + 1], sh) & msk[k];
                    as[k] = __funnelshift_r(vs[k], vs[k + 1], sh);
                }
            }
            // cost of this half-warp's candidate (window slot y0 << 16 | x0,
            // or -1: from the padded bit-planes in global memory); INF32 when
            // !valid (the lanes then read the window origin)
            auto eval = [&](bool valid, int slot, int qx, int qy) -> unsigned {
                if (!valid) { slot = H.use_win ? 0 : -1; qx = 0; qy = 0; }
                unsigned vn[NW], vs[NW];
                int sh;
                if (slot >= 0) {
                    const int bit = H.shw + (slot & 0xffff) * NCH, w = bit >> 5;
                    sh = bit & 31;
                    const unsigned o = 4u * (unsigned)(((slot >> 16) + rr) * G.bww + w);
#pragma unroll
                    for (int k = 0; k < NW; ++k) {
                        vn[k] = (unsigned)lds32(a_wn + o + 4u * k);
                        vs[k] = (unsigned)lds32(a_ws + o + 4u * k);
                    }
                } else {
                    const int bit = (qx - h + BORD) * NCH, w = bit >> 5;
                    sh = bit & 31;
                    const uint32_t* rowp = D.tgt_bits + (size_t)(qy - h + rr + BORD) * D.tbit_row + w;
#pragma unroll
                    for (int k = 0; k < NW; ++k) {
                        vn[k] = __ldg(rowp + k);
                        vs[k] = __ldg(rowp + tplane + k);
                    }
                }
                unsigned c = 0;
#pragma unroll
                for (int k = 0; k < NR; ++k) {
                    const unsigned tn = __funnelshift_r(vn[k], vn[k + 1], sh);
                    const unsigned ts = __funnelshift_r(vs[k], vs[k + 1], sh);
                    c += (unsigned)__popc((an[k] ^ tn) & msk[k]) +
                         ((unsigned)__popc(an[k] & tn & (as[k] ^ ts)) << fac);
                }
#pragma unroll
                for (int o = 8; o > 0; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
                const unsigned gl = __ballot_sync(FULL, valid && slot < 0);
                if (lane == 0) n_glob += __popc(gl & 0x00010001u);
                return valid ? c : INF32;
            };
            unsigned bc = have ? (unsigned)R.cost : INF32;   // R.cost is INF when refreshing
            if (mc.refresh) bc = INF32;
            int32_t bu = Ru;
            // stage 1 in order: the current match (refresh), the propagated ones
            unsigned pm = ((mc.refresh && have) ? 1u : 0u) | (R.nb0 != NO_CAND ? 2u : 0u) |
                          (R.nb1 != NO_CAND ? 4u : 0u);
            while (pm) {
                const int iA = __ffs(pm) - 1;
                pm &= pm - 1;
                const int iB = pm ? __ffs(pm) - 1 : -1;
                if (pm) pm &= pm - 1;
                const int me = hf ? iB : iA;
                const int cu = me == 0 ? Ru : me == 1 ? R.nb0 : R.nb1;
                const int sl = me == 0 ? R.wu : me == 1 ? R.w0 : R.w1;
                const unsigned c = eval(me >= 0, sl, px + lo16((uint32_t)cu), py + hi16((uint32_t)cu));
                const unsigned co = __shfl_xor_sync(FULL, c, 16);
                const unsigned cA = hf ? co : c, cB = hf ? c : co;
                const int uA = iA == 0 ? Ru : iA == 1 ? R.nb0 : R.nb1;
                const int uB = iB == 1 ? R.nb0 : R.nb1;
                if (iA == 0) ++n_cost; else ++n_eval;
                if (cA < bc) { bc = cA; bu = uA; have = true; }
                if (iB >= 0) {
                    ++n_eval;
                    if (cB < bc) { bc = cB; bu = uB; have = true; }
                }
            }
            // stage 2: the limited random search (Eq. 5) around the match held
            // after propagation, offsets k0 and k0 + 1 per step
            const int K = R.K;
            if (have && K > 0) {
                const int ux0 = lo16((uint32_t)bu), uy0 = hi16((uint32_t)bu);
                const bool atu = bu == Ru && (Rf & F_VALID);      // slots from the producer
                for (int k0 = 0; k0 < K; k0 += 2) {
                    const int k = k0 + hf;
                    int dx = 0, dy = 0;
                    if (k < 2) {
                        const uint32_t o = (uint32_t)(k ? R.r1 : R.r0);
                        dx = lo16(o);
                        dy = hi16(o);
                    } else if (k < K) {
                        const uint4 rq = philox(
                            make_uint4((uint32_t)s,
                                       ((uint32_t)B.visit << 16) | ((uint32_t)H.dir << 15) | (uint32_t)mc.t,
                                       ((uint32_t)B.level << 16) | (uint32_t)(k >> 1),
                                       B.stream_id[H.pair]),
                            mc.key0, mc.key1);
                        dx = rs_off((k & 1) ? rq.z : rq.x, k, mc.rs_W, mc.rs_mode);
                        dy = rs_off((k & 1) ? rq.w : rq.y, k, mc.rs_W, mc.rs_mode);
                    }
                    const int qx = px + ux0 + dx, qy = py + uy0 + dy;   // tested before packing
                    int sl;
                    bool valid;
                    if (atu && k < 2) {
                        const int w = k ? R.wr1 : R.wr0;
                        valid = w != -2;
                        sl = valid ? w : 0;
                    } else {
                        valid = k < K && !(dx == 0 && dy == 0) && inside(D, qx, qy);
                        sl = valid ? pr_slot<true>(G, H, P, qx, qy) : 0;
                    }
                    const unsigned c = eval(valid, sl, qx, qy);
                    const unsigned co = __shfl_xor_sync(FULL, c, 16);
                    const unsigned vb = __ballot_sync(FULL, valid);
                    const unsigned cA = hf ? co : c, cB = hf ? c : co;
                    const int dxA = __shfl_sync(FULL, dx, 0), dyA = __shfl_sync(FULL, dy, 0);
                    const int dxB = __shfl_sync(FULL, dx, 16), dyB = __shfl_sync(FULL, dy, 16);
                    if (vb & 1u) {
                        ++n_eval;
                        if (cA < bc) { bc = cA; bu = pack_u(ux0 + dxA, uy0 + dyA); }
                    }
                    if (vb & 0x10000u) {
                        ++n_eval;
                        if (cB < bc) { bc = cB; bu = pack_u(ux0 + dxB, uy0 + dyB); }
                    }
                }
            }
            if (lane == 0) {
                if (have && (mc.refresh || bu != Ru || !(Rf & F_VALID))) {
                    D.u[s] = bu;
                    D.cost[s] = (unsigned long long)bc;
                    D.flags[s] = (uint8_t)(Rf | F_VALID);
                } else if (!have && Rf != R.f0) {
                    D.flags[s] = (uint8_t)Rf;
                }
            }
        }
        if (lane == 0) {
            if (n_eval) atomicAdd(B.evals[H.pair] + H.dir, (unsigned long long)n_eval);
            if (n_cost) atomicAdd(B.evals[H.pair] + 2 + H.dir, (unsigned long long)n_cost);
            if (n_glob) atomicAdd(B.evals[H.pair] + 6 + H.dir, (unsigned long long)n_glob);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(empty0 + 8u * b);
    }
}

// the bit-plane kernel: its buffers are small, so more producer warps keep a
// deeper ring of staged tiles
constexpr int PB_PROD = 4, PB_CONS = 20, PB_NBUF = 8;

template <int NCH, int PC>
__global__ void __launch_bounds__(32 * (PB_PROD + PB_CONS), 1)
k_pm_b(const __grid_constant__ LvlBatch B, const MatchConst mc, const __grid_constant__ RowSched S,
       const __grid_constant__ RowMaps TM, const int buf_words, const int nbuf,
       const long long limit) {
    extern __shared__ __align__(128) uint32_t sm[];
    __shared__ RowRec s_rec[PB_NBUF][PR_NACT];
    __shared__ RowHdr s_hdr[PB_NBUF];
    __shared__ RowGeom s_geom[2];
    __shared__ __align__(8) unsigned long long s_full[PB_NBUF], s_empty[PB_NBUF];
    __shared__ int s_next[PB_NBUF];
    __shared__ int s_abort;
    pdl_trigger();                  // the next phase may start its prologue
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned a_sm = (unsigned)__cvta_generic_to_shared(sm);
    const unsigned full0 = (unsigned)__cvta_generic_to_shared(&s_full[0]);
    const unsigned empty0 = (unsigned)__cvta_generic_to_shared(&s_empty[0]);
    if (threadIdx.x < 2)
        s_geom[threadIdx.x] = rg_geom_bits(NCH, B.d[0][threadIdx.x].P, mc.sigma, mc.rs_W, mc.slack,
                                           mc.tile_w);
    if (threadIdx.x == 0) {
        for (int b = 0; b < nbuf; ++b) {
            mbar_init(full0 + 8u * b, 1);
            mbar_init(empty0 + 8u * b, PB_CONS);
        }
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    pdl_wait();                     // the previous phase is complete and visible
    volatile int* abort = &s_abort;
    if (warp >= PB_CONS)
        pr_produce<NCH, true, PB_PROD, PB_NBUF>(B, mc, S, TM, buf_words, nbuf, a_sm, s_rec, s_hdr,
                                                s_next, s_geom, full0, empty0, abort, limit,
                                                warp - PB_CONS, lane);
    else
        pr_consume_bits<NCH, PC>(B, mc, S, buf_words, nbuf, a_sm, s_rec, s_hdr, s_next, s_geom,
                                 full0, empty0, abort, limit, lane);
}

}  // namespace

// ===========================================================================
// ------------------------------------------------------------------
// Bit-plane search, one seed per lane.  A popcount cost is so cheap that a
// warp cooperating on one seed spends most of its instructions on the seed's
// bookkeeping; here a consumer warp takes a whole staged tile and every lane
// one of its 32 seeds, so that bookkeeping is paid once per lane instead of
// once per warp.  A lane first scores, row by row with its reference row
// loaded once, every candidate known when the tile was staged: the current
// match (cost refresh), the two propagated matches and the first two search
// candidates around the current match; then it takes the decisions in the
// paper's order.  Where a propagated match moved the search centre (or the
// search has more than two candidates) the remaining search candidates are
// scored afterwards, one per round, in order.  Results and evaluation counts
// are those of the sequential order.
constexpr int PS_PROD = 4, PS_CONS = 12, PS_NBUF = 16;
constexpr int PS_NC = 5;                      // candidates scored in the first round

// Cost rows [0, P) of NC candidates against the lane's reference patch.
// ok[j]: candidate j is scored; slot[j]: window corner (y0 << 16 | x0) or -1
// (read from the padded bit-planes in global memory, centre qx[j], qy[j]).
template <int NCH, int NC>
__device__ __forceinline__ void ps_rows(const RowGeom& G, const RowHdr& H, const DirLvl& D, int P,
                                        unsigned a_rn, unsigned a_rs, unsigned a_wn, unsigned a_ws,
                                        int rbit, int rrow, const bool (&ok)[NC],
                                        const int (&slot)[NC], const int (&qx)[NC],
                                        const int (&qy)[NC], unsigned fac, unsigned (&c)[NC],
                                        uint32_t* errp) {
    constexpr int NR = NCH == 6 ? 3 : 1, NW = NR + 1;
    const int h = P / 2;
    const int tplane = D.tbit_row * (D.th + 2 * BORD);
    unsigned msk[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        const int nb = P * NCH - 32 * k;
        msk[k] = nb <= 0 ? 0u : nb >= 32 ? 0xffffffffu : (1u << nb) - 1u;
    }
    // per candidate: the first word of its row 0 and the bit shift
    unsigned base[NC];
    const uint32_t* gp[NC];
    int sh[NC];
    bool sm_[NC], rd[NC];
    const bool rok = PGM_CHECK(rrow >= 0 && rrow + P <= G.ref_h && rbit >= 0 &&
                               (rbit >> 5) + NW <= G.bwr, errp);
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        c[j] = 0;
        rd[j] = ok[j] && rok;
        sm_[j] = ok[j] && slot[j] >= 0;
        base[j] = 0;
        gp[j] = D.tgt_bits;
        sh[j] = 0;
        if (sm_[j]) {
            const int bit = H.shw + (slot[j] & 0xffff) * NCH;
            sh[j] = bit & 31;
            base[j] = 4u * (unsigned)((slot[j] >> 16) * G.bww + (bit >> 5));
            rd[j] = rd[j] && PGM_CHECK((slot[j] >> 16) + P <= G.win_h && (bit >> 5) + NW <= G.bww,
                                       errp);
        } else if (ok[j]) {
            rd[j] = rd[j] && PGM_CHECK(qx[j] >= 0 && qy[j] >= 0 && qx[j] < D.tw && qy[j] < D.th &&
                                       h <= BORD, errp);
            const int bit = (qx[j] - h + BORD) * NCH;
            sh[j] = bit & 31;
            gp[j] = D.tgt_bits + (size_t)(qy[j] - h + BORD) * D.tbit_row + (bit >> 5);
        }
    }
    const int rsh = rbit & 31;
    unsigned rb = 4u * (unsigned)(rrow * G.bwr + (rbit >> 5));
    for (int r = 0; r < P; ++r) {
        unsigned an[NR], as[NR];
        {
            unsigned vn[NW], vs[NW];
#pragma unroll
            for (int k = 0; k < NW; ++k) {
                vn[k] = (unsigned)lds32(a_rn + rb + 4u * k);
                vs[k] = (unsigned)lds32(a_rs + rb + 4u * k);
            }
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                an[k] = __funnelshift_r(vn[k], vn[k + 1], rsh) & msk[k];
                as[k] = __funnelshift_r(vs[k], vs[k + 1], rsh);
            }
        }
        rb += 4u * (unsigned)G.bwr;
#pragma unroll
        for (int j = 0; j < NC; ++j) {
            if (!rd[j]) continue;
            unsigned vn[NW], vs[NW];
            if (sm_[j]) {
#pragma unroll
                for (int k = 0; k < NW; ++k) {
                    vn[k] = (unsigned)lds32(a_wn + base[j] + 4u * k);
                    vs[k] = (unsigned)lds32(a_ws + base[j] + 4u * k);
                }
                base[j] += 4u * (unsigned)G.bww;
            } else {
#pragma unroll
                for (int k = 0; k < NW; ++k) {
                    vn[k] = __ldg(gp[j] + k);
                    vs[k] = __ldg(gp[j] + tplane + k);
                }
                gp[j] += D.tbit_row;
            }
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                const unsigned tn = __funnelshift_r(vn[k], vn[k + 1], sh[j]);
                const unsigned ts = __funnelshift_r(vs[k], vs[k + 1], sh[j]);
                c[j] += (unsigned)__popc((an[k] ^ tn) & msk[k]) +
                        ((unsigned)__popc(an[k] & tn & (as[k] ^ ts)) << fac);
            }
        }
    }
}

template <int NCH, int PC>
__device__ void ps_consume(const LvlBatch& B, const MatchConst& mc, const RowSched& S, int buf_words,
                           int nbuf, unsigned a_sm, RowRec (*rec)[PR_NACT], const RowHdr* hdr,
                           const RowGeom* geom, unsigned full0, unsigned empty0,
                           volatile int* abort, long long limit, int cw, int lane) {
    constexpr unsigned INF32 = 0xffffffffu;
    const unsigned fac = mc.norm == PGM_L2SQ ? 2u : 1u;      // 4 = 1 << 2, 2 = 1 << 1
    int seen[PS_NBUF];                    // waits so far on this warp's full barrier of each buffer
#pragma unroll
    for (int b = 0; b < PS_NBUF; ++b) seen[b] = 0;
    for (int n = cw;; n += PS_CONS) {
        const int t = blockIdx.x + n * gridDim.x;
        if (t >= S.total) break;
        const int b = n % nbuf;
        const unsigned fb = full0 + 8u * (unsigned)(b * PS_CONS + cw);
        if (!__all_sync(FULL, mbar_wait(fb, (unsigned)(seen[b]++) & 1u, limit, abort))) {
            if (lane == 0 && !*abort) {
                for (int k = 0; k < B.n; ++k) atomicOr(B.err[k], (unsigned)PGM_ERR_TIMEOUT);
                *abort = 1;
            }
            break;
        }
        const RowHdr H = hdr[b];
        const RowGeom& G = geom[H.dir];
        const DirLvl& D = B.d[H.pair][H.dir];
        const int P = PC > 0 ? PC : G.P, h = P / 2;
        const unsigned buf = a_sm + 4u * (unsigned)(b * buf_words);
        const unsigned a_rn = buf, a_rs = buf + 4u * (unsigned)G.off_rs;
        const unsigned a_wn = buf + 4u * (unsigned)G.off_win, a_ws = buf + 4u * (unsigned)G.off_ws;
        const RowRec R = rec[b][lane];
        const int s = R.s, Rf = R.f, Ru = R.u, px = R.px, py = R.py;
        bool have = s >= 0 && (Rf & F_VALID);
        const bool idle = s < 0 || (!have && R.nb0 == NO_CAND && R.nb1 == NO_CAND);
        // round 1: the candidates known at staging time
        bool ok[PS_NC];
        int slot[PS_NC], qx[PS_NC], qy[PS_NC];
        ok[0] = !idle && mc.refresh && have;
        slot[0] = R.wu;
        qx[0] = px + lo16((uint32_t)Ru); qy[0] = py + hi16((uint32_t)Ru);
        ok[1] = !idle && R.nb0 != NO_CAND;
        slot[1] = R.w0;
        qx[1] = px + lo16((uint32_t)R.nb0); qy[1] = py + hi16((uint32_t)R.nb0);
        ok[2] = !idle && R.nb1 != NO_CAND;
        slot[2] = R.w1;
        qx[2] = px + lo16((uint32_t)R.nb1); qy[2] = py + hi16((uint32_t)R.nb1);
        ok[3] = !idle && R.wr0 != -2;
        slot[3] = R.wr0;
        qx[3] = qx[0] + lo16((uint32_t)R.r0); qy[3] = qy[0] + hi16((uint32_t)R.r0);
        ok[4] = !idle && R.wr1 != -2;
        slot[4] = R.wr1;
        qx[4] = qx[0] + lo16((uint32_t)R.r1); qy[4] = qy[0] + hi16((uint32_t)R.r1);
        // a lane without a seed (a tile at the lattice edge) still walks the
        // rows with its warp: its reference position is the region's corner
        const int rbit = idle ? 0 : H.shr + (px - h - H.rx0) * NCH;
        const int rrow = idle ? 0 : py - h - H.ry0;
        unsigned c[PS_NC];
        ps_rows<NCH, PS_NC>(G, H, D, P, a_rn, a_rs, a_wn, a_ws, rbit, rrow, ok, slot, qx, qy, fac, c,
                            B.err[H.pair]);
        unsigned n_eval = 0, n_cost = 0, n_glob = 0;
        // the decisions in the paper's order
        unsigned bc = have && !mc.refresh ? (unsigned)R.cost : INF32;
        int32_t bu = Ru;
        if (ok[0]) { bc = c[0]; ++n_cost; n_glob += slot[0] < 0; }
        if (ok[1]) {
            ++n_eval; n_glob += slot[1] < 0;
            if (c[1] < bc) { bc = c[1]; bu = R.nb0; have = true; }
        }
        if (ok[2]) {
            ++n_eval; n_glob += slot[2] < 0;
            if (c[2] < bc) { bc = c[2]; bu = R.nb1; have = true; }
        }
        const int K = idle ? 0 : R.K;
        int k2 = K;                   // the first search candidate of round 2
        const int cx0 = lo16((uint32_t)bu), cy0 = hi16((uint32_t)bu);
        if (have && K > 0) {
            if (bu == Ru && (Rf & F_VALID)) {        // centre = current match: round 1 scored them
#pragma unroll
                for (int j = 3; j < 5; ++j) {
                    if (!ok[j]) continue;
                    ++n_eval; n_glob += slot[j] < 0;
                    if (c[j] < bc) {
                        bc = c[j];
                        bu = pack_u(qx[j] - px, qy[j] - py);
                    }
                }
                k2 = 2;
            } else {
                k2 = 0;
            }
        }
        // round 2: the rest of the limited random search, one candidate per step
        const int rbit2 = rbit, rrow2 = rrow;
        for (int k = k2;; ++k) {
            const bool live = have && k < K;
            if (!__any_sync(FULL, live)) break;
            bool ok2[1] = {false};
            int sl2[1] = {-1}, qx2[1] = {0}, qy2[1] = {0};
            int dx = 0, dy = 0;
            if (live) {
                if (k < 2) {
                    const uint32_t o = (uint32_t)(k ? R.r1 : R.r0);
                    dx = lo16(o);
                    dy = hi16(o);
                } else {
                    const uint4 rq = philox(
                        make_uint4((uint32_t)s,
                                   ((uint32_t)B.visit << 16) | ((uint32_t)H.dir << 15) | (uint32_t)mc.t,
                                   ((uint32_t)B.level << 16) | (uint32_t)(k >> 1),
                                   B.stream_id[H.pair]),
                        mc.key0, mc.key1);
                    dx = rs_off((k & 1) ? rq.z : rq.x, k, mc.rs_W, mc.rs_mode);
                    dy = rs_off((k & 1) ? rq.w : rq.y, k, mc.rs_W, mc.rs_mode);
                }
                qx2[0] = px + cx0 + dx;
                qy2[0] = py + cy0 + dy;
                ok2[0] = !(dx == 0 && dy == 0) && inside(D, qx2[0], qy2[0]);
                if (ok2[0]) sl2[0] = pr_slot<true>(G, H, P, qx2[0], qy2[0]);
            }
            unsigned c2[1];
            ps_rows<NCH, 1>(G, H, D, P, a_rn, a_rs, a_wn, a_ws, rbit2, rrow2, ok2, sl2, qx2, qy2, fac, c2,
                            B.err[H.pair]);
            if (ok2[0]) {
                ++n_eval; n_glob += sl2[0] < 0;
                if (c2[0] < bc) { bc = c2[0]; bu = pack_u(cx0 + dx, cy0 + dy); }
            }
        }
        if (!idle) {
            if (have && (mc.refresh || bu != Ru || !(Rf & F_VALID))) {
                D.u[s] = bu;
                D.cost[s] = (unsigned long long)bc;
                D.flags[s] = (uint8_t)(Rf | F_VALID);
            } else if (!have && Rf != R.f0) {
                D.flags[s] = (uint8_t)Rf;
            }
        } else if (s >= 0 && Rf != R.f0) {
            D.flags[s] = (uint8_t)Rf;                 // the refresh dropped it
        }
        n_eval = __reduce_add_sync(FULL, n_eval);
        n_cost = __reduce_add_sync(FULL, n_cost);
        n_glob = __reduce_add_sync(FULL, n_glob);
        if (lane == 0) {
            if (n_eval) atomicAdd(B.evals[H.pair] + H.dir, (unsigned long long)n_eval);
            if (n_cost) atomicAdd(B.evals[H.pair] + 2 + H.dir, (unsigned long long)n_cost);
            if (n_glob) atomicAdd(B.evals[H.pair] + 6 + H.dir, (unsigned long long)n_glob);
        }
        __syncwarp();
        if (lane == 0)                                         // the tile's buffer is free again
            mbar_arrive(empty0 + 8u * (unsigned)(b * PS_PROD + (n + nbuf) % PS_PROD));
    }
}

template <int NCH, int PC>
__global__ void __launch_bounds__(32 * (PS_PROD + PS_CONS), 1)
k_pm_s(const __grid_constant__ LvlBatch B, const MatchConst mc, const __grid_constant__ RowSched S,
       const __grid_constant__ RowMaps TM, const int buf_words, const int nbuf,
       const long long limit) {
    extern __shared__ __align__(128) uint32_t sm[];
    __shared__ RowRec s_rec[PS_NBUF][PR_NACT];
    __shared__ RowHdr s_hdr[PS_NBUF];
    __shared__ RowGeom s_geom[2];
    __shared__ __align__(8) unsigned long long s_full[PS_NBUF * PS_CONS], s_empty[PS_NBUF * PS_PROD];
    __shared__ int s_next[PS_NBUF];
    __shared__ int s_abort;
    pdl_trigger();                  // the next phase may start its prologue
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned a_sm = (unsigned)__cvta_generic_to_shared(sm);
    const unsigned full0 = (unsigned)__cvta_generic_to_shared(&s_full[0]);
    const unsigned empty0 = (unsigned)__cvta_generic_to_shared(&s_empty[0]);
    if (threadIdx.x < 2)
        s_geom[threadIdx.x] = rg_geom_bits(NCH, B.d[0][threadIdx.x].P, mc.sigma, mc.rs_W, mc.slack,
                                           mc.tile_w);
    if (threadIdx.x == 0) {
        for (int b = 0; b < nbuf; ++b) {                 // per consumer and per producer
            for (int g = 0; g < PS_CONS; ++g) mbar_init(full0 + 8u * (b * PS_CONS + g), 1);
            for (int q = 0; q < PS_PROD; ++q) mbar_init(empty0 + 8u * (b * PS_PROD + q), 1);
        }
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    pdl_wait();                     // the previous phase is complete and visible
    volatile int* abort = &s_abort;
    if (warp >= PS_CONS)
        pr_produce<NCH, true, PS_PROD, PS_NBUF, PS_CONS>(B, mc, S, TM, buf_words, nbuf, a_sm, s_rec, s_hdr,
                                                s_next, s_geom, full0, empty0, abort, limit,
                                                warp - PS_CONS, lane);
    else
        ps_consume<NCH, PC>(B, mc, S, buf_words, nbuf, a_sm, s_rec, s_hdr, s_geom, full0, empty0,
                            abort, limit, warp, lane);
}

// Host side: launch configuration.  No device code below this line.

// The kernel's parameters (batch, constants, schedule, tensor maps, scalars)
// must fit the 32764-byte kernel parameter limit.
static_assert(sizeof(LvlBatch) + sizeof(MatchConst) + sizeof(RowSched) + sizeof(RowMaps) +
                  2 * sizeof(int) + sizeof(long long) + 256 <= 32764,
              "k_pm_r parameters exceed the kernel parameter limit");

static int device_sms() {
    static thread_local int dev_cached = -1, sms = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (dev != dev_cached) {
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
        dev_cached = dev;
    }
    return sms;
}

// ---------------------------------------------------------------- tensor maps
// cuTensorMapEncodeTiled from the driver (no link against it), and a cache of
// encoded maps keyed by their arguments: the maps of a level serve all of its
// phases, and repeated steps on the same buffers encode nothing.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

struct MapKey {
    const void* ptr;
    unsigned long long dim0, dim1, pitch;
    unsigned box0, box1, esize, pad;
    bool operator==(const MapKey& o) const {
        return ptr == o.ptr && dim0 == o.dim0 && dim1 == o.dim1 && pitch == o.pitch &&
               box0 == o.box0 && box1 == o.box1 && esize == o.esize;
    }
};
struct MapEntry { MapKey key; CUtensorMap map; bool used; };
constexpr int MAP_CACHE = 1024;
static std::mutex map_mu;
static MapEntry map_cache[MAP_CACHE];

// A 2D map of `esize`-byte elements (4 or 8): dim0 x dim1 elements, rows
// `pitch` bytes apart, box0 x box1 elements per copy, zero fill outside (a
// box may be larger than the array).  False when the arguments break a
// tensor-map rule (then the batch goes to the per-seed kernels).
static bool map2d(CUtensorMap* out, const void* ptr, unsigned long long dim0,
                  unsigned long long dim1, unsigned long long pitch, unsigned box0, unsigned box1,
                  unsigned esize) {
    if (box0 == 0 || box1 == 0 || box0 > 256 || box1 > 256 || (box0 * esize) % 16 != 0 ||
        pitch % 16 != 0 || ((uintptr_t)ptr & 15) != 0 || pitch < dim0 * esize)
        return false;
    const EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const MapKey key{ptr, dim0, dim1, pitch, box0, box1, esize, 0};
    size_t h = (uintptr_t)ptr;
    h = h * 1000003u ^ (size_t)dim0;
    h = h * 1000003u ^ (size_t)dim1;
    h = h * 1000003u ^ (size_t)pitch;
    h = h * 1000003u ^ (size_t)(box0 | (box1 << 9) | (esize << 18));
    std::lock_guard<std::mutex> lock(map_mu);
    MapEntry& e = map_cache[(h >> 4) % MAP_CACHE];
    if (e.used && e.key == key) {
        *out = e.map;
        return true;
    }
    const cuuint64_t gdim[2] = {dim0, dim1}, gstride[1] = {pitch};
    const cuuint32_t box[2] = {box0, box1}, estride[2] = {1, 1};
    if (fn(out, esize == 8 ? CU_TENSOR_MAP_DATA_TYPE_UINT64 : CU_TENSOR_MAP_DATA_TYPE_UINT32, 2,
           const_cast<void*>(ptr), gdim, gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    e.key = key;
    e.map = *out;
    e.used = true;
    return true;
}

// The three maps of one direction of one pair: the padded reference split
// words and target descriptor (16-byte colour pixels as two 8-byte elements,
// gray pixels as one 4-byte element), and the target sums.
static bool dir_maps(const DirLvl& D, int nch, const RowGeom& g, CUtensorMap* m) {
    const int pxw = px_words(nch);
    const unsigned long long rp = 2ull * D.ref_pitch, tp = 2ull * D.tgt_pitch;
    const uint8_t* rbase = reinterpret_cast<const uint8_t*>(D.ref_split) -
                           (size_t)BORD * rp - (size_t)BORD * 4 * pxw;
    const uint8_t* tbase = reinterpret_cast<const uint8_t*>(D.tgt) -
                           (size_t)BORD * tp - (size_t)BORD * 4 * pxw;
    const unsigned long long rw = (unsigned long long)(D.rw + 2 * BORD), tw = (unsigned long long)(D.tw + 2 * BORD);
    if (pxw == 4)
        return map2d(&m[0], rbase, 2 * rw, D.rh + 2 * BORD, rp, g.sp / 2, g.ref_h, 8) &&
               map2d(&m[1], tbase, 2 * tw, D.th + 2 * BORD, tp, g.sp / 2, g.win_h, 8) &&
               map2d(&m[2], D.sb2, D.sbp, D.th, 8ull * D.sbp, g.cwp, g.ch, 8);
    return map2d(&m[0], rbase, rw, D.rh + 2 * BORD, rp, g.sp, g.ref_h, 4) &&
           map2d(&m[1], tbase, tw, D.th + 2 * BORD, tp, g.sp, g.win_h, 4) &&
           map2d(&m[2], D.sb2, D.sbp, D.th, 8ull * D.sbp, g.cwp, g.ch, 8);
}

// The two maps of the bit-plane form: the reference and the target planes,
// each one array of 2 (H + 2 BORD) rows (nonzero rows, then sign rows).
static bool dir_maps_bits(const DirLvl& D, const RowGeom& g, CUtensorMap* m) {
    if (!D.ref_bits || !D.tgt_bits || D.rbit_row <= 0 || D.tbit_row <= 0) return false;
    return map2d(&m[0], D.ref_bits, D.rbit_row, 2ull * (D.rh + 2 * BORD), 4ull * D.rbit_row,
                 g.bwr, g.ref_h, 4) &&
           map2d(&m[1], D.tgt_bits, D.tbit_row, 2ull * (D.th + 2 * BORD), 4ull * D.tbit_row,
                 g.bww, g.win_h, 4);
}

// the search runs on the bit-planes (direction descriptor)
static bool use_bits(const MatchConst& mc) { return mc.descriptor == PGM_DIR; }

// Per-direction schedules S[0], S[1], the schedule of both directions
// together S[2], and the layouts; false when a buffer ring would not fit in
// shared memory, a slot would not fit its 16-bit fields, or a tensor map
// cannot be made (each is encoded here, and cached for the launches).
static bool pr_plan(const LvlBatch& B, const MatchConst& mc, int nch, RowSched* S, RowGeom* G) {
    const bool bits = use_bits(mc);
    if ((!bits && mc.norm != PGM_L2SQ) || B.n > PR_MAPS) return false;
    S[2].nk = 2 * B.n;
    S[2].total = 0;
    S[2].dir = 0;
    S[2].ndir = 2;
    for (int d = 0; d < 2; ++d) {
        S[d].nk = B.n;
        S[d].total = 0;
        S[d].dir = d;
        S[d].ndir = 1;
        G[d] = bits ? rg_geom_bits(nch, B.d[0][d].P, mc.sigma, mc.rs_W, mc.slack, mc.tile_w)
                    : rg_geom(nch, B.d[0][d].P, mc.sigma, mc.rs_W, mc.slack, mc.tile_w);
        if (B.d[0][d].P > MAXP || 2L * G[d].words * 4 > 200L * 1024 ||
            (long)G[d].sp * G[d].win_h >= 65536L || (long)G[d].cwp * G[d].ch >= 32768L)
            return false;
    }
    CUtensorMap m[3];
    for (int k = 0; k < B.n; ++k)
        for (int d = 0; d < 2; ++d) {
            const DirLvl& D = B.d[k][d];
            const int tiles = ((D.nx + G[d].tw - 1) / G[d].tw) * ((D.ny + G[d].th - 1) / G[d].th);
            S[d].cum[k] = S[d].total;
            S[d].total += tiles;
            S[2].cum[2 * k + d] = S[2].total;
            S[2].total += tiles;
            if (D.P != B.d[0][d].P || !(bits ? dir_maps_bits(D, G[d], m) : dir_maps(D, nch, G[d], m)))
                return false;
        }
    S[0].cum[B.n] = S[0].total;
    S[1].cum[B.n] = S[1].total;
    S[2].cum[2 * B.n] = S[2].total;
    return true;
}

// The maps of every slot of schedule S (one thread's launch parameters;
// cache hits after pr_plan).
static RowMaps& pr_maps(const LvlBatch& B, int nch, bool bits, const RowSched& S, const RowGeom* G) {
    static thread_local RowMaps TM;
    for (int k = 0; k < S.nk && k < PR_MAPS; ++k) {
        const int pair = S.ndir == 2 ? k >> 1 : k, dir = S.ndir == 2 ? (k & 1) : S.dir;
        if (bits) dir_maps_bits(B.d[pair][dir], G[dir], TM.m[k]);
        else dir_maps(B.d[pair][dir], nch, G[dir], TM.m[k]);
    }
    return TM;
}

// wait limit of the kernel's mbarrier waits (cycles); set by pgm_set_wait_limit
long long wait_limit();

template <int NCH, int PC, bool BITS = false, int SP = 0>
pgm_status launch_r(const LvlBatch& B, const MatchConst& mc, const RowSched& S, const RowMaps& TM,
                    int buf_words, cudaStream_t st) {
    const int sms = device_sms();
    if (sms <= 0) return cuda_fail("search: SM count", cudaErrorInvalidDevice);
    // bit planes: one seed per lane once every consumer warp of a CTA has
    // tiles of its own, else the warp-per-seed form (coarse levels)
    const bool per_lane = BITS && S.total >= PS_CONS * sms;
    auto kern = k_pm_r<NCH, PC, SP>;
    if constexpr (BITS) kern = per_lane ? k_pm_s<NCH, PC> : k_pm_b<NCH, PC>;
    if (pgm_status r = smem_opt_in((const void*)kern); r != PGM_OK) return r;
    // the ring: as many buffers as fit beside the kernel's static shared
    // memory (the bit-plane kernel's tile records take about 33 KB)
    cudaFuncAttributes fa;
    PGM_TRY(cudaFuncGetAttributes(&fa, (const void*)kern), "search: kernel attributes");
    const int most = BITS ? (per_lane ? PS_NBUF : PB_NBUF) : PR_NBUF;
    const long cap = fa.maxDynamicSharedSizeBytes < 200 * 1024 ? fa.maxDynamicSharedSizeBytes
                                                               : 200L * 1024;
    if (2L * buf_words * 4 > cap) return PGM_ERR_UNSUPPORTED;
    int nbuf = 2;
    while (nbuf < most && (nbuf + 1L) * buf_words * 4 <= cap) ++nbuf;
    const int smem = nbuf * buf_words * 4;
    const int grid = S.total < sms ? S.total : sms;       // one CTA per SM (shared memory)
    const int threads = !BITS ? 32 * (PR_PROD + pr_cons(NCH, PC))
                        : per_lane ? 32 * (PS_PROD + PS_CONS) : 32 * (PB_PROD + PB_CONS);
    PGM_TRY(launch_pdl(kern, dim3(grid), dim3(threads), smem, st, B, mc, S, TM, buf_words, nbuf,
                       wait_limit()),
            "search: launch");
    return launch_status("search: launch");
}

// The consumer specialisation of a direction's patch side: compile-time sides
// for the common 6-channel patches (15, 11) and 2-channel ones (15, 11, 8),
// else the run-time form.
template <int NCH>
pgm_status launch_dir(const LvlBatch& B, const MatchConst& mc, const RowSched& S, const RowGeom& G,
                      const RowMaps& TM, int buf_words, cudaStream_t st) {
    const int P = G.P;
    // fixed-pitch rows: their one-past reads must land in the next region
    if constexpr (NCH == 6)
        if (P == 15 && G.sp == PR_ROWS_SP && G.pxw == 4 && G.off_win >= G.sp * G.ref_h &&
            G.off_sb - G.off_win >= G.sp * G.win_h && G.words - G.off_sb >= G.sp + 4 * (P + 2) &&
            G.sp / 4 >= G.win_w + 2)
            return launch_r<NCH, 15, false, PR_ROWS_SP>(B, mc, S, TM, buf_words, st);
    if (P == 15) return launch_r<NCH, 15>(B, mc, S, TM, buf_words, st);
    if (P == 11) return launch_r<NCH, 11>(B, mc, S, TM, buf_words, st);
    if (NCH == 2 && P == 8) return launch_r<NCH, 8>(B, mc, S, TM, buf_words, st);
    return launch_r<NCH, 0>(B, mc, S, TM, buf_words, st);
}

bool pm_tile_fits(const LvlBatch& B, const MatchConst& mc, int nch) {
    RowSched S[3];
    RowGeom G[2];
    return pr_plan(B, mc, nch, S, G);
}

// Phases larger than one tile per SM run one launch per direction.
bool pm_tile_split(const LvlBatch& B, const MatchConst& mc, int nch) {
    RowSched S[3];
    RowGeom G[2];
    return pr_plan(B, mc, nch, S, G) && (S[2].total > device_sms() || 2 * B.n > PR_MAPS);
}

// *handled = false when pr_plan refuses the batch; the caller then uses the
// per-seed kernels.  A small phase (at most one tile per SM, the coarse
// levels) runs both directions in one launch of the run-time-P consumer; a
// larger one runs each direction in its own launch of the consumer for its
// patch side, the backward one on st2 when given (the two directions are
// independent within a phase).  *nlaunch: kernels launched.
pgm_status launch_pm_tile(const LvlBatch& B, const MatchConst& mc, int nch, int maxP, int* nlaunch,
                          bool* handled, cudaStream_t st, cudaStream_t st2) {
    (void)maxP;
    *handled = false;
    *nlaunch = 0;
    RowSched S[3];
    RowGeom G[2];
    if (!pr_plan(B, mc, nch, S, G)) return PGM_OK;
    *handled = true;
    if (S[2].total == 0) return PGM_OK;
    const bool bits = use_bits(mc);
    if (S[2].total <= device_sms() && 2 * B.n <= PR_MAPS) {
        const int words = G[0].words > G[1].words ? G[0].words : G[1].words;
        *nlaunch = 1;
        RowMaps& TM = pr_maps(B, nch, bits, S[2], G);
        if (bits)
            return nch == 2 ? launch_r<2, 0, true>(B, mc, S[2], TM, words, st)
                            : launch_r<6, 0, true>(B, mc, S[2], TM, words, st);
        return nch == 2 ? launch_r<2, 0>(B, mc, S[2], TM, words, st)
                        : launch_r<6, 0>(B, mc, S[2], TM, words, st);
    }
    for (int d = 0; d < 2; ++d) {
        if (S[d].total == 0) continue;
        RowMaps& TM = pr_maps(B, nch, bits, S[d], G);
        const cudaStream_t sd = d == 1 && st2 ? st2 : st;
        pgm_status r;
        if (bits)          // the bit-plane consumer's inner loops do not depend on P
            r = nch == 2 ? launch_r<2, 0, true>(B, mc, S[d], TM, G[d].words, sd)
                         : launch_r<6, 0, true>(B, mc, S[d], TM, G[d].words, sd);
        else
            r = nch == 2 ? launch_dir<2>(B, mc, S[d], G[d], TM, G[d].words, sd)
                         : launch_dir<6>(B, mc, S[d], G[d], TM, G[d].words, sd);
        if (r != PGM_OK) return r;
        ++*nlaunch;
    }
    return PGM_OK;
}

// The cost refresh of a visit without iterations: the same kernel scoring
// only the current matches.
pgm_status launch_cost_tile(const LvlBatch& B, const MatchConst& mc, int nch, bool* handled,
                            cudaStream_t st) {
    MatchConst m = mc;
    m.cost_only = 1;
    m.refresh = 1;
    m.t = 0;
    m.colour = 0;
    int nl = 0;
    *handled = false;
    // both colours: one launch each
    for (int col = 0; col < 2; ++col) {
        m.colour = col;
        const pgm_status r = launch_pm_tile(B, m, nch, 0, &nl, handled, st, nullptr);
        if (r != PGM_OK || !*handled) return r;
    }
    return PGM_OK;
}

}  // namespace pgm
