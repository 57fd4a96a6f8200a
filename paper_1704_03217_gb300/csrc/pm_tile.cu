// pm_tile.cu -- one checkerboard colour phase of propagation (Eq. 4) and
// limited random search (Eq. 5), and the cost refresh at the start of a
// visit, squared-L2 cost, on seed tiles staged in shared memory.
//
// A tile is 8 x 8 lattice seeds; the 32 seeds of the current colour update,
// one warp per seed at a time.  Before any cost is computed the tile's
// shared-memory buffer receives
//   - the reference region covering all patches of the tile, in the
//     split-byte form (a = 128 a_h + a_l) that the dp2a cross products use;
//   - a fixed-size target window around the tile's median displacement,
//     wide enough for the random-search square plus a margin, and the sum
//     |b|^2 of every patch centre inside it.
// Both are staged in unclamped pixel coordinates with the image border
// replicated, so the inner loop needs no border tests.  A region that lies
// inside its image moves as one 2D tensor copy (cp.async.bulk.tensor, a
// tensor map per array and slot); one that needs the replicated border moves
// row by row (a bulk copy per row plus 4-byte copies for the clamped words).
// Two producer warps prepare tile n + 1 (seed records, window position,
// copies) while the other warps score tile n.
//
// Lane l owns the words l, l + 32, ... of the flattened patch (P rows of P
// pixels times the words per pixel, no padding), and the shared row pitch is
// congruent to the patch row modulo 32: the 32 consecutive words that a warp
// reads fall in 32 different banks.  A candidate whose patch is not inside
// the window is scored from global memory instead.  The cost of a candidate is
//   D = sum |a|^2 + sum |b|^2 - 2 sum <a, b>,
// exact in integers, with sum |a|^2 per seed and sum |b|^2 per target pixel
// computed by other kernels of the same visit.
#include <limits.h>
#include <mutex>

#include <cuda.h>

#include "match_common.cuh"

namespace pgm {

constexpr int PT_TW = 8, PT_TH = 8;            // lattice seeds per tile
constexpr int PT_NACT = PT_TW * PT_TH / 2;     // seeds of one colour per tile

struct PtGeom {
    int wpp, wprp;         // words per pixel, words per patch row
    int ref_w, ref_h;      // staged reference region (px)
    int win_w, win_h;      // staged target window (px)
    int sp;                // shared row pitch (words)
    int cw, ch;            // candidate centres covered by the window
    int words;             // 32-bit shared words in all (descriptor rows, then uint64 sums)
};

__host__ __device__ inline PtGeom pt_geom(int nch, int P, int sigma, int rs_W, int slack) {
    PtGeom g;
    g.wpp = nch / 2;
    g.wprp = P * g.wpp;                               // words per patch row
    const int span_x = sigma * (PT_TW - 1) + P;
    const int span_y = sigma * (PT_TH - 1) + P;
    const int rho = rs_W > 1 ? rs_W : 1;
    g.ref_w = span_x;
    g.ref_h = span_y;
    g.win_w = span_x + 2 * (rho + slack);
    g.win_h = span_y + 2 * (rho + slack);
    const int need = (g.ref_w > g.win_w ? g.ref_w : g.win_w) * g.wpp;
    g.sp = need + (((g.wprp - need) % 32) + 32) % 32;
    g.cw = g.win_w - P + 1;                           // centres whose patch fits
    g.ch = g.win_h - P + 1;
    g.words = g.sp * (g.ref_h + g.win_h) + 2 * g.cw * g.ch + 2;   // +2: 8-byte alignment
    return g;
}

namespace {


// Copy a rows x (w px) block of 32-bit words with top-left pixel (x0, y0)
// (x0 a multiple of 4) of an image (iw x ih px, row pitch pw words) to shared
// memory (pitch sp), replicating the border.  Interior blocks move as 16-byte
// vectors, others word by word.
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(
                     (unsigned)__cvta_generic_to_shared(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(
                     (unsigned)__cvta_generic_to_shared(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ int lds32(unsigned addr) {
    int v;
    asm volatile("ld.shared.b32 %0, [%1];\n" : "=r"(v) : "r"(addr));
    return v;
}
__device__ __forceinline__ unsigned long long lds64(unsigned addr) {
    unsigned long long v;
    asm volatile("ld.shared.b64 %0, [%1];\n" : "=l"(v) : "r"(addr));
    return v;
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Start copying a rows x (w px) block of 32-bit words with top-left pixel
// (x0, y0) of an image (iw x ih px, row pitch pw words) into shared memory
// (pitch sp), replicating the border: asynchronous 4-byte copies, warps w0,
// w0 + nwarp, ... one row each, lanes across it; completion by
// cp_async_wait_all.
template <int WPP>
__device__ __forceinline__ void stage(uint32_t* dst, int sp, const uint32_t* src, int pw, int iw,
                                      int ih, int x0, int y0, int w, int rows, int w0, int nwarp) {
    const int lane = threadIdx.x & 31;
    const int wwords = w * WPP;
    if (x0 >= 0 && y0 >= 0 && x0 + w <= iw && y0 + rows <= ih) {
        for (int row = w0; row < rows; row += nwarp) {
            const uint32_t* s = src + (size_t)(y0 + row) * pw + (size_t)x0 * WPP;
            uint32_t* d = dst + row * sp;
            for (int wd = lane; wd < wwords; wd += 32) cp_async4(d + wd, s + wd);
        }
    } else {
        for (int row = w0; row < rows; row += nwarp) {
            const uint32_t* srow = src + (size_t)clampi(y0 + row, 0, ih - 1) * pw;
            for (int wd = lane; wd < wwords; wd += 32) {
                const int pix = wd / WPP, wi = wd - pix * WPP;      // WPP is 1 or 3
                cp_async4(dst + row * sp + wd, srow + (size_t)clampi(x0 + pix, 0, iw - 1) * WPP + wi);
            }
        }
    }
}

// Byte offsets of the lane-owned words k = lane + 32 m of a flattened patch
// (row k / wprp, column k % wprp of a staged block with row pitch sp).
template <int M>
struct Offs {
    unsigned p[M];
    __device__ __forceinline__ unsigned at(int m) const { return p[m]; }
};

// The same offsets walked incrementally (no division); bit m of vmask: word
// lane + 32 m is a real patch word.
template <int M>
__device__ __forceinline__ void patch_walk(int lane, int wpr, int nw, int sp, Offs<M>& off,
                                           unsigned& vmask) {
    int row = 0, col = lane;
    while (col >= wpr) { col -= wpr; ++row; }
    vmask = 0;
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const int k = lane + 32 * m;
        off.p[m] = k < nw ? 4u * (unsigned)(row * sp + col) : 0u;
        if (k < nw) vmask |= 1u << m;
        col += 32;
        while (col >= wpr) { col -= wpr; ++row; }
    }
}

// cross term from global memory with replicated borders (fallback)
template <int NCH, int MMAX>
__device__ __forceinline__ long long cross_global(const int (&b)[MMAX], const DirLvl& D, int wprp,
                                                  int qx, int qy, int lane) {
    constexpr int WPP = NCH / 2;
    const int P = D.P, h = P / 2, nw = P * wprp;
    const int pitchw = D.tgt_pitch >> 1;
    const uint32_t* t32 = reinterpret_cast<const uint32_t*>(D.tgt);
    int sl = 0, sh = 0;
#pragma unroll
    for (int m = 0; m < MMAX; ++m)
        if (32 * m < nw) {
            const int k = lane + 32 * m;
            const int row = k / wprp, col = k - row * wprp;
            const int pix = col / WPP, wi = col - pix * WPP;
            const int x = clampi(qx - h + pix, 0, D.tw - 1), y = clampi(qy - h + row, 0, D.th - 1);
            const uint32_t v = __ldg(t32 + (size_t)y * pitchw + (size_t)x * WPP + wi);
            sl = __dp2a_lo((int)v, b[m], sl);
            sh = __dp2a_hi((int)v, b[m], sh);
        }
    sl = __reduce_add_sync(FULL, sl);
    sh = __reduce_add_sync(FULL, sh);
    return (long long)sh * 128 + (long long)sl;
}

// Cost of target centre (qx, qy) for the reference words b: from the staged
// window when the padded patch lies inside it, else from global memory.
template <int NCH, int M>
__device__ __forceinline__ unsigned long long tile_cost(
    const int (&b)[M], const Offs<M>& off, const DirLvl& D, const PtGeom& G, unsigned a_tw,
    unsigned a_sb, bool use_win, int wx0, int wy0, unsigned long long sa, int qx, int qy, int lane,
    unsigned& n_glob) {
    constexpr int WPP = NCH / 2;
    const int P = D.P, h = P / 2;
    unsigned long long sb;
    long long cr;
    const int x0 = qx - h - wx0, y0 = qy - h - wy0;
    if (use_win && x0 >= 0 && y0 >= 0 && x0 + P <= G.win_w && y0 + P <= G.win_h) {
        sb = lds64(a_sb + 8u * (unsigned)(y0 * G.cw + x0));
        const unsigned base = a_tw + 4u * (unsigned)(y0 * G.sp + x0 * WPP);
        int sl0 = 0, sh0 = 0, sl1 = 0, sh1 = 0;     // two chains each
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const int v = lds32(base + off.at(m));
            if (m & 1) { sl1 = __dp2a_lo(v, b[m], sl1); sh1 = __dp2a_hi(v, b[m], sh1); }
            else { sl0 = __dp2a_lo(v, b[m], sl0); sh0 = __dp2a_hi(v, b[m], sh0); }
        }
        const int sl = __reduce_add_sync(FULL, sl0 + sl1);
        const int sh = __reduce_add_sync(FULL, sh0 + sh1);
        cr = (long long)sh * 128 + (long long)sl;
    } else {
        sb = D.sb2[(size_t)qy * D.tw + qx];
        cr = cross_global<NCH, M>(b, D, G.wprp, qx, qy, lane);
        ++n_glob;
    }
    return xcost(sa, sb, cr);
}

// ------------------------------------------------------------------
// Search kernel, persistent form.  A CTA holds two tile buffers in shared
// memory and walks its share of the launch's tiles (all pairs and both
// directions, flattened).  While the consumer warps score the active seeds
// of tile n from one buffer, the producer warps prepare tile n + 1 in the
// other: they read its seeds, drop the propagated candidates that cannot
// change the result (Eq. 4: an unusable neighbour, a centre outside the
// target, a repeat of the current match or of the other candidate), draw the
// first Philox block of every seed for the random search (Eq. 5), place the
// target window at the median match, and stage the reference region, the
// window and the window's sums |b|^2; then they join the consumers on tile
// n.  Rows move as bulk asynchronous copies (one per row, 16-byte aligned,
// completing on the buffer's mbarrier); the words outside the image
// (replicated border) and a ragged row end go by 4-byte copies.  A barrier
// per tile hands the buffers over.
//
// Shared layout.  Every staged row is 16-byte aligned: shared word j of a
// row holds image word x0 * wpp - sh + j, with sh = x0 * wpp mod 4.  The
// words of a flattened patch are spread over 32-word groups of two kinds:
//   A: words 32 j .. 32 j + 31 of patch row r (q = wprp / 32 per row; lane l
//      takes word 32 j + l): 32 consecutive words, conflict-free at any pitch;
//   B: the wl = wprp % 32 remaining words of g consecutive rows; lane l takes
//      word 32 q + l % S of row g b + l / S, with S the power of two >= wl and
//      g = 32 / S.  The window pitch is congruent to S modulo 32 (to 4 when
//      S < 4), so the g row pieces fall in disjoint banks.
// A lane without a word in a B group reads lane 0's word (a broadcast) and
// carries a zero reference.  The reference region has its own, narrower
// pitch; its lane offsets are read from a table when a seed's reference
// words are loaded, the window's stay in registers.
constexpr int PP_CONS = 10, PP_PROD = 2;          // consumer / producer warps
constexpr int PP_THREADS = 32 * (PP_CONS + PP_PROD);
constexpr int PP_MMAX = 24;                      // 32-word groups of the largest patch
constexpr long long PP_WAIT_CYCLES = 1ll << 31;  // bounded mbarrier wait (about 1 s)

struct PpGeom {
    int wpp, wprp, q, wl, S, g, nA, nB, M;
    int ref_w, ref_h, win_w, win_h;   // staged regions (px)
    int spr, spw;                     // words per shared row: reference region, window
    int cw, ch, cwp;                  // window centres (cw x ch), sums row pitch (even)
    int off_win, off_sb;              // word offsets in a buffer
    int words;                        // one buffer (multiple of 4)
};

__host__ __device__ inline int pp_pitch(int need, int res) {
    need = (need + 3) & ~3;
    return need + (((res - need) % 32) + 32) % 32;
}

__host__ __device__ inline PpGeom pp_geom(int nch, int P, int sigma, int rs_W, int slack) {
    PpGeom g;
    g.wpp = nch / 2;
    g.wprp = P * g.wpp;
    g.q = g.wprp / 32;
    g.wl = g.wprp % 32;
    g.S = 0;
    g.g = 0;
    if (g.wl > 0) {
        g.S = 1;
        while (g.S < g.wl) g.S <<= 1;
        g.g = 32 / g.S;
    }
    g.nA = P * g.q;
    g.nB = g.wl > 0 ? (P + g.g - 1) / g.g : 0;
    g.M = g.nA + g.nB;
    const int rho = rs_W > 1 ? rs_W : 1;
    g.ref_w = sigma * (PT_TW - 1) + P;
    g.ref_h = sigma * (PT_TH - 1) + P;
    g.win_w = g.ref_w + 2 * (rho + slack);
    g.win_h = g.ref_h + 2 * (rho + slack);
    const int res = g.S >= 4 ? (g.S & 31) : 4;
    g.spr = pp_pitch(3 + g.ref_w * g.wpp, res);       // + up to 3 words of alignment shift
    g.spw = pp_pitch(3 + g.win_w * g.wpp, res);
    g.cw = g.win_w - P + 1;
    g.ch = g.win_h - P + 1;
    g.cwp = (g.cw + 2) & ~1;                           // + 1 centre of alignment shift
    g.off_win = (g.spr * g.ref_h + 31) & ~31;          // regions start 128-byte aligned
    g.off_sb = (g.off_win + g.spw * g.win_h + 31) & ~31;
    g.words = (g.off_sb + 2 * g.cwp * g.ch + 31) & ~31;
    return g;
}

// Patch row and word of lane l in group m (A or B); *valid = false for a
// lane without a word (it then names lane 0's word of the group).
__host__ __device__ inline void pp_word(const PpGeom& g, int P, int m, int l, int* row, int* col,
                                        bool* valid) {
    if (m >= g.M) { *row = 0; *col = 0; *valid = false; return; }
    if (m < g.nA) {
        *row = m / g.q;
        *col = 32 * (m % g.q) + l;
        *valid = true;
        return;
    }
    const int b = m - g.nA;
    *row = b * g.g + l / g.S;
    *col = 32 * g.q + l % g.S;
    *valid = l % g.S < g.wl && *row < P;
    if (!*valid) { *row = b * g.g; *col = 32 * g.q; }
}

struct __align__(16) SeedRec {      // one active seed of a staged tile
    int s, px, py, f;               // seed index (-1: none), centre, flags
    int u, nb0, nb1, K;             // current match; propagated candidates to score; search count
    int r0, r1, pad0, pad1;         // random-search offsets k = 0, 1 (packed like u); flags as read
    int wu, w0, w1, pad2;           // window slots (pp_slot) of u, nb0, nb1
    unsigned long long cost, sa;    // current cost, sum |a|^2 of the reference patch
};

struct TileHdr { int pair, dir, i0, j0, rx0, wx0, wy0, use_win, shr, shw, shs, pad; };

// The flattened tiles of one launch: slot k owns tiles [cum[k], cum[k + 1]);
// ndir = 1: slot k is pair k in direction dir; ndir = 2: slot k is pair k / 2
// in direction k % 2.
struct PtSched { int nk, total, dir, ndir; int cum[2 * MAXB + 1]; };

constexpr int NO_CAND = INT_MIN;            // no propagated candidate

// Tensor maps of the staged arrays for each slot of a launch (slot k as in
// PtSched): [0] the reference split words (box spr x ref_h words), [1] the
// target words (box spw x win_h), [2] the target sums |b|^2 (uint64, box
// cwp x ch).  A region inside its image moves as one 2D copy; ok[k] = 0, or
// a region that needs the replicated border, goes row by row.
constexpr int PP_MAPS = 32;
struct PtMaps {
    CUtensorMap m[PP_MAPS][3];
    int ok[PP_MAPS];
};

__device__ __forceinline__ void tma2d(unsigned dst, const CUtensorMap* map, int x, int y,
                                      unsigned bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];\n"
        ::"r"(dst), "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void pp_bar_producers() {
    asm volatile("bar.sync 1, %0;\n" ::"n"(32 * PP_PROD) : "memory");
}
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    return ok != 0;
}
// wait for phase `parity` of an mbarrier, giving up after PP_WAIT_CYCLES
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > PP_WAIT_CYCLES) return false;
    return true;
}
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
        ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ int floor_div(int a, int b) {
    return a >= 0 ? a / b : -((-a + b - 1) / b);
}

// Column span of a staged region: shared words [0, nwords) of every row; the
// in-image, 16-byte aligned part [jb, je) goes by one bulk copy per row.
struct Span { int gw0, nwords, jb, je; };
__device__ __forceinline__ Span pp_span(int x0w, int sh, int wwords, int iw_words) {
    Span s;
    s.gw0 = x0w - sh;                                   // a multiple of 4
    s.nwords = (sh + wwords + 3) & ~3;
    const int lo = max(0, -s.gw0), hi = min(s.nwords, iw_words - s.gw0);
    s.jb = min(lo, s.nwords);
    s.je = hi > s.jb ? s.jb + ((hi - s.jb) & ~3) : s.jb;
    return s;
}

// Lane `lane` of one warp stages rows lane, lane + 32, ... of a region
// (row r from image row clamp(y0 + r)); the warp's bulk bytes were announced
// on `bar` by the caller.  Words outside the bulk span: 4-byte copies with the
// pixel clamped (the border replicated).
template <int WPP>
__device__ __forceinline__ void pp_stage_rows(unsigned dst, int sp, const uint32_t* src, int pw,
                                              int iw, int ih, int y0, int rows, const Span& s,
                                              unsigned bar, int lane) {
    const unsigned bulk = (unsigned)(s.je - s.jb) * 4u;
    for (int r = lane; r < rows; r += 32) {
        const uint32_t* srow = src + (size_t)clampi(y0 + r, 0, ih - 1) * pw;
        const unsigned drow = dst + 4u * (unsigned)(r * sp);
        if (bulk) bulk_g2s(drow + 4u * (unsigned)s.jb, srow + s.gw0 + s.jb, bulk, bar);
        for (int half = 0; half < 2; ++half) {          // the words left and right of it
            const int j1 = half ? s.nwords : s.jb;
            for (int j = half ? s.je : 0; j < j1; ++j) {
                const int gw = s.gw0 + j, p = floor_div(gw, WPP), wi = gw - p * WPP;
                const uint32_t* s4 = srow + (size_t)clampi(p, 0, iw - 1) * WPP + wi;
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n"
                             ::"r"(drow + 4u * (unsigned)j), "l"(s4) : "memory");
            }
        }
    }
}

__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

// Producer warps pw = 0, 1: prepare flattened tile t in the buffer at shared
// address `buf`; its bulk copies complete on `bar` (two arrivals: pw 0 after
// announcing the window rows, pw 1 after announcing the reference rows and
// the window sums).
template <int NCH>
__device__ __forceinline__ void pp_produce(const LvlBatch& B, const MatchConst& mc,
                                           const PtSched& S, const PtMaps& TM, int t, unsigned buf,
                                           SeedRec* rec, TileHdr* hdr, int* next,
                                           const PpGeom* geom, unsigned bar, int pw, int lane) {
    constexpr int WPP = NCH / 2;
    int lo = 0, hi = S.nk - 1;                   // slot holding tile t:
    while (lo < hi) {                            // the last k with cum[k] <= t
        const int mid = (lo + hi + 1) >> 1;
        if (S.cum[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const int k = lo, pair = S.ndir == 2 ? k >> 1 : k, dir = S.ndir == 2 ? (k & 1) : S.dir;
    const PpGeom& G = geom[dir];
    const DirLvl& D = B.d[pair][dir];
    const int tiles_x = (D.nx + PT_TW - 1) / PT_TW, tt = t - S.cum[k];
    const int i0 = (tt % tiles_x) * PT_TW, j0 = (tt / tiles_x) * PT_TH;
    const int P = D.P, h = P / 2, sig = mc.sigma;
    const int rx0 = mc.c + sig * i0 - h, ry0 = mc.c + sig * j0 - h;
    const int shr = ((rx0 * WPP) % 4 + 4) % 4;
    const bool tma = k < PP_MAPS && TM.ok[k] != 0 && (buf & 127u) == 0;
    fence_proxy_async();                         // earlier reads of this buffer come first

    if (pw == 1) {
        // the reference region does not depend on the seeds
        const Span sr = pp_span(rx0 * WPP, shr, G.ref_w * WPP, D.rw * WPP);
        if (tma && rx0 >= 0 && rx0 + G.ref_w <= D.rw && ry0 >= 0 && ry0 + G.ref_h <= D.rh) {
            if (lane == 0) {                     // inside the image: one 2D copy
                mbar_expect_tx(bar, 4u * (unsigned)(G.spr * G.ref_h));
                tma2d(buf, &TM.m[k][0], sr.gw0, ry0, bar);
            }
        } else {
            if (lane == 0 && sr.je > sr.jb)
                mbar_expect_tx(bar, (unsigned)(sr.je - sr.jb) * 4u * (unsigned)G.ref_h);
            __syncwarp();
            pp_stage_rows<WPP>(buf, G.spr, D.ref_split, D.ref_pitch >> 1, D.rw, D.rh, ry0, G.ref_h,
                               sr, bar, lane);
        }
    } else {
        const int t4 = mc.t & 3;
        const int sx = (t4 == 0 || t4 == 3) ? 1 : -1, sy = (t4 == 0 || t4 == 2) ? 1 : -1;
        const int a = lane, j = j0 + a / (PT_TW / 2);
        const int i = i0 + 2 * (a % (PT_TW / 2)) + ((j + mc.colour) & 1);
        SeedRec R;
        R.s = -1; R.px = 0; R.py = 0; R.f = 0; R.u = 0; R.nb0 = NO_CAND; R.nb1 = NO_CAND; R.K = 0;
        R.r0 = 0; R.r1 = 0; R.pad0 = 0; R.pad1 = 0; R.cost = INF; R.sa = 0;
        R.wu = -1; R.w0 = -1; R.w1 = -1; R.pad2 = 0;
        if (i < D.nx && j < D.ny) {
            const int s = j * D.nx + i;
            const int ni = i - sx, nj = j - sy;
            const bool okx = ni >= 0 && ni < D.nx, oky = nj >= 0 && nj < D.ny;
            const int sn0 = okx ? j * D.nx + ni : s, sn1 = oky ? nj * D.nx + i : s;
            const int f = D.flags[s], u = D.u[s];
            const int px = mc.c + sig * i, py = mc.c + sig * j;
            const unsigned long long cst = D.cost[s], sa = D.sa2img[(size_t)py * D.rw + px];
            const int f0 = D.flags[sn0], f1 = D.flags[sn1], u0 = D.u[sn0], u1 = D.u[sn1];
            // cost refresh (first iteration of a visit): a match whose centre
            // lies outside the target leaves the seed uninitialised
            bool have = f & F_VALID, ok_n0 = okx && (f0 & F_VALID), ok_n1 = oky && (f1 & F_VALID);
            if (mc.refresh) {
                have = have && inside(D, px + lo16((uint32_t)u), py + hi16((uint32_t)u));
                ok_n0 = ok_n0 && inside(D, px - sx * sig + lo16((uint32_t)u0), py + hi16((uint32_t)u0));
                ok_n1 = ok_n1 && inside(D, px + lo16((uint32_t)u1), py - sy * sig + hi16((uint32_t)u1));
            }
            const int c0 = ok_n0 ? u0 : NO_CAND;
            const int c1 = ok_n1 ? u1 : NO_CAND;
            const bool ok0 = c0 != NO_CAND && !(have && c0 == u) &&
                             inside(D, px + lo16((uint32_t)c0), py + hi16((uint32_t)c0));
            // a repeat of c0 scores the same and cannot be strictly better
            const bool ok1 = c1 != NO_CAND && c1 != c0 && !(have && c1 == u) &&
                             inside(D, px + lo16((uint32_t)c1), py + hi16((uint32_t)c1));
            R.s = s; R.px = px; R.py = py; R.u = u;
            R.f = have ? f : (f & ~F_VALID);
            R.pad0 = f;                           // flags as read
            R.nb0 = ok0 ? c0 : NO_CAND;
            R.nb1 = ok1 ? c1 : NO_CAND;
            R.cost = mc.refresh ? INF : cst;
            R.sa = sa;
            const int g = mc.rs_grid;             // PGM-C3/G3: level-0 search on a grid only
            R.K = (B.level == 0 && g > 0 && !(px % g == g / 2 && py % g == g / 2)) ? 0 : mc.K;
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
        // window centre: per component, the median of the valid current matches
        const bool v = R.s >= 0 && (R.f & F_VALID);
        const unsigned vm = __ballot_sync(FULL, v);
        const int nv = __popc(vm);
        const int ux = lo16((uint32_t)R.u), uy = hi16((uint32_t)R.u);
        // the (nv / 2)-th smallest of the valid components (0-based), one
        // bit at a time from the top of the order-preserving 16-bit keys
        const unsigned kx = (unsigned)(ux + 32768), ky = (unsigned)(uy + 32768);
        unsigned cx = vm, cy = vm;
        int nx = nv / 2, ny = nv / 2;
#pragma unroll
        for (int bit = 15; bit >= 0; --bit) {
            const unsigned zx = __ballot_sync(FULL, !((kx >> bit) & 1u)) & cx;
            const unsigned zy = __ballot_sync(FULL, !((ky >> bit) & 1u)) & cy;
            const int px = __popc(zx), py = __popc(zy);
            if (nx < px) cx = zx; else { nx -= px; cx &= ~zx; }
            if (ny < py) cy = zy; else { ny -= py; cy &= ~zy; }
        }
        const int rho = max(1, mc.rs_W);
        const int medx = __shfl_sync(FULL, ux, cx ? __ffs(cx) - 1 : 0);
        const int medy = __shfl_sync(FULL, uy, cy ? __ffs(cy) - 1 : 0);
        // the window slots of the candidates known now (the current match
        // and the propagated ones)
        const int wx0 = nv > 0 ? mc.c + sig * i0 - h + medx - rho - mc.slack : 0;
        const int wy0 = nv > 0 ? mc.c + sig * j0 - h + medy - rho - mc.slack : 0;
        const int shw = ((wx0 * WPP) % 4 + 4) % 4, shs = (wx0 + h) & 1;
        auto slot = [&](int32_t cu) {
            const int x0 = R.px + lo16((uint32_t)cu) - h - wx0;
            const int y0 = R.py + hi16((uint32_t)cu) - h - wy0;
            if (nv == 0 || cu == NO_CAND || x0 < 0 || y0 < 0 || x0 + P > G.win_w || y0 + P > G.win_h)
                return -1;
            return (int)(4u * (unsigned)(y0 * G.spw + shw + x0 * WPP)) |
                   ((y0 * G.cwp + shs + x0) << 16);
        };
        R.wu = slot(R.u);
        R.w0 = slot(R.nb0);
        R.w1 = slot(R.nb1);
        R.pad2 = 0;
        rec[a] = R;
        if (lane == 0) {
            TileHdr H;
            H.pair = pair; H.dir = dir; H.i0 = i0; H.j0 = j0; H.rx0 = rx0;
            H.use_win = nv > 0;
            H.wx0 = wx0;
            H.wy0 = wy0;
            H.shr = shr;
            H.shw = shw;
            H.shs = shs;
            H.pad = 0;
            *hdr = H;
            *next = 0;
        }
    }
    pp_bar_producers();                           // the window position is known
    const TileHdr H = *hdr;
    const unsigned win = buf + 4u * (unsigned)G.off_win, sbb = buf + 4u * (unsigned)G.off_sb;
    if (pw == 0) {
        const bool win_in = H.wx0 >= 0 && H.wx0 + G.win_w <= D.tw && H.wy0 >= 0 &&
                            H.wy0 + G.win_h <= D.th;
        if (H.use_win && tma && win_in) {
            if (lane == 0) {                     // inside the image: one 2D copy
                mbar_arrive_tx(bar, 4u * (unsigned)(G.spw * G.win_h));
                tma2d(win, &TM.m[k][1], H.wx0 * WPP - H.shw, H.wy0, bar);
            }
        } else if (H.use_win) {
            const Span sw = pp_span(H.wx0 * WPP, H.shw, G.win_w * WPP, D.tw * WPP);
            if (lane == 0) {
                if (sw.je > sw.jb) mbar_arrive_tx(bar, (unsigned)(sw.je - sw.jb) * 4u * (unsigned)G.win_h);
                else mbar_arrive(bar);
            }
            __syncwarp();
            pp_stage_rows<WPP>(win, G.spw, reinterpret_cast<const uint32_t*>(D.tgt),
                               D.tgt_pitch >> 1, D.tw, D.th, H.wy0, G.win_h, sw, bar, lane);
        } else if (lane == 0) {
            mbar_arrive(bar);
        }
    } else {
        // sums |b|^2 of the centres whose patch lies in the window; centres
        // outside the image are never scored, their entries are don't-care
        const int cx0 = H.wx0 + h, cy0 = H.wy0 + h;
        const bool bulk = H.use_win && (D.tw & 1) == 0;
        unsigned bytes = 0;
        int c_lo = 0;
        if (bulk && tma) {
            // one 2D copy; entries outside the image read as zero (don't-care)
            if (lane == 0) {
                mbar_arrive_tx(bar, 8u * (unsigned)(G.cwp * G.ch));
                tma2d(sbb, &TM.m[k][2], cx0 - H.shs, cy0, bar);
            }
        } else if (bulk) {
            const int a0 = cx0 - H.shs;                       // even
            c_lo = max(a0, 0);
            const int c_hi = min(a0 + G.cwp, D.tw);
            bytes = c_hi > c_lo ? (unsigned)(c_hi - c_lo) * 8u : 0u;
            if (lane == 0) {
                if (bytes) mbar_arrive_tx(bar, bytes * (unsigned)G.ch);
                else mbar_arrive(bar);
            }
            __syncwarp();
            if (bytes)
                for (int r = lane; r < G.ch; r += 32) {
                    const unsigned long long* srow =
                        D.sb2 + (size_t)clampi(cy0 + r, 0, D.th - 1) * D.tw;
                    bulk_g2s(sbb + 8u * (unsigned)(r * G.cwp + (c_lo - a0)), srow + c_lo, bytes, bar);
                }
        } else {
            if (lane == 0) mbar_arrive(bar);
            if (H.use_win)
                for (int r = 0; r < G.ch; ++r) {
                    const unsigned long long* srow =
                        D.sb2 + (size_t)clampi(cy0 + r, 0, D.th - 1) * D.tw;
                    for (int col = lane; col < G.cw; col += 32)
                        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n"
                                     ::"r"(sbb + 8u * (unsigned)(r * G.cwp + H.shs + col)),
                                     "l"(srow + clampi(cx0 + col, 0, D.tw - 1)) : "memory");
                }
        }
    }
    cp_async_wait_all();
}

// Group addressing of the consumer.  NA >= 0: groups [0, NA) are A groups
// of a layout with q = 1 (lane l reads word l of patch row m, at byte offset
// 4 (m sp + l) from the patch origin), groups [NA, M) take per-lane offsets
// from the tables; NA < 0: every group takes table offsets.
template <int M, int NA>
struct PpLay {
    static constexpr int A0 = NA >= 0 ? NA : 0;
    static constexpr int NB = M - A0 > 0 ? M - A0 : 1;
    // P = 15 with 6 channels: B groups of g = 2 rows, so a lane's word in B
    // group b sits b * 2 rows below its word in group 0 (the host checks g)
    static constexpr int GB = (M == 23 && NA == 15) ? 2 : 0;
};

// Window slot of target centre (qx, qy): the byte offset of its patch
// corner from the window start in the low 16 bits and the index of its sum
// |b|^2 above, or -1 when the patch is not inside the staged window.
__device__ __forceinline__ int pp_slot(const PpGeom& G, const TileHdr& H, int P, int wpp, int qx,
                                       int qy) {
    const int x0 = qx - P / 2 - H.wx0, y0 = qy - P / 2 - H.wy0;
    if (!H.use_win || x0 < 0 || y0 < 0 || x0 + P > G.win_w || y0 + P > G.win_h) return -1;
    return (int)(4u * (unsigned)(y0 * G.spw + H.shw + x0 * wpp)) | ((y0 * G.cwp + H.shs + x0) << 16);
}

// Cross term <a, b> of the reference words b with the target patch whose
// corner is at shared byte address `base` (window pitch SPW > 0 as a
// constant, else G.spw).
template <int M, int NA, int SPW>
__device__ __forceinline__ long long pp_dot_win(const int (&b)[M],
                                                const Offs<PpLay<M, NA>::NB>& off,
                                                const PpGeom& G, unsigned base, int lane) {
    constexpr int A0 = PpLay<M, NA>::A0, GB = SPW > 0 ? PpLay<M, NA>::GB : 0;
    const int spw = SPW > 0 ? SPW : G.spw;
    const unsigned basel = base + 4u * (unsigned)lane, baseb = base + off.at(0);
    int l0 = 0, l1 = 0, h0 = 0, h1 = 0;                 // two chains each
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const unsigned addr = m < A0 ? basel + 4u * (unsigned)(m * spw)
                              : GB > 0 ? baseb + 4u * (unsigned)((m - A0) * GB * spw)
                                       : base + off.at(m - A0);
        const int v = lds32(addr);
        if (m & 1) { l1 = __dp2a_lo(v, b[m], l1); h1 = __dp2a_hi(v, b[m], h1); }
        else { l0 = __dp2a_lo(v, b[m], l0); h0 = __dp2a_hi(v, b[m], h0); }
    }
    const int sl = __reduce_add_sync(FULL, l0 + l1), sh = __reduce_add_sync(FULL, h0 + h1);
    return (long long)sh * 128 + (long long)sl;
}

// The same from global memory with the border replicated (a patch outside
// the staged window).
template <int NCH, int M, int NA, int SPW>
__device__ __forceinline__ long long pp_dot_glob(const int (&b)[M],
                                                 const Offs<PpLay<M, NA>::NB>& off,
                                                 const unsigned short* offw, const DirLvl& D,
                                                 const PpGeom& G, int qx, int qy, int lane) {
    constexpr int GB = SPW > 0 ? PpLay<M, NA>::GB : 0;
    constexpr int WPP = NCH / 2, A0 = PpLay<M, NA>::A0;
    const int h = D.P / 2, spw = SPW > 0 ? SPW : G.spw;
    const int pitchw = D.tgt_pitch >> 1;
    const uint32_t* t32 = reinterpret_cast<const uint32_t*>(D.tgt);
    int sl = 0, sh = 0;
#pragma unroll
    for (int m = 0; m < M; ++m) {
        int row = m, col = lane;
        if (m >= A0) {
            const int o = (int)((GB > 0 ? (unsigned)offw[m * 32 + lane] : off.at(m - A0)) >> 2);
            row = o / spw;
            col = o - row * spw;
        }
        const int pix = col / WPP, wi = col - pix * WPP;
        const int x = clampi(qx - h + pix, 0, D.tw - 1), y = clampi(qy - h + row, 0, D.th - 1);
        const int v = (int)__ldg(t32 + (size_t)y * pitchw + (size_t)x * WPP + wi);
        sl = __dp2a_lo(v, b[m], sl);
        sh = __dp2a_hi(v, b[m], sh);
    }
    sl = __reduce_add_sync(FULL, sl);
    sh = __reduce_add_sync(FULL, sh);
    return (long long)sh * 128 + (long long)sl;
}

// Consumer warps: the active seeds of the tile in the buffer at `buf`, taken
// one at a time from a shared counter.  M = 32-word groups of the patch;
// NA as for PpLay (NA < 0: M is an upper bound and the masks come from the
// geometry at run time); SPW, SPR > 0: window / reference pitches as
// constants.
template <int NCH, int M, int NA, int SPW, int SPR>
__device__ __forceinline__ void pp_consume(const LvlBatch& B, const MatchConst& mc,
                                           const TileHdr& H, const PpGeom& G, const SeedRec* rec,
                                           unsigned buf, const unsigned short* offr,
                                           const unsigned short* offw, int* next, int lane) {
    constexpr int WPP = NCH / 2, A0 = PpLay<M, NA>::A0, NB = PpLay<M, NA>::NB;
    const DirLvl& D = B.d[H.pair][H.dir];
    const int P = D.P, h = P / 2, sig = mc.sigma, spr = SPR > 0 ? SPR : G.spr;
    const unsigned a_ref = buf, a_tw = buf + 4u * (unsigned)G.off_win;
    const unsigned a_sb = buf + 4u * (unsigned)G.off_sb;
    constexpr int GB = SPW > 0 && SPR > 0 ? PpLay<M, NA>::GB : 0;
    Offs<NB> off;                           // byte offsets of the lane's table-addressed words
#pragma unroll
    for (int m = 0; m < NB; ++m)
        off.p[m] = A0 + m < M && (GB == 0 || m == 0) ? offw[(A0 + m) * 32 + lane] : 0u;
    // zero references: B-group lanes without a word, and past the last row
    const bool has_b = G.S == 0 || lane % G.S < G.wl;
    const int mask_b = has_b ? -1 : 0;
    const int mask_last = (has_b && (G.nB == 0 || (G.nB - 1) * G.g + lane / G.S < P)) ? -1 : 0;
    unsigned n_eval = 0, n_cost = 0, n_glob = 0;
    for (;;) {
        int a = 0;
        if (lane == 0) a = atomicAdd(next, 1);
        a = __shfl_sync(FULL, a, 0);
        if (a >= PT_NACT) break;
        const SeedRec R = rec[a];
        if (R.s < 0) continue;
        bool have = R.f & F_VALID;
        if (!have && R.nb0 == NO_CAND && R.nb1 == NO_CAND) {          // nothing to score
            if (lane == 0 && R.f != R.pad0) D.flags[R.s] = (uint8_t)R.f;   // refresh dropped it
            continue;
        }
        int32_t bu = R.u;
        unsigned long long bc = have ? R.cost : INF;
        int b[M];
        const unsigned rbase = a_ref + 4u * (unsigned)((a / (PT_TW / 2)) * sig * spr + H.shr +
                                                       (R.px - h - H.rx0) * WPP);
        const unsigned rbasel = rbase + 4u * (unsigned)lane;
        const unsigned rbaseb = GB > 0 ? rbase + offr[A0 * 32 + lane] : 0u;
#pragma unroll
        for (int m = 0; m < M; ++m) {
            b[m] = lds32(m < A0 ? rbasel + 4u * (unsigned)(m * spr)
                         : GB > 0 ? rbaseb + 4u * (unsigned)((m - A0) * GB * spr)
                                  : rbase + offr[m * 32 + lane]);
            if (NA >= 0) {
                if (m >= NA) b[m] &= (m == M - 1) ? mask_last : mask_b;
            } else {
                b[m] &= m < G.nA ? -1 : (m < G.M - 1 ? mask_b : (m == G.M - 1 ? mask_last : 0));
            }
        }
        // one loop over the candidate sequence (one inlined cost site each for
        // the window and for global memory): c = -1: the current match (cost
        // refresh); c = 0, 1: propagated matches (Eq. 4); c >= 2: random
        // search (Eq. 5) around the match held after propagation.  The first
        // three come with their window slots.
        int ux0 = 0, uy0 = 0;
        uint4 r = make_uint4(0, 0, 0, 0);
#pragma unroll 1
        for (int c = (mc.refresh && have) ? -1 : 0; c < 2 + R.K; ++c) {
            int32_t cu;
            int qx, qy, slot;
            if (c < 2) {
                cu = c < 0 ? R.u : (c ? R.nb1 : R.nb0);
                if (cu == NO_CAND) continue;
                slot = c < 0 ? R.wu : (c ? R.w1 : R.w0);
                qx = R.px + lo16((uint32_t)cu);
                qy = R.py + hi16((uint32_t)cu);
            } else {
                if (!have) break;
                const int k = c - 2;
                if (k == 0) { ux0 = lo16((uint32_t)bu); uy0 = hi16((uint32_t)bu); }
                int dx, dy;
                if (k < 2) {
                    const uint32_t o = (uint32_t)(k ? R.r1 : R.r0);
                    dx = lo16(o);
                    dy = hi16(o);
                } else {
                    if ((k & 1) == 0)
                        r = philox(make_uint4((uint32_t)R.s,
                                              ((uint32_t)B.visit << 16) | ((uint32_t)H.dir << 15) |
                                                  (uint32_t)mc.t,
                                              ((uint32_t)B.level << 16) | (uint32_t)(k >> 1),
                                              B.stream_id[H.pair]),
                                   mc.key0, mc.key1);
                    dx = rs_off((k & 1) ? r.z : r.x, k, mc.rs_W, mc.rs_mode);
                    dy = rs_off((k & 1) ? r.w : r.y, k, mc.rs_W, mc.rs_mode);
                }
                if (dx == 0 && dy == 0) continue;
                qx = R.px + ux0 + dx;               // tested before packing into 16 bits
                qy = R.py + uy0 + dy;
                if (!inside(D, qx, qy)) continue;
                cu = pack_u(ux0 + dx, uy0 + dy);
                slot = pp_slot(G, H, P, WPP, qx, qy);
            }
            if (c < 0) ++n_cost; else ++n_eval;
            unsigned long long sb;
            long long cr;
            if (slot >= 0) {
                sb = lds64(a_sb + 8u * (unsigned)(slot >> 16));
                cr = pp_dot_win<M, NA, SPW>(b, off, G, a_tw + (unsigned)(slot & 0xffff), lane);
            } else {
                sb = D.sb2[(size_t)qy * D.tw + qx];
                cr = pp_dot_glob<NCH, M, NA, SPW>(b, off, offw, D, G, qx, qy, lane);
                ++n_glob;
            }
            const unsigned long long cst = xcost(R.sa, sb, cr);
            if (cst < bc) { bc = cst; bu = cu; have = true; }
        }
        if (lane == 0) {
            if (have && (mc.refresh || bu != R.u || !(R.f & F_VALID))) {
                D.u[R.s] = bu;
                D.cost[R.s] = bc;
                D.flags[R.s] = (uint8_t)(R.f | F_VALID);
            } else if (!have && R.f != R.pad0) {
                D.flags[R.s] = (uint8_t)R.f;
            }
        }
    }
    if (lane == 0) {
        if (n_eval) atomicAdd(B.evals[H.pair] + H.dir, (unsigned long long)n_eval);
        if (n_cost) atomicAdd(B.evals[H.pair] + 2 + H.dir, (unsigned long long)n_cost);
        if (n_glob) atomicAdd(B.evals[H.pair] + 6 + H.dir, (unsigned long long)n_glob);
    }
}

// One colour phase of one direction for all pairs of the launch; the
// consumer is specialised at compile time (M, NA, SPW, SPR as for
// pp_consume), so each specialisation is its own kernel with its own register
// allocation.
template <int NCH, int M, int NA, int SPW, int SPR>
__global__ void __launch_bounds__(PP_THREADS, 2)
k_pm_t(const __grid_constant__ LvlBatch B, const MatchConst mc, const __grid_constant__ PtSched S,
       const __grid_constant__ PtMaps TM, const int buf_words) {
    extern __shared__ __align__(128) uint32_t sm[];
    __shared__ SeedRec s_rec[2][PT_NACT];
    __shared__ TileHdr s_hdr[2];
    __shared__ PpGeom s_geom[2];
    __shared__ unsigned short s_offr[2][PP_MMAX * 32], s_offw[2][PP_MMAX * 32];
    __shared__ __align__(8) unsigned long long s_bar[2];
    __shared__ int s_next[2], s_abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned a_sm = (unsigned)__cvta_generic_to_shared(sm);
    const unsigned bar0 = (unsigned)__cvta_generic_to_shared(&s_bar[0]);
    if (threadIdx.x < 2)
        s_geom[threadIdx.x] = pp_geom(NCH, B.d[0][threadIdx.x].P, mc.sigma, mc.rs_W, mc.slack);
    if (threadIdx.x == 0) {
        mbar_init(bar0, 2);
        mbar_init(bar0 + 8, 2);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    constexpr int MT0 = NA >= 0 ? NA : 0;        // groups read through the tables: [MT0, M)
    const int d0 = S.ndir == 2 ? 0 : S.dir, nd = S.ndir == 2 ? 2 : 1;
    for (int e = threadIdx.x; e < nd * (M - MT0) * 32; e += PP_THREADS) {
        const int d = d0 + e / ((M - MT0) * 32), i = MT0 * 32 + e % ((M - MT0) * 32);
        const int m = i >> 5, l = i & 31;
        const PpGeom& G = s_geom[d];
        int row, col;
        bool valid;
        pp_word(G, B.d[0][d].P, m, l, &row, &col, &valid);
        s_offr[d][i] = (unsigned short)(4 * (row * G.spr + col));
        s_offw[d][i] = (unsigned short)(4 * (row * G.spw + col));
    }
    int t = blockIdx.x;                          // the host launches at most S.total CTAs
    if (warp >= PP_CONS)
        pp_produce<NCH>(B, mc, S, TM, t, a_sm, s_rec[0], &s_hdr[0], &s_next[0], s_geom, bar0,
                        warp - PP_CONS, lane);
    __syncthreads();
    unsigned pend_bar = 0, pend_par = 0;         // producers: copies not yet waited for
    for (int n = 0; t < S.total; ++n, t += gridDim.x) {
        const int cur = n & 1;
        if (warp >= PP_CONS) {
            pend_bar = 0;
            if (t + (int)gridDim.x < S.total) {
                pend_bar = bar0 + 8u * (unsigned)(cur ^ 1);
                pend_par = (unsigned)((n + 1) >> 1) & 1u;
                pp_produce<NCH>(B, mc, S, TM, t + gridDim.x, a_sm + 4u * (unsigned)((cur ^ 1) * buf_words),
                                s_rec[cur ^ 1], &s_hdr[cur ^ 1], &s_next[cur ^ 1], s_geom, pend_bar,
                                warp - PP_CONS, lane);
            }
        }
        {   // every warp: the current tile's seeds (producers join once done)
            const TileHdr H = s_hdr[cur];
            if (!__all_sync(FULL, mbar_wait(bar0 + 8u * (unsigned)cur, (unsigned)(n >> 1) & 1u))) {
                if (lane == 0) {
                    atomicOr(B.err[H.pair], (unsigned)PGM_ERR_TIMEOUT);
                    s_abort = 1;
                }
            } else {
                pp_consume<NCH, M, NA, SPW, SPR>(B, mc, H, s_geom[H.dir], s_rec[cur],
                                                 a_sm + 4u * (unsigned)(cur * buf_words),
                                                 s_offr[H.dir], s_offw[H.dir], &s_next[cur], lane);
            }
        }
        __syncthreads();
        if (s_abort) break;
    }
    // after a timed-out wait: let this thread's bulk copies land before leaving
    if (pend_bar && s_abort) (void)mbar_wait(pend_bar, pend_par);
}

// ------------------------------------------------------------------
// Cost refresh at the start of a visit, tile form: all 64 seeds of a tile
// score their current match with the same staging as the search kernel (the
// window sits at the median of the tile's current matches).  A seed whose
// match centre lies outside the target becomes uninitialised.  Every seed's
// sum |a|^2 is copied from the reference box image for the search kernel.
constexpr int PC_N = PT_TW * PT_TH;

template <int NCH, int M, bool EXACT>
__device__ __forceinline__ void cost_seeds(const LvlBatch& B, const MatchConst& mc,
                                           const DirLvl& D, const PtGeom& G, const int* s_seed,
                                           const int* s_u, const unsigned char* s_f,
                                           const unsigned long long* s_sa, const uint32_t* s_ref,
                                           const uint32_t* s_tw, const unsigned long long* s_sb,
                                           int i0, int j0, int rx0, bool use_win, int wx0,
                                           int wy0) {
    constexpr int WPP = NCH / 2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int pair = blockIdx.z, dir = blockIdx.y;
    const int P = D.P, h = P / 2, sig = mc.sigma, nw = P * G.wprp;
    const unsigned a_ref = (unsigned)__cvta_generic_to_shared(s_ref);
    const unsigned a_tw = (unsigned)__cvta_generic_to_shared(s_tw);
    const unsigned a_sb = (unsigned)__cvta_generic_to_shared(s_sb);
    Offs<M> off;
    unsigned vmask;
    patch_walk<M>(lane, G.wprp, nw, G.sp, off, vmask);
    unsigned n_eval = 0, n_glob = 0;
    for (int a = warp; a < PC_N; a += 8) {
        const int s = s_seed[a];
        if (s < 0 || !(s_f[a] & F_VALID)) continue;
        const int i = i0 + a % PT_TW, j = j0 + a / PT_TW;
        const int px = mc.c + sig * i, py = mc.c + sig * j;
        const int qx = px + lo16((uint32_t)s_u[a]), qy = py + hi16((uint32_t)s_u[a]);
        if (!inside(D, qx, qy)) {
            if (lane == 0) D.flags[s] = s_f[a] & ~F_VALID;
            continue;
        }
        const unsigned rbase = a_ref + 4u * (unsigned)(sig * (j - j0) * G.sp + (px - h - rx0) * WPP);
        int b[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            b[m] = lds32(rbase + off.at(m));
            if (!EXACT || m == M - 1) b[m] &= (int)(0u - ((vmask >> m) & 1u));
        }
        const unsigned long long c = tile_cost<NCH, M>(b, off, D, G, a_tw, a_sb, use_win, wx0, wy0,
                                                       s_sa[a], qx, qy, lane, n_glob);
        ++n_eval;
        if (lane == 0) D.cost[s] = c;
    }
    if (lane == 0 && n_eval) atomicAdd(B.evals[pair] + 2 + dir, (unsigned long long)n_eval);
}

template <int NCH>
__global__ void __launch_bounds__(256, (NCH == 6 ? 2 : 3))
k_cost_t(const __grid_constant__ LvlBatch B, const MatchConst mc) {
    constexpr int WPP = NCH / 2;
    extern __shared__ __align__(128) uint32_t sm[];
    __shared__ int s_seed[PC_N], s_u[PC_N], s_ux[PC_N], s_uy[PC_N];
    __shared__ unsigned char s_f[PC_N];
    __shared__ unsigned long long s_sa[PC_N];
    __shared__ int s_med[2];
    const int dir = blockIdx.y;
    const DirLvl& D = B.d[blockIdx.z][dir];
    const int tiles_x = (D.nx + PT_TW - 1) / PT_TW, tiles_y = (D.ny + PT_TH - 1) / PT_TH;
    if ((int)blockIdx.x >= tiles_x * tiles_y) return;
    const int i0 = ((int)blockIdx.x % tiles_x) * PT_TW, j0 = ((int)blockIdx.x / tiles_x) * PT_TH;
    const int P = D.P, h = P / 2, sig = mc.sigma;
    const PtGeom G = pt_geom(NCH, P, sig, mc.rs_W, mc.slack);
    uint32_t* s_ref = sm;
    uint32_t* s_tw = sm + G.ref_h * G.sp;
    unsigned long long* s_sb = reinterpret_cast<unsigned long long*>(
        sm + ((G.sp * (G.ref_h + G.win_h) + 1) & ~1));
    const int rx0 = mc.c + sig * i0 - h, ry0 = mc.c + sig * j0 - h;
    stage<WPP>(s_ref, G.sp, D.ref_split, D.ref_pitch >> 1, D.rw, D.rh, rx0, ry0, G.ref_w, G.ref_h,
               threadIdx.x >> 5, 8);

    bool valid = false;
    if (threadIdx.x < PC_N) {
        const int a = threadIdx.x;
        const int i = i0 + a % PT_TW, j = j0 + a / PT_TW;
        int s = -1, u = 0, f = 0;
        if (i < D.nx && j < D.ny) {
            s = j * D.nx + i;
            f = D.flags[s];
            u = D.u[s];
            const unsigned long long sa =
                D.sa2img[(size_t)(mc.c + sig * j) * D.rw + (mc.c + sig * i)];
            s_sa[a] = sa;
            D.sa2[s] = sa;
        }
        s_seed[a] = s;
        s_u[a] = u;
        s_f[a] = (unsigned char)f;
        valid = s >= 0 && (f & F_VALID);
        s_ux[a] = valid ? lo16((uint32_t)u) : INT_MAX;
        s_uy[a] = valid ? hi16((uint32_t)u) : INT_MAX;
        if (a == 0) { s_med[0] = INT_MIN; s_med[1] = INT_MIN; }
    }
    const int nv = __syncthreads_count(valid);
    // median of the valid current displacements: rank by (value, index)
    if (threadIdx.x < PC_N && valid) {
        const int a = threadIdx.x, ux = s_ux[a], uy = s_uy[a];
        int rx = 0, ry = 0;
        for (int o = 0; o < PC_N; ++o) {          // invalid entries hold INT_MAX
            const int ox = s_ux[o], oy = s_uy[o];
            rx += ox < ux || (ox == ux && o < a);
            ry += oy < uy || (oy == uy && o < a);
        }
        if (rx == nv / 2) s_med[0] = ux;
        if (ry == nv / 2) s_med[1] = uy;
    }
    __syncthreads();
    const int rho = max(1, mc.rs_W);
    const bool use_win = s_med[0] != INT_MIN;
    const int wx0 = use_win ? mc.c + sig * i0 - h + s_med[0] - rho - mc.slack : 0;
    const int wy0 = use_win ? mc.c + sig * j0 - h + s_med[1] - rho - mc.slack : 0;
    if (use_win) {
        stage<WPP>(s_tw, G.sp, reinterpret_cast<const uint32_t*>(D.tgt), D.tgt_pitch >> 1, D.tw,
                   D.th, wx0, wy0, G.win_w, G.win_h, threadIdx.x >> 5, 8);
        const int cx0 = wx0 + h, cy0 = wy0 + h, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int row = warp; row < G.ch; row += 8) {
            const unsigned long long* srow = D.sb2 + (size_t)clampi(cy0 + row, 0, D.th - 1) * D.tw;
            for (int col = lane; col < G.cw; col += 32)
                cp_async8(s_sb + row * G.cw + col, srow + clampi(cx0 + col, 0, D.tw - 1));
        }
    }
    cp_async_wait_all();
    __syncthreads();
    const int groups = (P * G.wprp + 31) / 32;
#define PGM_COST_SEEDS(MM, EX)                                                                 \
    cost_seeds<NCH, MM, EX>(B, mc, D, G, s_seed, s_u, s_f, s_sa, s_ref, s_tw, s_sb, i0, j0, rx0,   \
                        use_win, wx0, wy0)
    if (NCH == 6) {
        if (groups == 6) PGM_COST_SEEDS(6, true);
        else if (groups == 12) PGM_COST_SEEDS(12, true);
        else if (groups == 22) PGM_COST_SEEDS(22, true);
        else if (groups == 24) PGM_COST_SEEDS(24, true);
        else if (groups <= 4) PGM_COST_SEEDS(4, false);
        else if (groups <= 8) PGM_COST_SEEDS(8, false);
        else if (groups <= 16) PGM_COST_SEEDS(16, false);
        else PGM_COST_SEEDS(24, false);
    } else {
        if (groups == 2) PGM_COST_SEEDS(2, true);
        else if (groups == 4) PGM_COST_SEEDS(4, true);
        else if (groups == 8) PGM_COST_SEEDS(8, true);
        else if (groups <= 2) PGM_COST_SEEDS(2, false);
        else if (groups <= 4) PGM_COST_SEEDS(4, false);
        else PGM_COST_SEEDS(8, false);
    }
#undef PGM_COST_SEEDS
}

// ===========================================================================
// Host side: launch configuration.  No device code below this line.

// The search kernel's parameters (batch, constants, schedule, tensor maps)
// must fit the 32764-byte kernel parameter limit.
static_assert(sizeof(LvlBatch) + sizeof(MatchConst) + sizeof(PtSched) + sizeof(PtMaps) +
                  sizeof(int) + 256 <= 32764,
              "k_pm_t parameters exceed the kernel parameter limit");

// Per-thread caches keyed by device: the shared-memory opt-in of a kernel is a
// per-device attribute, and calls may come from several host threads.
static bool opt_in_smem(const void* kern, int smem, int* cfg_dev, int* configured) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (dev != *cfg_dev) {
        *cfg_dev = dev;
        *configured = 0;
    }
    if (*configured < smem) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
            cudaSuccess) return false;
        *configured = smem;
    }
    return true;
}

template <int NCH>
pgm_status launch_c(const LvlBatch& B, const MatchConst& mc, int tiles, int smem_bytes,
                    cudaStream_t st) {
    static thread_local int cfg_dev = -1, configured = 0;
    if (!opt_in_smem((const void*)k_cost_t<NCH>, smem_bytes, &cfg_dev, &configured))
        return PGM_ERR_CUDA;
    k_cost_t<NCH><<<dim3(tiles, 2, B.n), 256, smem_bytes, st>>>(B, mc);
    return cudaGetLastError() == cudaSuccess ? PGM_OK : PGM_ERR_CUDA;
}

// Grid of the persistent search kernel: as many CTAs as fit on the device at
// once (the occupancy query is cached per specialisation, device and
// shared-memory size), never more than there are tiles.
template <int NCH, int M, int NA, int SPW, int SPR>
pgm_status launch_t(const LvlBatch& B, const MatchConst& mc, const PtSched& S, const PtMaps& TM,
                    int buf_words, cudaStream_t st) {
    const int smem = 2 * buf_words * 4;
    static thread_local int cfg_dev = -1, configured = 0;   // opt-in above 48 KB
    static thread_local int cache_dev = -1, cache_smem = -1, cache_cap = 0;
    auto kern = k_pm_t<NCH, M, NA, SPW, SPR>;
    if (!opt_in_smem((const void*)kern, smem, &cfg_dev, &configured)) return PGM_ERR_CUDA;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PGM_ERR_CUDA;
    if (dev != cache_dev || smem != cache_smem) {
        int sms = 0, per = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, PP_THREADS, smem) !=
                cudaSuccess || per < 1)
            return PGM_ERR_CUDA;
        cache_cap = sms * per;
        cache_dev = dev;
        cache_smem = smem;
    }
    const int grid = S.total < cache_cap ? S.total : cache_cap;
    kern<<<grid, PP_THREADS, smem, st>>>(B, mc, S, TM, buf_words);
    return cudaGetLastError() == cudaSuccess ? PGM_OK : PGM_ERR_CUDA;
}

// The consumer specialisation for a direction's layout: exact layouts of the
// common patch sides (6 channels: P 15, 11, 16), with constant pitches for
// the default geometry (seed stride 3, W = 2, margin 2); other layouts take
// an upper bound of the group count with run-time masks.
template <int NCH>
pgm_status launch_dir(const LvlBatch& B, const MatchConst& mc, const PtSched& S, const PpGeom& G,
                      const PtMaps& TM, int buf_words, cudaStream_t st) {
    if constexpr (NCH == 6) {
        if (G.q == 1 && G.M == 23 && G.nA == 15)
            return (G.spw == 144 && G.spr == 112 && G.g == 2) ? launch_t<6, 23, 15, 144, 112>(B, mc, S, TM, buf_words, st)
                                                  : launch_t<6, 23, 15, 0, 0>(B, mc, S, TM, buf_words, st);
        if (G.q == 1 && G.M == 12 && G.nA == 11)
            return (G.spw == 132 && G.spr == 100) ? launch_t<6, 12, 11, 132, 100>(B, mc, S, TM, buf_words, st)
                                                  : launch_t<6, 12, 11, 0, 0>(B, mc, S, TM, buf_words, st);
        if (G.q == 1 && G.M == 24 && G.nA == 16) return launch_t<6, 24, 16, 0, 0>(B, mc, S, TM, buf_words, st);
        if (G.M <= 8) return launch_t<6, 8, -1, 0, 0>(B, mc, S, TM, buf_words, st);
        if (G.M <= 16) return launch_t<6, 16, -1, 0, 0>(B, mc, S, TM, buf_words, st);
        return launch_t<6, 24, -1, 0, 0>(B, mc, S, TM, buf_words, st);
    } else {
        return launch_t<NCH, 8, -1, 0, 0>(B, mc, S, TM, buf_words, st);   // 2 channels: M <= 8
    }
}
}  // namespace

// the packed 16-bit byte offsets of a patch must fit
static bool pt_offsets_fit(const LvlBatch& B, int nch, const MatchConst& mc) {
    for (int k = 0; k < B.n; ++k)
        for (int d = 0; d < 2; ++d) {
            const int P = B.d[k][d].P;
            const PtGeom g = pt_geom(nch, P, mc.sigma, mc.rs_W, mc.slack);
            if (4L * ((long)(P - 1) * g.sp + g.wprp) >= 65536L) return false;
        }
    return true;
}

// Per-direction schedules S[0], S[1], the schedule of both directions
// together S[2], and the layouts; false when two tile buffers would not fit
// in shared memory, a lane offset would not fit in 16 bits or a staged row
// could not move by 16-byte bulk copies.
static bool pp_plan(const LvlBatch& B, const MatchConst& mc, int nch, PtSched* S, PpGeom* G) {
    bool ok = true;
    S[2].nk = 2 * B.n;
    S[2].total = 0;
    S[2].dir = 0;
    S[2].ndir = 2;
    for (int d = 0; d < 2; ++d) {
        S[d].nk = B.n;
        S[d].total = 0;
        S[d].dir = d;
        S[d].ndir = 1;
        G[d] = pp_geom(nch, B.d[0][d].P, mc.sigma, mc.rs_W, mc.slack);
        if (G[d].M > PP_MMAX || 4L * ((long)(B.d[0][d].P - 1) * G[d].spw + G[d].wprp) >= 65536L ||
            2L * G[d].words * 4 > 200L * 1024 || 4L * G[d].spw * G[d].win_h >= 65536L ||
            (long)G[d].cwp * G[d].ch >= 32768L)
            ok = false;
    }
    for (int k = 0; k < B.n; ++k)
        for (int d = 0; d < 2; ++d) {
            const DirLvl& D = B.d[k][d];
            const int tiles = ((D.nx + PT_TW - 1) / PT_TW) * ((D.ny + PT_TH - 1) / PT_TH);
            S[d].cum[k] = S[d].total;
            S[d].total += tiles;
            S[2].cum[2 * k + d] = S[2].total;
            S[2].total += tiles;
            if (D.P != B.d[0][d].P) ok = false;
            if ((((uintptr_t)D.ref_split | (uintptr_t)D.tgt | (uintptr_t)D.sb2) & 15) != 0 ||
                (D.ref_pitch * 2) % 16 != 0 || (D.tgt_pitch * 2) % 16 != 0)
                ok = false;
        }
    S[0].cum[B.n] = S[0].total;
    S[1].cum[B.n] = S[1].total;
    S[2].cum[2 * B.n] = S[2].total;
    return ok;
}

bool pm_tile_fits(const LvlBatch& B, const MatchConst& mc, int nch) {
    PtSched S[3];
    PpGeom G[2];
    return mc.norm == PGM_L2SQ && pp_plan(B, mc, nch, S, G);
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
// `pitch` bytes apart, box0 x box1 elements per copy, zero fill outside.
// False when the arguments break a tensor-map rule (then the slot stages
// row by row).
static bool map2d(CUtensorMap* out, const void* ptr, unsigned long long dim0,
                  unsigned long long dim1, unsigned long long pitch, unsigned box0, unsigned box1,
                  unsigned esize) {
    if (box0 == 0 || box1 == 0 || box0 > 256 || box1 > 256 || box0 > dim0 || box1 > dim1 ||
        (box0 * esize) % 16 != 0 || pitch % 16 != 0 || ((uintptr_t)ptr & 15) != 0 ||
        pitch < dim0 * esize)
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

// The maps of every slot of schedule S (one thread's launch parameters).
static PtMaps& pp_maps(const LvlBatch& B, int nch, const PtSched& S, const PpGeom* G) {
    static thread_local PtMaps TM;
    const int wpp = nch / 2;
    for (int k = 0; k < PP_MAPS; ++k) {
        TM.ok[k] = 0;
        if (k >= S.nk) continue;
        const int pair = S.ndir == 2 ? k >> 1 : k, dir = S.ndir == 2 ? (k & 1) : S.dir;
        const DirLvl& D = B.d[pair][dir];
        const PpGeom& g = G[dir];
        TM.ok[k] = (D.tw & 1) == 0 &&
                   map2d(&TM.m[k][0], D.ref_split, (unsigned long long)D.rw * wpp, D.rh,
                         2ull * D.ref_pitch, g.spr, g.ref_h, 4) &&
                   map2d(&TM.m[k][1], D.tgt, (unsigned long long)D.tw * wpp, D.th,
                         2ull * D.tgt_pitch, g.spw, g.win_h, 4) &&
                   map2d(&TM.m[k][2], D.sb2, D.tw, D.th, 8ull * D.tw, g.cwp, g.ch, 8);
    }
    return TM;
}

static int device_sms();

bool pm_tile_split(const LvlBatch& B, const MatchConst& mc, int nch) {
    PtSched S[3];
    PpGeom G[2];
    return mc.norm == PGM_L2SQ && pp_plan(B, mc, nch, S, G) && S[2].total > 2 * device_sms();
}

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

// *handled = false when pp_plan refuses the batch; the caller then uses the
// per-seed kernel.  A small phase (at most one tile per resident CTA, the
// coarse levels) runs both directions in one launch of the general
// consumer; a larger one runs each direction in its own launch of the
// consumer specialised for its layout, the backward one on st2 when given
// (the two directions are independent within a phase).  *nlaunch: kernels
// launched.
pgm_status launch_pm_tile(const LvlBatch& B, const MatchConst& mc, int nch, int maxP, int* nlaunch,
                          bool* handled, cudaStream_t st, cudaStream_t st2) {
    (void)maxP;
    *handled = false;
    *nlaunch = 0;
    PtSched S[3];
    PpGeom G[2];
    if (!pp_plan(B, mc, nch, S, G)) return PGM_OK;
    *handled = true;
    if (S[2].total == 0) return PGM_OK;
    const int words = G[0].words > G[1].words ? G[0].words : G[1].words;
    if (S[2].total <= 2 * device_sms()) {
        const int m = G[0].M > G[1].M ? G[0].M : G[1].M;
        *nlaunch = 1;
        PtMaps& TM = pp_maps(B, nch, S[2], G);
        if (nch == 2) return launch_t<2, 8, -1, 0, 0>(B, mc, S[2], TM, words, st);
        if (m <= 8) return launch_t<6, 8, -1, 0, 0>(B, mc, S[2], TM, words, st);
        if (m <= 16) return launch_t<6, 16, -1, 0, 0>(B, mc, S[2], TM, words, st);
        return launch_t<6, 24, -1, 0, 0>(B, mc, S[2], TM, words, st);
    }
    for (int d = 0; d < 2; ++d) {
        if (S[d].total == 0) continue;
        PtMaps& TM = pp_maps(B, nch, S[d], G);
        const cudaStream_t sd = d == 1 && st2 ? st2 : st;
        const pgm_status r = nch == 2 ? launch_dir<2>(B, mc, S[d], G[d], TM, G[d].words, sd)
                                      : launch_dir<6>(B, mc, S[d], G[d], TM, G[d].words, sd);
        if (r != PGM_OK) return r;
        ++*nlaunch;
    }
    return PGM_OK;
}

pgm_status launch_cost_tile(const LvlBatch& B, const MatchConst& mc, int nch, bool* handled,
                            cudaStream_t st) {
    *handled = false;
    int tiles = 0, words = 0, maxw = 0;
    for (int k = 0; k < B.n; ++k)
        for (int d = 0; d < 2; ++d) {
            const DirLvl& D = B.d[k][d];
            const int t = ((D.nx + PT_TW - 1) / PT_TW) * ((D.ny + PT_TH - 1) / PT_TH);
            if (t > tiles) tiles = t;
            const PtGeom g = pt_geom(nch, D.P, mc.sigma, mc.rs_W, mc.slack);
            if (g.words > words) words = g.words;
            if (D.P * g.wprp > maxw) maxw = D.P * g.wprp;
        }
    const int smem_bytes = words * 4;
    if (smem_bytes > 160 * 1024 || (maxw + 31) / 32 > 24 || !pt_offsets_fit(B, nch, mc))
        return PGM_OK;
    *handled = true;
    if (tiles == 0) return PGM_OK;
    return nch == 2 ? launch_c<2>(B, mc, tiles, smem_bytes, st)
                    : launch_c<6>(B, mc, tiles, smem_bytes, st);
}

}  // namespace pgm
