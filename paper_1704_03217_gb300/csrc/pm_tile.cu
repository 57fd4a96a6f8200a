// pm_tile.cu -- one checkerboard colour phase of propagation (Eq. 4) and
// limited random search (Eq. 5), squared-L2 cost, on seed tiles staged in
// shared memory.
//
// A CTA owns an 8 x 8 tile of lattice seeds; the 32 seeds of the current
// colour update, one warp per seed at a time.  Before any cost is computed the
// CTA stages into shared memory
//   - the reference region covering all patches of the tile, in the
//     split-byte form (a = 128 a_h + a_l) that the dp2a cross products use;
//   - a fixed-size target window around the tile's median displacement,
//     wide enough for the random-search square plus a slack.
// Both are staged in unclamped pixel coordinates with the image border
// replicated, so the inner loop needs no border tests.
//
// Patch rows are padded to a multiple of 4 words (the padding words carry a
// zero reference, so they add nothing), which makes every staged row 16-byte
// aligned, and the shared row pitch is congruent to the padded row modulo 32:
// the 32 consecutive words of a flattened patch that a warp reads fall in 32
// different banks.  A candidate whose padded patch is not inside the window is
// scored from global memory instead.  The cost of a candidate is
//   D = sum |a|^2 + sum |b|^2 - 2 sum <a, b>,
// exact in integers, with sum |a|^2 per seed and sum |b|^2 per target pixel
// computed by other kernels of the same visit.
#include <limits.h>

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
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(
                     (unsigned)__cvta_generic_to_shared(dst)), "l"(src) : "memory");
}
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
// (pitch sp), replicating the border: asynchronous 4-byte copies, one warp
// per row, lanes across it; completion by cp_async_wait_all.
template <int WPP>
__device__ __forceinline__ void stage(uint32_t* dst, int sp, const uint32_t* src, int pw, int iw,
                                      int ih, int x0, int y0, int w, int rows) {
    const int lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    const int wwords = w * WPP;
    if (x0 >= 0 && y0 >= 0 && x0 + w <= iw && y0 + rows <= ih) {
        for (int row = threadIdx.x >> 5; row < rows; row += nwarp) {
            const uint32_t* s = src + (size_t)(y0 + row) * pw + (size_t)x0 * WPP;
            uint32_t* d = dst + row * sp;
            for (int wd = lane; wd < wwords; wd += 32) cp_async4(d + wd, s + wd);
        }
    } else {
        for (int row = threadIdx.x >> 5; row < rows; row += nwarp) {
            const uint32_t* srow = src + (size_t)clampi(y0 + row, 0, ih - 1) * pw;
            for (int wd = lane; wd < wwords; wd += 32) {
                const int pix = wd / WPP, wi = wd - pix * WPP;      // WPP is 1 or 3
                cp_async4(dst + row * sp + wd, srow + (size_t)clampi(x0 + pix, 0, iw - 1) * WPP + wi);
            }
        }
    }
}

// Lane-owned words of the flattened (padded) patch: word k = lane + 32 m has
// row k / wprp and column k % wprp; walked incrementally (no division).
// byte offsets of the lane's words packed two per register (each < 2^16)
template <int M>
struct Offs {
    unsigned p[(M + 1) / 2];
    __device__ __forceinline__ unsigned at(int m) const {
        return (m & 1) ? (p[m >> 1] >> 16) : (p[m >> 1] & 0xffffu);
    }
};

// Lane-owned words of the flattened patch: word k = lane + 32 m has row
// k / wpr and column k % wpr; walked incrementally (no division).
template <int M>
__device__ __forceinline__ void patch_walk(int lane, int wpr, int nw, int sp, Offs<M>& off,
                                           unsigned& vmask) {
    int row = 0, col = lane;
    while (col >= wpr) { col -= wpr; ++row; }
    vmask = 0;
#pragma unroll
    for (int m = 0; m < (M + 1) / 2; ++m) off.p[m] = 0;
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const int k = lane + 32 * m;
        const unsigned o = k < nw ? 4u * (unsigned)(row * sp + col) : 0u;   // byte offset
        off.p[m >> 1] |= o << (16 * (m & 1));
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

struct TileCtx {
    const uint32_t* s_ref; const uint32_t* s_tw; const unsigned long long* s_sb;
    const int* s_seed; const int* s_u; const int (*s_nb)[2]; const unsigned char* s_f;
    const unsigned long long* s_cost; const unsigned long long* s_sa; const uint4* s_rnd;
    int i0, j0, rx0, wx0, wy0;
    bool use_win;
    int sig, h, P, nw, sx, sy, lane, warp;
};

constexpr int NO_CAND = INT_MIN;            // no propagated candidate

// The seeds of one tile and colour, one warp each.  M = number of 32-word
// groups of the flattened patch: no per-group test is needed, the words of
// the last group that lie past the patch read a valid shared word and
// multiply it by a zero reference.
template <int NCH, int M, bool EXACT>
__device__ __forceinline__ void seeds(const LvlBatch& B, const MatchConst& mc, const DirLvl& D,
                                      const PtGeom& G, const TileCtx& T) {
    constexpr int WPP = NCH / 2;
    const int lane = T.lane, P = T.P, h = T.h, sig = T.sig;
    const int pair = blockIdx.z, dir = blockIdx.y;
    const unsigned a_ref = (unsigned)__cvta_generic_to_shared(T.s_ref);
    const unsigned a_tw = (unsigned)__cvta_generic_to_shared(T.s_tw);
    const unsigned a_sb = (unsigned)__cvta_generic_to_shared(T.s_sb);
    Offs<M> off;                            // byte offsets of the lane's patch words
    unsigned vmask;                         // bit m: word lane + 32 m is a real patch word
    patch_walk<M>(lane, G.wprp, T.nw, G.sp, off, vmask);

    for (int a = T.warp; a < PT_NACT; a += 8) {
        const int s = T.s_seed[a];
        if (s < 0) continue;
        const int j = T.j0 + a / (PT_TW / 2);
        const int i = T.i0 + 2 * (a % (PT_TW / 2)) + ((j + mc.colour) & 1);
        const int px = mc.c + sig * i, py = mc.c + sig * j;
        const uint8_t f0 = T.s_f[a];
        bool have = f0 & F_VALID;
        int32_t bu = T.s_u[a];
        unsigned long long bc = have ? T.s_cost[a] : INF;
        const int32_t u_in = bu;
        const bool have_in = have;
        const unsigned long long sa = T.s_sa[a];

        int b[M];
        bool loaded = false;
        unsigned n_eval = 0, n_glob = 0;
        auto score = [&](int qx, int qy) -> unsigned long long {
            if (!loaded) {
                const unsigned rbase =
                    a_ref + 4u * (unsigned)(sig * (j - T.j0) * G.sp + (mc.c + sig * i - h - T.rx0) * WPP);
#pragma unroll
                for (int m = 0; m < M; ++m) {
                    b[m] = lds32(rbase + off.at(m));
                    // words past the patch read a valid shared word; zero their weight
                    if (!EXACT || m == M - 1) b[m] &= (int)(0u - ((vmask >> m) & 1u));
                }
                loaded = true;
            }
            ++n_eval;
            return tile_cost<NCH, M>(b, off, D, G, a_tw, a_sb, T.use_win, T.wx0, T.wy0, sa, qx, qy,
                                     lane, n_glob);
        };

        // one loop over the candidate sequence (a single inlined cost site):
        // c = 0, 1: propagated matches (Eq. 4); c >= 2: random search (Eq. 5)
        // around the match held after propagation
        int ux0 = 0, uy0 = 0;
        uint4 r = T.s_rnd[a];
        const int g = mc.rs_grid;             // PGM-C3/G3: level-0 search on a grid only
        const int K = (B.level == 0 && g > 0 && !(px % g == g / 2 && py % g == g / 2)) ? 0 : mc.K;
#pragma unroll 1
        for (int c = 0; c < 2 + K; ++c) {
            int32_t cu;
            int qx, qy;
            if (c < 2) {
                cu = T.s_nb[a][c];
                if (cu == NO_CAND || (have && cu == bu)) continue;
                qx = px + lo16((uint32_t)cu);
                qy = py + hi16((uint32_t)cu);
            } else {
                if (!have) break;
                const int k = c - 2;
                if (k == 0) { ux0 = lo16((uint32_t)bu); uy0 = hi16((uint32_t)bu); }
                if (k > 0 && (k & 1) == 0)
                    r = philox(make_uint4((uint32_t)s,
                                          ((uint32_t)B.visit << 16) | ((uint32_t)dir << 15) | (uint32_t)mc.t,
                                          ((uint32_t)B.level << 16) | (uint32_t)(k >> 1),
                                          B.stream_id[pair]),
                               mc.key0, mc.key1);
                const uint32_t rx = (k & 1) ? r.z : r.x, ry = (k & 1) ? r.w : r.y;
                const int dx = rs_off(rx, k, mc.rs_W, mc.rs_mode), dy = rs_off(ry, k, mc.rs_W, mc.rs_mode);
                if (dx == 0 && dy == 0) continue;
                qx = px + ux0 + dx;                 // tested before packing into 16 bits
                qy = py + uy0 + dy;
                cu = pack_u(ux0 + dx, uy0 + dy);
            }
            if (!inside(D, qx, qy)) continue;
            const unsigned long long cst = score(qx, qy);
            if (cst < bc) { bc = cst; bu = cu; have = true; }
        }
        if (lane == 0) {
            if (n_eval) atomicAdd(B.evals[pair] + dir, (unsigned long long)n_eval);
            if (n_glob) atomicAdd(B.evals[pair] + 6 + dir, (unsigned long long)n_glob);
            if (have && (bu != u_in || !have_in)) {
                D.u[s] = bu;
                D.cost[s] = bc;
                D.flags[s] = f0 | F_VALID;
            }
        }
    }
}

template <int NCH>
__global__ void __launch_bounds__(256, 3)
k_pm_t(const __grid_constant__ LvlBatch B, const MatchConst mc) {
    constexpr int WPP = NCH / 2;
    extern __shared__ __align__(16) uint32_t sm[];
    __shared__ int s_seed[PT_NACT];         // seed index, -1 if none
    __shared__ int s_u[PT_NACT];            // current displacement
    __shared__ int s_nb[PT_NACT][2];        // propagated displacement, or the sentinel
    __shared__ unsigned char s_f[PT_NACT];  // flags
    __shared__ unsigned long long s_cost[PT_NACT], s_sa[PT_NACT];
    __shared__ uint4 s_rnd[PT_NACT];        // Philox block 0 of the seed (random search)
    __shared__ int s_med[2];

    const int pair = blockIdx.z, dir = blockIdx.y;
    const DirLvl& D = B.d[pair][dir];
    const int tiles_x = (D.nx + PT_TW - 1) / PT_TW, tiles_y = (D.ny + PT_TH - 1) / PT_TH;
    if ((int)blockIdx.x >= tiles_x * tiles_y) return;
    const int i0 = ((int)blockIdx.x % tiles_x) * PT_TW, j0 = ((int)blockIdx.x / tiles_x) * PT_TH;
    const int P = D.P, h = P / 2;
    const int sig = mc.sigma;
    const PtGeom G = pt_geom(NCH, P, sig, mc.rs_W, mc.slack);
    const int nw = P * G.wprp;
    uint32_t* s_ref = sm;
    uint32_t* s_tw = sm + G.ref_h * G.sp;
    const int t4 = mc.t & 3;
    const int sx = (t4 == 0 || t4 == 3) ? 1 : -1, sy = (t4 == 0 || t4 == 2) ? 1 : -1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    // ---- C1: start staging the reference region (independent of the seeds)
    const int rx0 = mc.c + sig * i0 - h, ry0 = mc.c + sig * j0 - h;
    stage<WPP>(s_ref, G.sp, D.ref_split, D.ref_pitch >> 1, D.rw, D.rh, rx0, ry0, G.ref_w, G.ref_h);

    // ---- A: the active seeds (warp 0, one lane per seed); their first
    // Philox block is drawn by warp 1 meanwhile
    if (warp == 1 && mc.K > 0) {
        const int a = lane, j = j0 + a / (PT_TW / 2);
        const int i = i0 + 2 * (a % (PT_TW / 2)) + ((j + mc.colour) & 1);
        if (i < D.nx && j < D.ny)
            s_rnd[a] = philox(make_uint4((uint32_t)(j * D.nx + i),
                                         ((uint32_t)B.visit << 16) | ((uint32_t)dir << 15) | (uint32_t)mc.t,
                                         ((uint32_t)B.level << 16), B.stream_id[pair]),
                              mc.key0, mc.key1);
    }
    if (warp == 0) {
        const int a = lane, r = a / (PT_TW / 2), k = a % (PT_TW / 2);
        const int j = j0 + r, i = i0 + 2 * k + ((j + mc.colour) & 1);
        int s = -1, u = 0, f = 0;
        if (i < D.nx && j < D.ny) {
            s = j * D.nx + i;
            const int ni = i - sx, nj = j - sy;
            const bool okx = ni >= 0 && ni < D.nx, oky = nj >= 0 && nj < D.ny;
            const int sn0 = okx ? j * D.nx + ni : s, sn1 = oky ? nj * D.nx + i : s;
            // independent loads, issued together
            f = D.flags[s];
            u = D.u[s];
            const unsigned long long cst = D.cost[s], sa2 = D.sa2[s];
            const int f0 = D.flags[sn0], f1 = D.flags[sn1];
            const int u0 = D.u[sn0], u1 = D.u[sn1];
            s_cost[a] = cst;
            s_sa[a] = sa2;
            s_nb[a][0] = (okx && (f0 & F_VALID)) ? u0 : NO_CAND;
            s_nb[a][1] = (oky && (f1 & F_VALID)) ? u1 : NO_CAND;
        }
        s_seed[a] = s;
        s_u[a] = u;
        s_f[a] = (unsigned char)f;
        // median of the valid current displacements: rank by (value, lane)
        const bool v = s >= 0 && (f & F_VALID);
        const unsigned vm = __ballot_sync(FULL, v);
        const int nv = __popc(vm);
        const int ux = lo16((uint32_t)u), uy = hi16((uint32_t)u);
        int rx = 0, ry = 0;
        for (int o = 0; o < 32; ++o) {
            const int ox = __shfl_sync(FULL, ux, o), oy = __shfl_sync(FULL, uy, o);
            if ((vm >> o) & 1) {
                rx += ox < ux || (ox == ux && o < lane);
                ry += oy < uy || (oy == uy && o < lane);
            }
        }
        if (lane == 0) { s_med[0] = INT_MIN; s_med[1] = INT_MIN; }
        __syncwarp();
        if (v && rx == nv / 2) s_med[0] = ux;
        if (v && ry == nv / 2) s_med[1] = uy;
    }
    __syncthreads();

    // ---- B: window around the median match (unclamped pixel coordinates)
    const int rho = max(1, mc.rs_W);
    const bool use_win = s_med[0] != INT_MIN;
    const int wx0 = use_win ? mc.c + sig * i0 - h + s_med[0] - rho - mc.slack : 0;
    const int wy0 = use_win ? mc.c + sig * j0 - h + s_med[1] - rho - mc.slack : 0;

    // ---- C2: stage the window and its sums of |b|^2
    unsigned long long* s_sb = reinterpret_cast<unsigned long long*>(
        sm + ((G.sp * (G.ref_h + G.win_h) + 1) & ~1));
    if (use_win) {
        stage<WPP>(s_tw, G.sp, reinterpret_cast<const uint32_t*>(D.tgt), D.tgt_pitch >> 1, D.tw,
                   D.th, wx0, wy0, G.win_w, G.win_h);
        // sum |b|^2 of every centre whose patch lies in the window (centres
        // outside the image are never scored; their entries are don't-care)
        const int cx0 = wx0 + h, cy0 = wy0 + h;
        for (int row = warp; row < G.ch; row += 8) {
            const unsigned long long* srow = D.sb2 + (size_t)clampi(cy0 + row, 0, D.th - 1) * D.tw;
            for (int col = lane; col < G.cw; col += 32)
                cp_async8(s_sb + row * G.cw + col, srow + clampi(cx0 + col, 0, D.tw - 1));
        }
    }
    cp_async_wait_all();
    __syncthreads();

    // ---- D: one warp per active seed, specialised on the exact number of
    // 32-word groups of this direction's patch
    TileCtx T{s_ref, s_tw, s_sb, s_seed, s_u, s_nb, s_f, s_cost, s_sa, s_rnd,
              i0, j0, rx0, wx0, wy0, use_win, sig, h, P, nw, sx, sy, lane, warp};
    const int groups = (nw + 31) / 32;
    // exact group counts of the common patch sides (6 ch: P 8, 11, 15, 16;
    // 2 ch: P 8, 11, 15/16) need only the last group masked
#define PGM_SEEDS(MM, EX) seeds<NCH, MM, EX>(B, mc, D, G, T)
    if (NCH == 6) {
        if (groups == 6) PGM_SEEDS(6, true);
        else if (groups == 12) PGM_SEEDS(12, true);
        else if (groups == 22) PGM_SEEDS(22, true);
        else if (groups == 24) PGM_SEEDS(24, true);
        else if (groups <= 4) PGM_SEEDS(4, false);
        else if (groups <= 8) PGM_SEEDS(8, false);
        else if (groups <= 16) PGM_SEEDS(16, false);
        else PGM_SEEDS(24, false);
    } else {
        if (groups == 2) PGM_SEEDS(2, true);
        else if (groups == 4) PGM_SEEDS(4, true);
        else if (groups == 8) PGM_SEEDS(8, true);
        else if (groups <= 2) PGM_SEEDS(2, false);
        else if (groups <= 4) PGM_SEEDS(4, false);
        else PGM_SEEDS(8, false);
    }
#undef PGM_SEEDS
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
    extern __shared__ __align__(16) uint32_t sm[];
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
    stage<WPP>(s_ref, G.sp, D.ref_split, D.ref_pitch >> 1, D.rw, D.rh, rx0, ry0, G.ref_w, G.ref_h);

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
                   D.th, wx0, wy0, G.win_w, G.win_h);
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

template <int NCH>
pgm_status launch_c(const LvlBatch& B, const MatchConst& mc, int tiles, int smem_bytes,
                    cudaStream_t st) {
    static int configured = 0;
    if (configured < smem_bytes) {
        if (cudaFuncSetAttribute(k_cost_t<NCH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem_bytes) != cudaSuccess) return PGM_ERR_CUDA;
        configured = smem_bytes;
    }
    k_cost_t<NCH><<<dim3(tiles, 2, B.n), 256, smem_bytes, st>>>(B, mc);
    return cudaGetLastError() == cudaSuccess ? PGM_OK : PGM_ERR_CUDA;
}

template <int NCH>
pgm_status launch_t(const LvlBatch& B, const MatchConst& mc, int tiles, int smem_bytes,
                    cudaStream_t st) {
    static int configured = 0;                 // opt-in above 48 KB once per instantiation
    if (configured < smem_bytes) {
        if (cudaFuncSetAttribute(k_pm_t<NCH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem_bytes) != cudaSuccess) return PGM_ERR_CUDA;
        configured = smem_bytes;
    }
    k_pm_t<NCH><<<dim3(tiles, 2, B.n), 256, smem_bytes, st>>>(B, mc);
    return cudaGetLastError() == cudaSuccess ? PGM_OK : PGM_ERR_CUDA;
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

// *handled = false when the staged tile would not fit in shared memory; the
// caller then uses the per-seed kernel.
pgm_status launch_pm_tile(const LvlBatch& B, const MatchConst& mc, int nch, int maxP,
                          bool* handled, cudaStream_t st) {
    (void)maxP;
    *handled = false;
    int tiles = 0, words = 0, maxw = 0;
    for (int k = 0; k < B.n; ++k)
        for (int d = 0; d < 2; ++d) {
            const DirLvl& D = B.d[k][d];
            const int t = ((D.nx + PT_TW - 1) / PT_TW) * ((D.ny + PT_TH - 1) / PT_TH);
            if (t > tiles) tiles = t;
            const PtGeom g = pt_geom(nch, D.P, mc.sigma, mc.rs_W, mc.slack);
            if (g.words > words) words = g.words;
            const int nwp = D.P * g.wprp;
            if (nwp > maxw) maxw = nwp;
        }
    const int smem_bytes = words * 4;
    if (smem_bytes > 160 * 1024 || !pt_offsets_fit(B, nch, mc)) return PGM_OK;
    *handled = true;
    if (tiles == 0) return PGM_OK;
    if ((maxw + 31) / 32 > 24) return PGM_ERR_UNSUPPORTED;
    return nch == 2 ? launch_t<2>(B, mc, tiles, smem_bytes, st)
                    : launch_t<6>(B, mc, tiles, smem_bytes, st);
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
