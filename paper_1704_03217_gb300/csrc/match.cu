// match.cu -- the matching kernels of one pyramid level (Sec. III-B, III-D).
//
//   k_init      exhaustive nearest-neighbour initialisation at the coarsest
//               level (the exact field the KD-tree init of Sec. III-D
//               approximates); one CTA per seed, threads over targets.
//   k_cost      D_r (Eq. 3) of every initialised seed's current match.
//   k_pm        one checkerboard colour phase of propagation (Eq. 4) and
//               limited random search (Eq. 5); one warp per seed.
//   k_consist   forward-backward consistency + outlier-record update (Eq. 6).
//   k_transfer  field (Eq. 7) and outlier-record (Eq. 8) propagation.
//
// All arithmetic is integer: descriptors are int16, a patch distance is an
// exact uint64 sum, so the result does not depend on the reduction order.
#include "match_common.cuh"

namespace pgm {
namespace {

// ------------------------------------------------------------------
// Warp-cooperative patch distance.  Lane l holds patch pixels l, l+32, ...
// (row-major in the P x P patch) of the reference, NCH channels each.
template <int NCH, int PPL>
struct Ref {
    int a[PPL][NCH];
    int ox[PPL], oy[PPL];
};

template <int NCH, int PPL>
__device__ __forceinline__ void load_ref(Ref<NCH, PPL>& R, const DirLvl& D, int px, int py,
                                         int lane) {
    const int P = D.P, h = P / 2;
#pragma unroll
    for (int m = 0; m < PPL; ++m) {
        int k = lane + 32 * m;
        int kk = k < P * P ? k : 0;
        R.ox[m] = kk % P - h;
        R.oy[m] = kk / P - h;
        int x = clampi(px + R.ox[m], 0, D.rw - 1), y = clampi(py + R.oy[m], 0, D.rh - 1);
        const uint32_t* w = reinterpret_cast<const uint32_t*>(D.ref + (size_t)y * D.ref_pitch +
                                                              (size_t)x * 2 * px_words(NCH));
#pragma unroll
        for (int c = 0; c < NCH / 2; ++c) {
            uint32_t v = (k < P * P) ? __ldg(w + c) : 0u;
            R.a[m][2 * c] = lo16(v);
            R.a[m][2 * c + 1] = hi16(v);
        }
    }
}

template <int NCH, int PPL, int NORM>
__device__ __forceinline__ unsigned long long warp_cost(const Ref<NCH, PPL>& R, const DirLvl& D,
                                                        int qx, int qy, int lane) {
    const int P2 = D.P * D.P;
    unsigned long long acc = 0;
#pragma unroll
    for (int m = 0; m < PPL; ++m) {
        if (lane + 32 * m < P2) {
            int x = clampi(qx + R.ox[m], 0, D.tw - 1), y = clampi(qy + R.oy[m], 0, D.th - 1);
            const uint32_t* w = reinterpret_cast<const uint32_t*>(
                D.tgt + (size_t)y * D.tgt_pitch + (size_t)x * 2 * px_words(NCH));
            uint32_t s = 0;
#pragma unroll
            for (int c = 0; c < NCH / 2; ++c) {
                uint32_t v = __ldg(w + c);
                int d0 = lo16(v) - R.a[m][2 * c], d1 = hi16(v) - R.a[m][2 * c + 1];
                if (NORM == PGM_L2SQ) s += (uint32_t)(d0 * d0) + (uint32_t)(d1 * d1);
                else s += (uint32_t)(abs(d0) + abs(d1));
            }
            acc += s;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
    return acc;
}


// ------------------------------------------------------------------
// Squared-L2 path.  Over integers Eq. 3 splits exactly into
//   D = sum |a|^2 + sum |b|^2 - 2 sum <a, b>
// (a: reference patch, b: target patch, borders replicated in each image).
// sum |a|^2 is computed once per seed (k_cost_x), sum |b|^2 once per target
// pixel (box filter, k_box_h / k_box_v), so a candidate needs only the cross
// term.  Each reference value a (|a| <= 12240) is split into two signed bytes
// a = 128 a_h + a_l, a_l in [-64, 63], a_h in [-96, 96], so one dp2a
// instruction multiplies a whole 32-bit target word (two int16 values) by
// the low bytes and one by the high bytes.  Lane partial sums and their warp
// totals stay below 2^31 for patches up to 16 x 16 x 6 values:
//   |sum b a_l| <= 1536 * 12240 * 64 < 1.3e9,  |sum b a_h| <= 1536 * 12240 * 96 < 1.9e9.

// Box filter of N(x, y) = sum_c G_c(x, y)^2 over the P x P patch with
// replicated borders (the sums |a|^2 and |b|^2 of Eq. 3 expanded), exact in
// uint64 (N itself fits 32 bits: 6 values of at most 24480^2).  A CTA makes a
// BOX_TW x BOX_TH block of one map: N over the block and a halo of P / 2
// (clamped coordinates) into shared memory, then running row sums over runs
// of BOX_RUN outputs, then running column sums the same way.
// blockIdx.y = 2 * direction + (0: target image -> sb2, 1: reference ->
// sa2img); blockIdx.x = block of that map (the grid covers the largest map).
constexpr int BOX_TW = 64, BOX_TH = 32, BOX_H = MAXP / 2, BOX_RUN = 8;
template <int NCH>
__global__ void __launch_bounds__(256) k_box(const __grid_constant__ LvlBatch B) {
    __shared__ uint32_t sN[BOX_TH + 2 * BOX_H][BOX_TW + 2 * BOX_H];
    __shared__ unsigned long long sR[BOX_TH + 2 * BOX_H][BOX_TW];
    const DirLvl& D = B.d[blockIdx.z][blockIdx.y >> 1];
    const bool ref = blockIdx.y & 1;
    const int w = ref ? D.rw : D.tw, hh = ref ? D.rh : D.th, P = D.P, h = P / 2;
    const int tx = (w + BOX_TW - 1) / BOX_TW, ty = (hh + BOX_TH - 1) / BOX_TH;
    if ((int)blockIdx.x >= tx * ty) return;
    const int x0 = ((int)blockIdx.x % tx) * BOX_TW, y0 = ((int)blockIdx.x / tx) * BOX_TH;
    const int16_t* img = ref ? D.ref : D.tgt;
    const int pitch = ref ? D.ref_pitch : D.tgt_pitch;
    const int iw = BOX_TW + P - 1, ih = BOX_TH + P - 1;
    // a warp per row, lanes along it
    for (int r = threadIdx.x >> 5; r < ih; r += blockDim.x >> 5) {
        const uint32_t* row = reinterpret_cast<const uint32_t*>(
            img + (size_t)clampi(y0 - h + r, 0, hh - 1) * pitch);
        for (int c = threadIdx.x & 31; c < iw; c += 32) {
            const uint32_t* px = row + (size_t)clampi(x0 - h + c, 0, w - 1) * px_words(NCH);
            uint32_t n = 0;
#pragma unroll
            for (int c2 = 0; c2 < NCH / 2; ++c2) {
                const uint32_t v = __ldg(px + c2);
                const int a = lo16(v), b = hi16(v);
                n += (uint32_t)(a * a) + (uint32_t)(b * b);
            }
            sN[r][c] = n;
        }
    }
    __syncthreads();
    // row sums: thread -> (row, run of BOX_RUN outputs); consecutive threads
    // take consecutive runs of one row
    constexpr int RUNS_X = BOX_TW / BOX_RUN;
    for (int e = threadIdx.x; e < ih * RUNS_X; e += blockDim.x) {
        const int r = e / RUNS_X, c0 = (e - r * RUNS_X) * BOX_RUN;
        unsigned long long s = 0;
        for (int o = 0; o < P; ++o) s += sN[r][c0 + o];
        sR[r][c0] = s;
#pragma unroll
        for (int k = 1; k < BOX_RUN; ++k) {
            s += (unsigned long long)sN[r][c0 + k + P - 1] - sN[r][c0 + k - 1];
            sR[r][c0 + k] = s;
        }
    }
    __syncthreads();
    // column sums: thread -> (column, run of BOX_RUN rows); a warp covers 32
    // consecutive columns, so the stores of one row are coalesced
    unsigned long long* out = ref ? D.sa2img : D.sb2;
    const int opitch = ref ? w : D.sbp;
    constexpr int RUNS_Y = BOX_TH / BOX_RUN;
    for (int e = threadIdx.x; e < BOX_TW * RUNS_Y; e += blockDim.x) {
        const int c = e % BOX_TW, r0 = (e / BOX_TW) * BOX_RUN, x = x0 + c;
        unsigned long long s = 0;
        for (int o = 0; o < P; ++o) s += sR[r0 + o][c];
#pragma unroll
        for (int k = 0; k < BOX_RUN; ++k) {
            if (k > 0) s += sR[r0 + k + P - 1][c] - sR[r0 + k - 1][c];
            const int y = y0 + r0 + k;
            if (x < w && y < hh) out[(size_t)y * opitch + x] = s;
        }
    }
}

// Lane l owns words l, l + 32, ... of the P x P x NCH patch, flattened row by
// row (a patch row is P * NCH / 2 consecutive 32-bit words of the image row).
// Word offsets of the flattened patch inside an interior target patch; the
// same for every warp of a block (one pair, one direction), kept in shared
// memory: s_off[k] for k = lane + 32 m.
template <int NCH, int MMAX>
__device__ __forceinline__ void fill_offsets(int* s_off, const DirLvl& D) {
    constexpr int WPP = NCH / 2;
    const int wpr = D.P * WPP, nw = D.P * wpr, pitchw = D.tgt_pitch >> 1;
    for (int k = threadIdx.x; k < 32 * MMAX; k += blockDim.x) {
        const int row = k / wpr, col = k - row * wpr, pix = col / WPP, wi = col - pix * WPP;
        s_off[k] = k < nw ? row * pitchw + pix * px_words(NCH) + wi : 0;
    }
}

// Loads this lane's reference words; returns the lane's partial sum of a^2
// when WANT_SA2.
template <int NCH, int MMAX, bool WANT_SA2>
__device__ __forceinline__ unsigned long long xload_ref(XRef<MMAX>& R, const DirLvl& D, int px,
                                                        int py, int lane) {
    constexpr int WPP = NCH / 2;
    const int P = D.P, h = P / 2, wpr = P * WPP, nw = P * wpr;
    const int rpitchw = D.ref_pitch >> 1;
    const uint32_t* ref32 = reinterpret_cast<const uint32_t*>(D.ref);
    unsigned long long sa = 0;
#pragma unroll
    for (int m = 0; m < MMAX; ++m) {
        const int k = lane + 32 * m;
        R.b[m] = 0;
        if (k < nw) {
            const int row = k / wpr, col = k - row * wpr;
            const int pix = col / WPP, wi = col - pix * WPP;
            const int x = clampi(px - h + pix, 0, D.rw - 1), y = clampi(py - h + row, 0, D.rh - 1);
            const uint32_t v = __ldg(ref32 + (size_t)y * rpitchw + (size_t)x * px_words(NCH) + wi);
            const int a0 = lo16(v), a1 = hi16(v);
            R.b[m] = split_bytes(a0, a1);
            if (WANT_SA2) sa += (uint32_t)(a0 * a0) + (uint32_t)(a1 * a1);
        }
    }
    return sa;
}

// sum <a, b> over the patch at target centre (qx, qy), warp-uniform result
template <int NCH, int MMAX>
__device__ __forceinline__ long long xcross(const XRef<MMAX>& R, const int* s_off, const DirLvl& D,
                                            int qx, int qy, int lane) {
    constexpr int WPP = NCH / 2;
    const int P = D.P, h = P / 2, wpr = P * WPP, nw = P * wpr;
    const int pitchw = D.tgt_pitch >> 1;
    const uint32_t* t32 = reinterpret_cast<const uint32_t*>(D.tgt);
    const int x0 = qx - h, y0 = qy - h;
    int sl = 0, sh = 0;
    if (x0 >= 0 && y0 >= 0 && x0 + P <= D.tw && y0 + P <= D.th) {
        const uint32_t* base = t32 + (size_t)y0 * pitchw + (size_t)x0 * px_words(NCH);
        constexpr int CH = MMAX < 8 ? MMAX : 8;      // loads in flight per chunk
#pragma unroll
        for (int m0 = 0; m0 < MMAX; m0 += CH) {
            uint32_t v[CH];
#pragma unroll
            for (int c = 0; c < CH; ++c)
                if (32 * (m0 + c) < nw) v[c] = __ldg(base + s_off[lane + 32 * (m0 + c)]);
#pragma unroll
            for (int c = 0; c < CH; ++c)
                if (32 * (m0 + c) < nw) {
                    sl = __dp2a_lo((int)v[c], R.b[m0 + c], sl);
                    sh = __dp2a_hi((int)v[c], R.b[m0 + c], sh);
                }
        }
    } else {                                   // patch crosses the border: replicate
#pragma unroll
        for (int m = 0; m < MMAX; ++m)
            if (32 * m < nw) {
                const int k = lane + 32 * m;
                const int row = k / wpr, col = k - row * wpr;
                const int pix = col / WPP, wi = col - pix * WPP;
                const int x = clampi(x0 + pix, 0, D.tw - 1), y = clampi(y0 + row, 0, D.th - 1);
                const uint32_t v = __ldg(t32 + (size_t)y * pitchw + (size_t)x * px_words(NCH) + wi);
                sl = __dp2a_lo((int)v, R.b[m], sl);
                sh = __dp2a_hi((int)v, R.b[m], sh);
            }
    }
    sl = __reduce_add_sync(FULL, sl);
    sh = __reduce_add_sync(FULL, sh);
    return (long long)sh * 128 + (long long)sl;
}

template <int NCH, int MMAX>
__global__ void __launch_bounds__(256, 3) k_cost_x(const __grid_constant__ LvlBatch B, const MatchConst mc) {
    const int pair = blockIdx.z, dir = blockIdx.y;
    const DirLvl& D = B.d[pair][dir];
    __shared__ int s_off[32 * MMAX];
    fill_offsets<NCH, MMAX>(s_off, D);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int s = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (s >= D.nx * D.ny) return;
    const int i = s % D.nx, j = s / D.nx;
    const int px = mc.c + mc.sigma * i, py = mc.c + mc.sigma * j;
    XRef<MMAX> R;
    unsigned long long sa = xload_ref<NCH, MMAX, true>(R, D, px, py, lane);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sa += __shfl_xor_sync(FULL, sa, o);
    if (lane == 0) D.sa2[s] = sa;                 // needed by every seed, valid or not
    const uint8_t f = D.flags[s];
    if (!(f & F_VALID)) return;
    const int32_t u = D.u[s];
    const int qx = px + lo16(u), qy = py + hi16(u);
    if (!inside(D, qx, qy)) {
        if (lane == 0) D.flags[s] = f & ~F_VALID;
        return;
    }
    const unsigned long long sb = D.sb2[(size_t)qy * D.sbp + qx];
    const long long cr = xcross<NCH, MMAX>(R, s_off, D, qx, qy, lane);
    if (lane == 0) {
        D.cost[s] = xcost(sa, sb, cr);
        atomicAdd(B.evals[pair] + 2 + dir, 1ull);
    }
}

template <int NCH, int MMAX>
__global__ void __launch_bounds__(256, 3) k_pm_x(const __grid_constant__ LvlBatch B, const MatchConst mc) {
    const int pair = blockIdx.z, dir = blockIdx.y;
    const DirLvl& D = B.d[pair][dir];
    __shared__ int s_off[32 * MMAX];
    fill_offsets<NCH, MMAX>(s_off, D);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int wid = blockIdx.x * 8 + (threadIdx.x >> 5);
    const int hw = (D.nx + 1) >> 1;
    if (wid >= hw * D.ny) return;
    const int j = wid / hw;
    const int i = 2 * (wid - j * hw) + ((j + mc.colour) & 1);
    if (i >= D.nx) return;
    const int s = j * D.nx + i;
    const int px = mc.c + mc.sigma * i, py = mc.c + mc.sigma * j;

    const uint8_t f0 = D.flags[s];
    bool have = f0 & F_VALID;
    int32_t bu = D.u[s];
    unsigned long long bc = have ? D.cost[s] : INF;
    const int32_t u_in = bu;
    const bool have_in = have;
    const unsigned long long sa = D.sa2[s];

    const int t4 = mc.t & 3;
    const int sx = (t4 == 0 || t4 == 3) ? 1 : -1;
    const int sy = (t4 == 0 || t4 == 2) ? 1 : -1;

    XRef<MMAX> R;
    bool loaded = false;
    unsigned n_eval = 0;
#pragma unroll
    for (int k = 0; k < 2; ++k) {             // Eq. 4
        const int ni = k == 0 ? i - sx : i, nj = k == 0 ? j : j - sy;
        if (ni < 0 || nj < 0 || ni >= D.nx || nj >= D.ny) continue;
        const int ns = nj * D.nx + ni;
        if (!(D.flags[ns] & F_VALID)) continue;
        const int32_t cu = D.u[ns];
        if (have && cu == bu) continue;
        const int qx = px + lo16(cu), qy = py + hi16(cu);
        if (!inside(D, qx, qy)) continue;
        const unsigned long long sb = D.sb2[(size_t)qy * D.sbp + qx];
        if (!loaded) { xload_ref<NCH, MMAX, false>(R, D, px, py, lane); loaded = true; }
        const unsigned long long c = xcost(sa, sb, xcross<NCH, MMAX>(R, s_off, D, qx, qy, lane));
        ++n_eval;
        if (c < bc) { bc = c; bu = cu; have = true; }
    }
    if (!have) {
        if (lane == 0 && n_eval) atomicAdd(B.evals[pair] + dir, (unsigned long long)n_eval);
        return;
    }
    const int ux0 = lo16(bu), uy0 = hi16(bu);
    uint4 r = make_uint4(0, 0, 0, 0);
    const int grid = mc.rs_grid;           // PGM-C3/G3: level-0 search on a grid only
    const int Kl = (B.level == 0 && grid > 0 && !(px % grid == grid / 2 && py % grid == grid / 2))
                       ? 0 : mc.K;
    for (int k = 0; k < Kl; ++k) {          // Eq. 5
        if ((k & 1) == 0) {
            uint4 ctr = make_uint4((uint32_t)s,
                                   ((uint32_t)B.visit << 16) | ((uint32_t)dir << 15) | (uint32_t)mc.t,
                                   ((uint32_t)B.level << 16) | (uint32_t)(k >> 1),
                                   B.stream_id[pair]);
            r = philox(ctr, mc.key0, mc.key1);
        }
        const uint32_t rx = (k & 1) ? r.z : r.x, ry = (k & 1) ? r.w : r.y;
        const int dx = rs_off(rx, k, mc.rs_W, mc.rs_mode), dy = rs_off(ry, k, mc.rs_W, mc.rs_mode);
        if (dx == 0 && dy == 0) continue;
        const int cx = ux0 + dx, cy = uy0 + dy;
        const int qx = px + cx, qy = py + cy;
        if (!inside(D, qx, qy)) continue;
        const unsigned long long sb = D.sb2[(size_t)qy * D.sbp + qx];
        if (!loaded) { xload_ref<NCH, MMAX, false>(R, D, px, py, lane); loaded = true; }
        const unsigned long long c = xcost(sa, sb, xcross<NCH, MMAX>(R, s_off, D, qx, qy, lane));
        ++n_eval;
        if (c < bc) { bc = c; bu = pack_u(cx, cy); }
    }
    if (lane == 0 && n_eval) atomicAdd(B.evals[pair] + dir, (unsigned long long)n_eval);
    if (lane == 0 && (bu != u_in || !have_in)) {
        D.u[s] = bu;
        D.cost[s] = bc;
        D.flags[s] = f0 | F_VALID;
    }
}

// ---------------------------------------------------------------- init
template <int NCH, int NORM>
__global__ void __launch_bounds__(256) k_init(const __grid_constant__ LvlBatch B, const MatchConst mc) {
    const int pair = blockIdx.z, dir = blockIdx.y;
    const DirLvl& D = B.d[pair][dir];
    const int s = blockIdx.x;
    if (s >= D.nx * D.ny) return;
    __shared__ int ref[MAXP * MAXP][NCH];
    __shared__ unsigned long long red[8];
    const int i = s % D.nx, j = s / D.nx;
    const int px = mc.c + mc.sigma * i, py = mc.c + mc.sigma * j;
    const int P = D.P, h = P / 2, P2 = P * P;
    for (int k = threadIdx.x; k < P2; k += blockDim.x) {
        int x = clampi(px + k % P - h, 0, D.rw - 1), y = clampi(py + k / P - h, 0, D.rh - 1);
        const uint32_t* w = reinterpret_cast<const uint32_t*>(D.ref + (size_t)y * D.ref_pitch +
                                                              (size_t)x * 2 * px_words(NCH));
#pragma unroll
        for (int c = 0; c < NCH / 2; ++c) {
            uint32_t v = __ldg(w + c);
            ref[k][2 * c] = lo16(v);
            ref[k][2 * c + 1] = hi16(v);
        }
    }
    __syncthreads();
    unsigned long long best = INF;
    const int nq = D.tw * D.th;
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
        const int qx = q % D.tw, qy = q / D.tw;
        unsigned long long cost = 0;
        for (int oy = 0; oy < P; ++oy) {
            const int y = clampi(qy + oy - h, 0, D.th - 1);
            const int16_t* row = D.tgt + (size_t)y * D.tgt_pitch;
            for (int ox = 0; ox < P; ++ox) {
                const int x = clampi(qx + ox - h, 0, D.tw - 1);
                const uint32_t* w = reinterpret_cast<const uint32_t*>(row + (size_t)x * 2 * px_words(NCH));
                const int* r = ref[oy * P + ox];
                uint32_t sacc = 0;
#pragma unroll
                for (int c = 0; c < NCH / 2; ++c) {
                    uint32_t v = __ldg(w + c);
                    int d0 = lo16(v) - r[2 * c], d1 = hi16(v) - r[2 * c + 1];
                    if (NORM == PGM_L2SQ) sacc += (uint32_t)(d0 * d0) + (uint32_t)(d1 * d1);
                    else sacc += (uint32_t)(abs(d0) + abs(d1));
                }
                cost += sacc;
            }
        }
        // ties: lower cost, then smaller target raster index (y, then x)
        unsigned long long key = (cost << 24) | (unsigned long long)q;
        best = key < best ? key : best;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long v = __shfl_xor_sync(FULL, best, o);
        best = v < best ? v : best;
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(B.evals[pair] + 4 + dir, (unsigned long long)nq);
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) best = red[w] < best ? red[w] : best;
        const int q = (int)(best & 0xffffffull);
        D.u[s] = pack_u(q % D.tw - px, q / D.tw - py);
        D.cost[s] = best >> 24;
        D.flags[s] = F_VALID;
    }
}

// ---------------------------------------------------------- cost fill
template <int NCH, int PPL, int NORM>
__global__ void __launch_bounds__(256) k_cost(const __grid_constant__ LvlBatch B, const MatchConst mc) {
    const int pair = blockIdx.z, dir = blockIdx.y;
    const DirLvl& D = B.d[pair][dir];
    const int lane = threadIdx.x & 31;
    const int s = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (s >= D.nx * D.ny) return;
    const uint8_t f = D.flags[s];
    if (!(f & F_VALID)) return;
    const int i = s % D.nx, j = s / D.nx;
    const int px = mc.c + mc.sigma * i, py = mc.c + mc.sigma * j;
    const int32_t u = D.u[s];
    const int qx = px + lo16(u), qy = py + hi16(u);
    if (!inside(D, qx, qy)) {            // match centre left the target image
        if (lane == 0) D.flags[s] = f & ~F_VALID;
        return;
    }
    Ref<NCH, PPL> R;
    load_ref(R, D, px, py, lane);
    unsigned long long c = warp_cost<NCH, PPL, NORM>(R, D, qx, qy, lane);
    if (lane == 0) { D.cost[s] = c; atomicAdd(B.evals[pair] + 2 + dir, 1ull); }
}

// ------------------------------------------------------ PatchMatch phase
// Seeds of colour (i + j) & 1 == mc.colour update from the current field;
// all their lattice neighbours have the other colour and stay fixed.
template <int NCH, int PPL, int NORM>
__global__ void __launch_bounds__(256) k_pm(const __grid_constant__ LvlBatch B, const MatchConst mc) {
    const int pair = blockIdx.z, dir = blockIdx.y;
    const DirLvl& D = B.d[pair][dir];
    const int lane = threadIdx.x & 31;
    const int wid = blockIdx.x * 8 + (threadIdx.x >> 5);
    const int hw = (D.nx + 1) >> 1;
    if (wid >= hw * D.ny) return;
    const int j = wid / hw;
    const int i = 2 * (wid - j * hw) + ((j + mc.colour) & 1);
    if (i >= D.nx) return;
    const int s = j * D.nx + i;
    const int px = mc.c + mc.sigma * i, py = mc.c + mc.sigma * j;

    const uint8_t f0 = D.flags[s];
    bool have = f0 & F_VALID;
    int32_t bu = D.u[s];
    unsigned long long bc = have ? D.cost[s] : INF;
    const int32_t u_in = bu;
    const bool have_in = have;

    // propagation direction of iteration t: (+,+), (-,-), (-,+), (+,-)
    const int t4 = mc.t & 3;
    const int sx = (t4 == 0 || t4 == 3) ? 1 : -1;
    const int sy = (t4 == 0 || t4 == 2) ? 1 : -1;

    Ref<NCH, PPL> R;
    bool loaded = false;
    unsigned n_eval = 0;
    // Eq. 4: candidates u(p - dx), u(p - dy) (displacement form)
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int ni = k == 0 ? i - sx : i, nj = k == 0 ? j : j - sy;
        if (ni < 0 || nj < 0 || ni >= D.nx || nj >= D.ny) continue;
        const int ns = nj * D.nx + ni;
        if (!(D.flags[ns] & F_VALID)) continue;
        const int32_t cu = D.u[ns];
        if (have && cu == bu) continue;                 // same match, same cost
        const int qx = px + lo16(cu), qy = py + hi16(cu);
        if (!inside(D, qx, qy)) continue;
        if (!loaded) { load_ref(R, D, px, py, lane); loaded = true; }
        const unsigned long long c = warp_cost<NCH, PPL, NORM>(R, D, qx, qy, lane);
        ++n_eval;
        if (c < bc) { bc = c; bu = cu; have = true; }
    }
    if (!have) {
        if (lane == 0 && n_eval) atomicAdd(B.evals[pair] + dir, (unsigned long long)n_eval);
        return;
    }
    // Eq. 5: K candidates around the post-propagation match
    const int ux0 = lo16(bu), uy0 = hi16(bu);
    uint4 r = make_uint4(0, 0, 0, 0);
    const int grid = mc.rs_grid;           // PGM-C3/G3: level-0 search on a grid only
    const int Kl = (B.level == 0 && grid > 0 && !(px % grid == grid / 2 && py % grid == grid / 2))
                       ? 0 : mc.K;
    for (int k = 0; k < Kl; ++k) {
        if ((k & 1) == 0) {
            uint4 ctr = make_uint4((uint32_t)s,
                                   ((uint32_t)B.visit << 16) | ((uint32_t)dir << 15) | (uint32_t)mc.t,
                                   ((uint32_t)B.level << 16) | (uint32_t)(k >> 1),
                                   B.stream_id[pair]);
            r = philox(ctr, mc.key0, mc.key1);
        }
        const uint32_t rx = (k & 1) ? r.z : r.x, ry = (k & 1) ? r.w : r.y;
        const int dx = rs_off(rx, k, mc.rs_W, mc.rs_mode), dy = rs_off(ry, k, mc.rs_W, mc.rs_mode);
        if (dx == 0 && dy == 0) continue;
        const int cx = ux0 + dx, cy = uy0 + dy;
        const int qx = px + cx, qy = py + cy;
        if (!inside(D, qx, qy)) continue;
        if (!loaded) { load_ref(R, D, px, py, lane); loaded = true; }
        const unsigned long long c = warp_cost<NCH, PPL, NORM>(R, D, qx, qy, lane);
        ++n_eval;
        if (c < bc) { bc = c; bu = pack_u(cx, cy); }
    }
    if (lane == 0 && n_eval) atomicAdd(B.evals[pair] + dir, (unsigned long long)n_eval);
    if (lane == 0 && (bu != u_in || !have_in)) {
        D.u[s] = bu;
        D.cost[s] = bc;
        D.flags[s] = f0 | F_VALID;
    }
}

// ------------------------------------------------------- consistency
// C = yes unless both ends are initialised and |u_f(p) + u_b(q^)|^2 <= tau2,
// q^ the seed of the other lattice nearest to q = p + u_f.  Then Eq. 6 read
// as "outlier when either is yes": O <- O or C if O was propagated, else C.
// Only the other direction's VALID bit and u are read; this kernel writes
// only OUTL bits, so the two directions can be updated in one launch.
__global__ void k_consist(const __grid_constant__ LvlBatch B, const MatchConst mc) {
    pdl_trigger();
    pdl_wait();
    const int pair = blockIdx.z, dir = blockIdx.y;
    const DirLvl& D = B.d[pair][dir];
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= D.nx * D.ny) return;
    const uint8_t f = D.flags[s];
    int out = 1;
    if ((f & F_VALID) && D.onx > 0 && D.ony > 0) {
        const int i = s % D.nx, j = s / D.nx;
        const int32_t u = D.u[s];
        const int ux = lo16(u), uy = hi16(u);
        const int qx = mc.c + mc.sigma * i + ux, qy = mc.c + mc.sigma * j + uy;
        int a = qx - mc.c + mc.sigma / 2, b = qy - mc.c + mc.sigma / 2;
        a = (a >= 0 ? a : a - mc.sigma + 1) / mc.sigma;     // floor division
        b = (b >= 0 ? b : b - mc.sigma + 1) / mc.sigma;
        const int g = clampi(b, 0, D.ony - 1) * D.onx + clampi(a, 0, D.onx - 1);
        if (PGM_CHECK(g >= 0 && g < D.onx * D.ony, B.err[pair]) && (D.oflags[g] & F_VALID)) {
            const int32_t ou = D.ou[g];
            const int ex = ux + lo16(ou), ey = uy + hi16(ou);
            out = (long long)ex * ex + (long long)ey * ey > (long long)mc.tau2;
        }
    }
    const int o_new = (f & F_OINIT) ? (((f & F_OUTL) != 0) | out) : out;
    D.flags[s] = (uint8_t)((f & ~F_OUTL) | (o_new ? F_OUTL : 0));
}

// ------------------------------------------------------------ transfer
__global__ void k_transfer(const __grid_constant__ XferBatch X) {
    pdl_trigger();
    pdl_wait();
    const int pair = blockIdx.z, dir = blockIdx.y;
    const XferDir& T = X.d[pair][dir];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T.dnx * T.dny) return;
    const int x = t % T.dnx, y = t / T.dnx;
    long long sx = 0, sy = 0;
    int n = 0, n_inl = 0;
    if (X.up) {                       // children {2x,2x+1} x {2y,2y+1} of the finer lattice
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) {
                const int cx = 2 * x + a, cy = 2 * y + b;
                if (cx >= T.snx || cy >= T.sny) continue;
                const int cs = cy * T.snx + cx;
                const uint8_t f = T.sflags[cs];
                const bool inl = !(f & F_OUTL);
                n_inl += inl;
                if (inl || (X.prop_all && (f & F_VALID))) {
                    const int32_t u = T.su[cs];
                    sx += lo16(u); sy += hi16(u); ++n;
                }
            }
    } else if (T.snx > 0 && T.sny > 0) {   // the parent on the coarser lattice
        const int cs = min(y / 2, T.sny - 1) * T.snx + min(x / 2, T.snx - 1);
        const uint8_t f = T.sflags[cs];
        const bool inl = !(f & F_OUTL);
        n_inl = inl;
        if (inl || (X.prop_all && (f & F_VALID))) {
            const int32_t u = T.su[cs];
            sx = 2LL * lo16(u); sy = 2LL * hi16(u); n = 1;
        }
    }
    int ux = 0, uy = 0;
    if (n > 0) {
        if (X.up) {                   // mean of the children, halved, half away from zero
            const long long d = 2LL * n;
            const long long ax = sx < 0 ? -sx : sx, ay = sy < 0 ? -sy : sy;
            const long long rx = (ax + n) / d, ry = (ay + n) / d;
            ux = (int)(sx < 0 ? -rx : rx);
            uy = (int)(sy < 0 ? -ry : ry);
        } else {
            ux = (int)sx; uy = (int)sy;
        }
    }
    T.du[t] = pack_u(ux, uy);
    T.dcost[t] = INF;
    uint8_t f = n > 0 ? F_VALID : 0;
    if (X.with_o) f |= F_OINIT | (n_inl == 0 ? F_OUTL : 0);
    T.dflags[t] = f;
}

// ------------------------------------------------------------ dispatch
inline int ppl_of(int maxP) {
    int p2 = maxP * maxP;
    return p2 <= 32 ? 1 : p2 <= 64 ? 2 : p2 <= 128 ? 4 : 8;
}

#define PGM_DISPATCH_NCH_PPL_NORM(KERNEL, GRID, ...)                                    \
    do {                                                                                \
        int ppl = ppl_of(maxP);                                                         \
        if (nch == 2) {                                                                 \
            if (mc.norm == 0) {                                                         \
                if (ppl == 1) KERNEL<2, 1, 0><<<GRID, 256, 0, st>>>(__VA_ARGS__);       \
                else if (ppl == 2) KERNEL<2, 2, 0><<<GRID, 256, 0, st>>>(__VA_ARGS__);  \
                else if (ppl == 4) KERNEL<2, 4, 0><<<GRID, 256, 0, st>>>(__VA_ARGS__);  \
                else KERNEL<2, 8, 0><<<GRID, 256, 0, st>>>(__VA_ARGS__);                \
            } else {                                                                    \
                if (ppl == 1) KERNEL<2, 1, 1><<<GRID, 256, 0, st>>>(__VA_ARGS__);       \
                else if (ppl == 2) KERNEL<2, 2, 1><<<GRID, 256, 0, st>>>(__VA_ARGS__);  \
                else if (ppl == 4) KERNEL<2, 4, 1><<<GRID, 256, 0, st>>>(__VA_ARGS__);  \
                else KERNEL<2, 8, 1><<<GRID, 256, 0, st>>>(__VA_ARGS__);                \
            }                                                                           \
        } else {                                                                        \
            if (mc.norm == 0) {                                                         \
                if (ppl == 1) KERNEL<6, 1, 0><<<GRID, 256, 0, st>>>(__VA_ARGS__);       \
                else if (ppl == 2) KERNEL<6, 2, 0><<<GRID, 256, 0, st>>>(__VA_ARGS__);  \
                else if (ppl == 4) KERNEL<6, 4, 0><<<GRID, 256, 0, st>>>(__VA_ARGS__);  \
                else KERNEL<6, 8, 0><<<GRID, 256, 0, st>>>(__VA_ARGS__);                \
            } else {                                                                    \
                if (ppl == 1) KERNEL<6, 1, 1><<<GRID, 256, 0, st>>>(__VA_ARGS__);       \
                else if (ppl == 2) KERNEL<6, 2, 1><<<GRID, 256, 0, st>>>(__VA_ARGS__);  \
                else if (ppl == 4) KERNEL<6, 4, 1><<<GRID, 256, 0, st>>>(__VA_ARGS__);  \
                else KERNEL<6, 8, 1><<<GRID, 256, 0, st>>>(__VA_ARGS__);                \
            }                                                                           \
        }                                                                               \
    } while (0)

inline pgm_status last_status() {
    return launch_status("match: launch");
}

}  // namespace

pgm_status launch_init(const LvlBatch& B, const MatchConst& mc, int nch, int maxP, int max_seeds,
                       cudaStream_t st) {
    (void)maxP;
    if (max_seeds <= 0) return PGM_OK;
    KScope ks(PGM_K_INIT, st);
    bool handled = false;
    const pgm_status r = launch_init_tile(B, mc, nch, &handled, st, &ks.n);
    if (r != PGM_OK || handled) return r;
    dim3 g(max_seeds, 2, B.n);
    if (nch == 2) {
        if (mc.norm == 0) k_init<2, 0><<<g, 256, 0, st>>>(B, mc);
        else k_init<2, 1><<<g, 256, 0, st>>>(B, mc);
    } else {
        if (mc.norm == 0) k_init<6, 0><<<g, 256, 0, st>>>(B, mc);
        else k_init<6, 1><<<g, 256, 0, st>>>(B, mc);
    }
    return last_status();
}

// words per lane of the squared-L2 kernels, a few fixed sizes
inline int mmax_of(int nch, int maxP) {
    const int m = (maxP * maxP * (nch / 2) + 31) / 32;
    const int sizes[6] = {2, 4, 8, 12, 16, 24};
    for (int k = 0; k < 6; ++k)
        if (m <= sizes[k]) return sizes[k];
    return 24;
}

#define PGM_DISPATCH_X(KERNEL, GRID, ...)                                                  \
    do {                                                                                   \
        const int mm = mmax_of(nch, maxP);                                                 \
        if (nch == 2) {                                                                    \
            if (mm <= 2) KERNEL<2, 2><<<GRID, 256, 0, st>>>(__VA_ARGS__);                  \
            else if (mm <= 4) KERNEL<2, 4><<<GRID, 256, 0, st>>>(__VA_ARGS__);             \
            else KERNEL<2, 8><<<GRID, 256, 0, st>>>(__VA_ARGS__);                          \
        } else {                                                                           \
            if (mm <= 2) KERNEL<6, 2><<<GRID, 256, 0, st>>>(__VA_ARGS__);                  \
            else if (mm <= 4) KERNEL<6, 4><<<GRID, 256, 0, st>>>(__VA_ARGS__);             \
            else if (mm <= 8) KERNEL<6, 8><<<GRID, 256, 0, st>>>(__VA_ARGS__);             \
            else if (mm <= 12) KERNEL<6, 12><<<GRID, 256, 0, st>>>(__VA_ARGS__);           \
            else if (mm <= 16) KERNEL<6, 16><<<GRID, 256, 0, st>>>(__VA_ARGS__);           \
            else KERNEL<6, 24><<<GRID, 256, 0, st>>>(__VA_ARGS__);                         \
        }                                                                                  \
    } while (0)

pgm_status launch_cost_fill(const LvlBatch& B, const MatchConst& mc, int nch, int maxP,
                            int max_seeds, cudaStream_t st) {
    if (max_seeds <= 0) return PGM_OK;
    KScope ks(PGM_K_COST, st);
    dim3 g((max_seeds + 7) / 8, 2, B.n);
    if (mc.norm == PGM_L2SQ) {
        bool handled = false;
        pgm_status r = launch_cost_tile(B, mc, nch, &handled, st);
        if (r != PGM_OK || handled) return r;
        PGM_DISPATCH_X(k_cost_x, g, B, mc);
    }
    else PGM_DISPATCH_NCH_PPL_NORM(k_cost, g, B, mc);
    return last_status();
}

pgm_status launch_pm_phase(const LvlBatch& B, const MatchConst& mc, int nch, int maxP,
                           int max_seeds, cudaStream_t st, cudaStream_t st2) {
    if (max_seeds <= 0) return PGM_OK;
    KScope ks(PGM_K_PM, st);
    dim3 g((max_seeds + 7) / 8, 2, B.n);   // max_seeds: half-row width x rows
    if (mc.norm == PGM_L2SQ) {
        bool handled = false;
        int nl = 0;
        pgm_status r = launch_pm_tile(B, mc, nch, maxP, &nl, &handled, st, st2);
        if (handled) ks.n = nl;
        if (r != PGM_OK || handled) return r;
        if (mc.refresh) return PGM_ERR_UNSUPPORTED;     // the per-seed kernel does no refresh
        PGM_DISPATCH_X(k_pm_x, g, B, mc);
    }
    else PGM_DISPATCH_NCH_PPL_NORM(k_pm, g, B, mc);
    return last_status();
}

pgm_status launch_box(const LvlBatch& B, int nch, int max_pixels, cudaStream_t st) {
    (void)max_pixels;
    int tiles = 0;
    for (int k = 0; k < B.n; ++k)
        for (int d = 0; d < 2; ++d) {
            const DirLvl& D = B.d[k][d];
            const int t1 = ((D.tw + BOX_TW - 1) / BOX_TW) * ((D.th + BOX_TH - 1) / BOX_TH);
            const int t2 = ((D.rw + BOX_TW - 1) / BOX_TW) * ((D.rh + BOX_TH - 1) / BOX_TH);
            tiles = t1 > tiles ? t1 : tiles;
            tiles = t2 > tiles ? t2 : tiles;
        }
    if (tiles <= 0) return PGM_OK;
    KScope ks(PGM_K_COST, st);
    dim3 g(tiles, 4, B.n);
    if (nch == 2) k_box<2><<<g, 256, 0, st>>>(B);
    else k_box<6><<<g, 256, 0, st>>>(B);
    return last_status();
}

pgm_status launch_consist(const LvlBatch& B, const MatchConst& mc, int max_seeds,
                          cudaStream_t st) {
    if (max_seeds <= 0) return PGM_OK;
    KScope ks(PGM_K_CONSIST, st);
    PGM_TRY(launch_pdl(k_consist, dim3((max_seeds + 255) / 256, 2, B.n), dim3(256), 0, st, B, mc),
            "consistency: launch");
    return last_status();
}

pgm_status launch_transfer(const XferBatch& X, int max_seeds, cudaStream_t st) {
    if (max_seeds <= 0) return PGM_OK;
    KScope ks(PGM_K_TRANSFER, st);
    PGM_TRY(launch_pdl(k_transfer, dim3((max_seeds + 255) / 256, 2, X.n), dim3(256), 0, st, X),
            "transfer: launch");
    return last_status();
}

}  // namespace pgm
