// interp.cu -- sparse-to-dense interpolation of the exported matches
// (Sec. III-G): every pixel of the reference image takes its K geodesically
// nearest matches and interpolates their displacements by a Nadaraya-Watson
// average (NW) or a locally weighted affine fit (LA), LA when the matches
// exceed 2.2 % of the image.
//
//   step cost     c(p) = 1 + (sum over descriptor channels of |g(p)|) >> shift
//   edge p - q    c(p) + c(q) on the 4-connected grid
//   neighbours    the K smallest (geodesic distance, match index) pairs
//   weights       exp(-(d - d_nearest) / lambda), in double precision
//
// The K-nearest lists are found by relaxation: a list entry (d, i) is a path
// of length d from match i, every pixel keeps its K best entries with
// distinct labels, and a pixel's candidates are its 4 neighbours' entries
// plus the step.  The fixed point is the exact K-nearest set (if match i is
// among the K nearest of p, it is among the K nearest of every pixel on a
// shortest path from i to p), and the relaxation reaches it from any order of
// updates, so the result is deterministic.  A launch relaxes 16 x 16 tiles in
// shared memory until each tile is stable; launches repeat until none
// changes anything.
#include <stdint.h>

#include "pgm_device.cuh"

namespace pgm {
namespace {

constexpr int IT_W = 16;                 // tile side (pixels), one thread each
constexpr int IT_H = IT_W + 2;           // with the 1-pixel halo
constexpr int IK_MAX = 16;               // neighbours per pixel at most
constexpr int IT_INNER = 64;             // relaxation rounds per launch and tile
constexpr unsigned long long EMPTY = ~0ull;

// key = distance << 32 | match index; ascending keys are the (d, i) order
__device__ __forceinline__ unsigned lab_of(unsigned long long k) { return (unsigned)k; }

// Insert a candidate into a sorted list of k distinct labels: a worse entry
// of the same label gives way, a better one keeps the candidate out.
// True when the list changed.
__device__ __forceinline__ bool list_insert(unsigned long long (&L)[IK_MAX], int k,
                                            unsigned long long cand) {
    const unsigned lab = lab_of(cand);
    int same = -1;
#pragma unroll
    for (int e = 0; e < IK_MAX; ++e)
        if (e < k && L[e] != EMPTY && lab_of(L[e]) == lab) same = e;
    if (same >= 0) {
        bool worse = false;
#pragma unroll
        for (int e = 0; e < IK_MAX; ++e)
            if (e == same) worse = L[e] > cand;
        if (!worse) return false;
        // drop it: the entries after it move up one place
#pragma unroll
        for (int e = 0; e < IK_MAX - 1; ++e)
            if (e >= same && e < k - 1) L[e] = L[e + 1];
#pragma unroll
        for (int e = 0; e < IK_MAX; ++e)
            if (e == k - 1) L[e] = EMPTY;
    } else {
        bool full_worse = false;
#pragma unroll
        for (int e = 0; e < IK_MAX; ++e)
            if (e == k - 1) full_worse = cand >= L[e];
        if (full_worse) return false;
    }
#pragma unroll
    for (int e = 0; e < IK_MAX; ++e)
        if (e < k && cand < L[e]) {
            const unsigned long long t = L[e];
            L[e] = cand;
            cand = t;
        }
    return true;
}

// step costs and empty lists
__global__ void k_icost(const int16_t* desc, int row, int pxe, int nch, int w, int h, int shift,
                        int k, uint32_t* cost, unsigned long long* keys) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (int64_t)w * h) return;
    const int x = (int)(p % w), y = (int)(p / w);
    const int16_t* g = desc + (int64_t)y * row + (int64_t)x * pxe;
    long long s = 0;
    for (int c = 0; c < nch; ++c) s += g[c] < 0 ? -(int)g[c] : (int)g[c];
    cost[p] = 1u + (uint32_t)(s >> shift);
    for (int e = 0; e < k; ++e) keys[p * k + e] = EMPTY;
}

// every match enters its pixel's list at distance 0 (the smaller index where
// two share a pixel)
__global__ void k_iseed(const int32_t* rows, const int32_t* count, int64_t max_rows, int w, int h,
                        int k, unsigned long long* keys) {
    const int64_t n = min((int64_t)*count, max_rows);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int x = rows[4 * i], y = rows[4 * i + 1];
        if (x < 0 || y < 0 || x >= w || y >= h) continue;
        atomicMin(keys + ((int64_t)y * w + x) * k, (unsigned long long)i);
    }
}

// KT > 0: k fixed at compile time (the default 16), which keeps the list in
// registers; KT = 0: any k
template <int KT>
__global__ void __launch_bounds__(IT_W * IT_W) k_irelax(const uint32_t* cost, int w, int h, int k_,
                                                        unsigned long long* keys, unsigned* changed) {
    const int k = KT > 0 ? KT : k_;
    __shared__ unsigned long long sl[IT_H * IT_H][IK_MAX];
    __shared__ uint32_t sc[IT_H * IT_H];
    __shared__ uint8_t dirty[2][IT_H * IT_H];     // the list changed in the last round
    const int tx = threadIdx.x % IT_W, ty = threadIdx.x / IT_W;
    const int x0 = blockIdx.x * IT_W - 1, y0 = blockIdx.y * IT_W - 1;
    for (int t = threadIdx.x; t < IT_H * IT_H; t += IT_W * IT_W) {
        const int x = x0 + t % IT_H, y = y0 + t / IT_H;
        const bool in = x >= 0 && y >= 0 && x < w && y < h;
        const int64_t p = (int64_t)y * w + x;
        sc[t] = in ? cost[p] : 0u;
        for (int e = 0; e < IK_MAX; ++e) sl[t][e] = in && e < k ? keys[p * k + e] : EMPTY;
        dirty[0][t] = 1;                         // round 0 looks at every neighbour
        dirty[1][t] = 0;
    }
    __syncthreads();
    const int x = x0 + 1 + tx, y = y0 + 1 + ty, me = (ty + 1) * IT_H + tx + 1;
    const bool live = x < w && y < h;
    unsigned long long L[IK_MAX];
#pragma unroll
    for (int e = 0; e < IK_MAX; ++e) L[e] = sl[me][e];
    bool any = false;
    for (int it = 0; it < IT_INNER; ++it) {
        bool ch = false;
        const int cur = it & 1;
        if (live) {
            const int nb[4] = {me - 1, me + 1, me - IT_H, me + IT_H};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int t = nb[q];
                if (sc[t] == 0u) continue;                       // outside the image
                if (!dirty[cur][t]) continue;                    // nothing new there
                const unsigned long long step = (unsigned long long)(sc[me] + sc[t]) << 32;
                for (int e = 0; e < k; ++e) {
                    const unsigned long long key = sl[t][e];
                    if (key == EMPTY) break;
                    if ((key >> 32) + (step >> 32) >= 0xffffffffull) break;   // out of range
                    const unsigned long long cand = key + step;
                    // a full list whose worst entry is no worse than this
                    // candidate gains nothing from it or the larger ones after it
                    unsigned long long worst = EMPTY;
#pragma unroll
                    for (int f = 0; f < IK_MAX; ++f)
                        if (f == k - 1) worst = L[f];
                    if (worst != EMPTY && cand >= worst) break;
                    ch |= list_insert(L, k, cand);
                }
            }
        }
        __syncthreads();                                         // everyone has read
        if (ch) {
#pragma unroll
            for (int e = 0; e < IK_MAX; ++e) sl[me][e] = L[e];
        }
        dirty[cur ^ 1][me] = ch;                                 // read in the next round
        if (threadIdx.x < 4 * IT_H) {                            // the halo does not change
            const int e = threadIdx.x, t = e < IT_H ? e : e < 2 * IT_H ? (IT_H - 1) * IT_H + e - IT_H
                                              : e < 3 * IT_H ? (e - 2 * IT_H) * IT_H
                                                             : (e - 3 * IT_H) * IT_H + IT_H - 1;
            dirty[cur ^ 1][t] = 0;
        }
        any |= ch;
        if (!__syncthreads_or(ch)) break;                        // the tile is stable
    }
    if (live && any) {
        const int64_t p = (int64_t)y * w + x;
#pragma unroll
        for (int e = 0; e < IK_MAX; ++e)
            if (e < k) keys[p * k + e] = L[e];
    }
    if (__syncthreads_or(any) && threadIdx.x == 0) atomicOr(changed, 1u);
}

// NW or LA at every pixel; double precision without contraction, in the
// order of the plain definition
__global__ void k_iflow(const unsigned long long* keys, int w, int h, int k, const int32_t* rows,
                        const int32_t* count, int64_t max_rows, int mode, int permyriad,
                        double lambda, float* flow) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (int64_t)w * h) return;
    const int64_t n = min((int64_t)*count, max_rows);
    const bool use_la = mode == PGM_INTERP_LA ||
                        (mode == PGM_INTERP_AUTO && n * 10000 > (int64_t)permyriad * w * h);
    const int x = (int)(p % w), y = (int)(p / w);
    double sw = 0, nwx = 0, nwy = 0;
    double M[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, bx[3] = {0, 0, 0}, by[3] = {0, 0, 0};
    const unsigned long long d0 = keys[p * k] >> 32;
    for (int e = 0; e < k; ++e) {
        const unsigned long long key = keys[p * k + e];
        if (key == EMPTY) break;
        const int64_t i = (int64_t)(key & 0xffffffffu);
        const double wgt = exp(-(double)((key >> 32) - d0) / lambda);
        const int sx = rows[4 * i], sy = rows[4 * i + 1];
        const double fx = (double)(rows[4 * i + 2] - sx), fy = (double)(rows[4 * i + 3] - sy);
        const double v[3] = {(double)(sx - x), (double)(sy - y), 1.0};
        sw = __dadd_rn(sw, wgt);
        nwx = __dadd_rn(nwx, __dmul_rn(wgt, fx));
        nwy = __dadd_rn(nwy, __dmul_rn(wgt, fy));
#pragma unroll
        for (int a = 0; a < 3; ++a) {
#pragma unroll
            for (int b = 0; b < 3; ++b) M[a][b] = __dadd_rn(M[a][b], __dmul_rn(__dmul_rn(wgt, v[a]), v[b]));
            bx[a] = __dadd_rn(bx[a], __dmul_rn(__dmul_rn(wgt, fx), v[a]));
            by[a] = __dadd_rn(by[a], __dmul_rn(__dmul_rn(wgt, fy), v[a]));
        }
    }
    double ox = 0, oy = 0;
    if (sw > 0) {
        ox = nwx / sw;
        oy = nwy / sw;
        if (use_la) {
            auto mul = [](double a, double b) { return __dmul_rn(a, b); };
            auto sub = [](double a, double b) { return __dsub_rn(a, b); };
            auto add = [](double a, double b) { return __dadd_rn(a, b); };
            const double det = add(sub(mul(M[0][0], sub(mul(M[1][1], M[2][2]), mul(M[1][2], M[2][1]))),
                                       mul(M[0][1], sub(mul(M[1][0], M[2][2]), mul(M[1][2], M[2][0])))),
                                   mul(M[0][2], sub(mul(M[1][0], M[2][1]), mul(M[1][1], M[2][0]))));
            if (det > mul(mul(mul(1e-6, sw), sw), sw)) {
                const double dx = add(sub(mul(M[0][0], sub(mul(M[1][1], bx[2]), mul(bx[1], M[2][1]))),
                                          mul(M[0][1], sub(mul(M[1][0], bx[2]), mul(bx[1], M[2][0])))),
                                      mul(bx[0], sub(mul(M[1][0], M[2][1]), mul(M[1][1], M[2][0]))));
                const double dy = add(sub(mul(M[0][0], sub(mul(M[1][1], by[2]), mul(by[1], M[2][1]))),
                                          mul(M[0][1], sub(mul(M[1][0], by[2]), mul(by[1], M[2][0])))),
                                      mul(by[0], sub(mul(M[1][0], M[2][1]), mul(M[1][1], M[2][0]))));
                ox = dx / det;
                oy = dy / det;
            }
        }
    }
    flow[2 * p] = (float)ox;
    flow[2 * p + 1] = (float)oy;
}

}  // namespace

// workspace: the lists (w h k keys), the step costs, the change flag
struct IPlan { size_t off_keys, off_cost, off_flag, bytes; };
static bool make_iplan(int w, int h, int k, IPlan* ip) {
    if (w < 1 || h < 1 || w > 32767 || h > 32767 || k < 1 || k > IK_MAX) return false;
    auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
    const size_t n = (size_t)w * h;
    ip->off_keys = 0;
    ip->off_cost = al(n * k * 8);
    ip->off_flag = ip->off_cost + al(n * 4);
    ip->bytes = ip->off_flag + 256;
    return true;
}

}  // namespace pgm

using namespace pgm;

extern "C" {

void pgm_interp_default_params(pgm_interp_params* ip) {
    if (!ip) return;
    ip->k = 16;
    ip->mode = PGM_INTERP_AUTO;
    ip->cost_shift = 10;
    ip->la_permyriad = 220;
    ip->lambda = 32.0;
}

size_t pgm_interp_workspace_bytes(int w, int h, const pgm_interp_params* ip) {
    IPlan pl;
    return ip && make_iplan(w, h, ip->k, &pl) ? pl.bytes : 0;
}

pgm_status pgm_interpolate(const pgm_params* p, const void* d_pyr1, int w, int h,
                           const int32_t* d_matches, const int32_t* d_count, int64_t max_matches,
                           const pgm_interp_params* ip, void* d_ws, size_t ws_bytes,
                           float* d_flow, void* stream) {
    pgm_status r = check_params(p);
    if (r != PGM_OK) return r;
    if (!ip || !d_pyr1 || !d_count || !d_ws || !d_flow || max_matches < 0 ||
        (max_matches > 0 && !d_matches) || ip->cost_shift < 0 || ip->cost_shift > 31 ||
        !(ip->lambda > 0) || ip->la_permyriad < 0 || ip->mode < PGM_INTERP_AUTO ||
        ip->mode > PGM_INTERP_LA || (((uintptr_t)d_ws) & 255u))
        return PGM_ERR_ARG;
    PyrPlan pp;
    IPlan pl;
    if (!make_pyr_plan(p, w, h, &pp) || !make_iplan(w, h, ip->k, &pl)) return PGM_ERR_ARG;
    if (ws_bytes < pl.bytes) return PGM_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint8_t* ws = static_cast<uint8_t*>(d_ws);
    auto* keys = reinterpret_cast<unsigned long long*>(ws + pl.off_keys);
    auto* cost = reinterpret_cast<uint32_t*>(ws + pl.off_cost);
    auto* flag = reinterpret_cast<unsigned*>(ws + pl.off_flag);
    const int16_t* desc = reinterpret_cast<const int16_t*>(static_cast<const uint8_t*>(d_pyr1) +
                                                           pp.desc_off[0][0]);
    Range range("pgm_interpolate");
    const int64_t n = (int64_t)w * h;
    const int blocks = (int)((n + 255) / 256);
    k_icost<<<blocks, 256, 0, st>>>(desc, pp.desc_row[0], 2 * pp.pxw, pp.nch, w, h, ip->cost_shift,
                                    ip->k, cost, keys);
    if ((r = launch_status("interpolate: costs")) != PGM_OK) return r;
    if (max_matches > 0) {
        k_iseed<<<152, 256, 0, st>>>(d_matches, d_count, max_matches, w, h, ip->k, keys);
        if ((r = launch_status("interpolate: seeds")) != PGM_OK) return r;
    }
    // relax until a launch changes nothing; a bound far above any path length
    // in tiles keeps a defect from looping for ever
    const dim3 grid((w + IT_W - 1) / IT_W, (h + IT_W - 1) / IT_W);
    const long long most = 4ll * (long long)w * h / (IT_W * IT_W) + 64;
    unsigned host_flag = 1;
    long long launches = 0;
    while (host_flag) {
        if (launches++ > most) return PGM_ERR_UNSUPPORTED;
        PGM_TRY(cudaMemsetAsync(flag, 0, 4, st), "interpolate: clear the flag");
        if (ip->k == IK_MAX) k_irelax<IK_MAX><<<grid, IT_W * IT_W, 0, st>>>(cost, w, h, ip->k, keys, flag);
        else k_irelax<0><<<grid, IT_W * IT_W, 0, st>>>(cost, w, h, ip->k, keys, flag);
        if ((r = launch_status("interpolate: relax")) != PGM_OK) return r;
        PGM_TRY(cudaMemcpyAsync(&host_flag, flag, 4, cudaMemcpyDeviceToHost, st),
                "interpolate: read the flag");
        PGM_TRY(cudaStreamSynchronize(st), "interpolate: synchronize");
    }
    k_iflow<<<blocks, 256, 0, st>>>(keys, w, h, ip->k, d_matches, d_count, max_matches, ip->mode,
                                    ip->la_permyriad, ip->lambda, d_flow);
    return launch_status("interpolate: flow");
}

}  // extern "C"
