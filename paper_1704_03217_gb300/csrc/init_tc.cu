// init_tc.cu -- exhaustive nearest-neighbour initialisation at the coarsest
// level (Sec. III-D; every seed starts from the target centre of least patch
// distance, Eq. 3, ties to the smaller raster index) on the tensor cores, for
// the six-channel descriptors and the squared-L2 cost.
//
// Over integers D(s, q) = sum |a|^2 + sum |b|^2 - 2 X(s, q), and the cross
// terms of all seeds against all target centres form one dense contraction
//   X(s, q) = sum_k A(s, k) B(q, k),   k = (patch row r, column p, channel).
// tcgen05.mma (kind::f16) multiplies fp16 operands from shared memory into
// fp32 accumulators in tensor memory.  To make that exact, every descriptor
// value v (|v| <= 12240, Sobel-5 on 8-bit channels) is split as
// v = 128 v_h + v_l with v_l in [-64, 63] and v_h in [-96, 96], both exact in
// fp16, and
//   X = 2^14 <a_h, b_h> + 2^7 (<a_h, b_l> + <a_l, b_h>) + <a_l, b_l>
// takes three accumulators.  Each product is an integer of magnitude at most
// 96 * 96 (one accumulator) or 2 * 96 * 64 (the middle one, two products per
// element), so for patches up to 15 x 15 x 6 every partial sum is an integer
// below 2^24 (225 * 6 * 12288 = 16588800) and fp32 holds it exactly.
//
// No operand is copied out patch by patch.  One MMA step (K = 16) is two
// pixels of 8 fp16 values (16 bytes: the six channels and two zero pads), and
// the tensor core reads an operand as groups of eight 16-byte rows, 16 bytes
// apart, the groups 128 bytes apart, the second 8-value half of the step at a
// free distance (the descriptor's leading-byte offset):
// - target centres, flattened as n = y Wt + x over a copy of the target with a
//   border of P / 2 on every side (row pitch Wt = tw + P - 1): pixel (p, r) of
//   centre n is staged pixel n + r Wt + p, so consecutive centres are
//   consecutive rows of every step;
// - seeds, on a lattice of stride sigma: the reference is staged as sigma^2
//   phase images R_{phi,psi}(u, v) = R(sigma u + phi + o, sigma v + psi + o),
//   o = c - P / 2, of row pitch Wu = nx + (P - 1) / sigma; seed (i, j),
//   flattened as m = j Wu + i, reads pixel (p, r) in phase
//   (p mod sigma, r mod sigma) at m + (r div sigma) Wu + p div sigma, so
//   consecutive seeds are again consecutive rows.
// The two pixels of a step are any two whose staged addresses increase in both
// operands; a pixel left without a partner (P^2 is odd) takes a block of zeros
// on the target side.  Flattened seeds with i >= nx and centres with x >= tw
// are computed and ignored.
//
// A CTA takes one tile of 128 flattened seeds (the MMA's M, one tensor-memory
// lane each) of one direction of one pair and a band of TC_NT tiles of 160
// flattened centres (the MMA's N; three fp32 accumulators of 160 columns).
// Eight warps stage and convert the operands; one thread issues the MMAs of a
// tile and commits them to an mbarrier; then every warp reads its lanes'
// accumulators (warp w: lanes 32 (w mod 4) .., columns 80 (w div 4) ..),
// forms the exact costs and keeps per seed the least (cost, raster index),
// packed as cost << 24 | q (cost < 2^40 for these patches, q < 2^24).  The
// bands of a seed meet in an atomicMin on its cost word, cleared before and
// unpacked after.
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>

#include "match_common.cuh"

namespace pgm {

long long wait_limit();      // the mbarrier wait limit (pgm_set_wait_limit)

namespace {

constexpr int TC_M = 128;              // flattened seeds per tile
constexpr int TC_N = 160;              // flattened target centres per tile
constexpr int TC_NT = 2;               // centre tiles per CTA
constexpr int TC_THREADS = 256;
constexpr int TC_MAXP = 15;            // the exact-accumulation bound above
constexpr int TC_MAXSTEP = 128;        // K steps of a 15 x 15 patch: 113
constexpr int TC_HDR = 8;              // header pixels: mbarrier, tensor-memory address, abort
constexpr int TC_TMEM_COLS = 512;      // 3 x 160 accumulator columns, rounded to a power of 2
constexpr long long TC_DRAIN_CYCLES = 1ll << 31;

struct TcPairs {                       // the K steps of each direction's patch
    int n[2];
    uint16_t pr[2][TC_MAXSTEP];        // p1 | r1 << 4 | p2 << 8 | r2 << 12; p2 = 15: zero partner
};

struct TcGeom {
    int e, Wu, mtiles, LA, Wt, ntiles, bands, LB, ctas, phases;
};

__host__ __device__ inline TcGeom tc_geom(const DirLvl& D, int sigma) {
    TcGeom g;
    g.e = (D.P - 1) / sigma;
    g.Wu = D.nx + g.e;
    g.mtiles = (D.ny * g.Wu + TC_M - 1) / TC_M;
    // one phase slice: a tile starts up to Wu - 1 pixels into its first row and
    // reads 128 rows, up to e Wu + e further, and one more for a zero partner
    g.LA = g.Wu * (g.e + 1) + TC_M + g.e;
    g.Wt = D.tw + D.P - 1;
    g.ntiles = (D.th * g.Wt + TC_N - 1) / TC_N;
    g.bands = (g.ntiles + TC_NT - 1) / TC_NT;
    g.LB = TC_NT * TC_N + (D.P - 1) * (g.Wt + 1);
    g.ctas = g.mtiles * g.bands;
    g.phases = sigma * sigma;
    return g;
}

// shared memory in 16-byte units: header, centre table (sum |b|^2 and raster
// index per column), K-step table, reference phase slices (high, then low
// parts), target band (high, low), zero block, per-seed results of the two
// column halves
__host__ __device__ inline int tc_units(const TcGeom& g) {
    return TC_HDR + TC_NT * TC_N + TC_MAXSTEP + 2 * g.phases * g.LA + 2 * g.LB + TC_N + 2 * TC_M;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void tc_mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ bool tc_mbar_test(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    return ok != 0;
}
// wait for phase `parity`; false after `limit` cycles
__device__ __forceinline__ bool tc_mbar_wait(uint32_t bar, uint32_t parity, long long limit) {
    const long long t0 = clock64();
    for (;;) {
        if (tc_mbar_test(bar, parity)) return true;
        if (clock64() - t0 > limit) return false;
    }
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}
// K-major operand without swizzling: groups of eight 16-byte rows, 128 bytes
// apart (stride-dimension offset); the second 8-value half of the step `lbo`
// bytes after the first (leading-dimension offset); descriptor version 1
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo) {
    return (uint64_t)((addr >> 4) & 0x3fffu) | ((uint64_t)((lbo >> 4) & 0x3fffu) << 16) |
           ((uint64_t)(128u >> 4) << 32) | (1ull << 46);
}
// D[tmem] (+)= A B^T for one K step of 16; accumulate = 0 overwrites
__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate) : "memory");
}
// arrive on the mbarrier once every MMA this thread issued has completed
__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                 ::"r"(bar) : "memory");
}
// 16 consecutive accumulator columns of this thread's lane (32-bit each),
// waited for before the registers are used
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
          "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr) : "memory");
}

// the eight int16 of a pixel (six values, two zero pads) as fp16 high and low
// parts, v = 128 v_h + v_l
__device__ __forceinline__ void tc_split(const uint4 w, uint4& hi, uint4& lo) {
    const uint32_t in[4] = {w.x, w.y, w.z, w.w};
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        uint32_t hv = 0, lv = 0;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int v = (int)(int16_t)(uint16_t)(in[i] >> (16 * k));
            const int vl = ((v + 64) & 127) - 64, vh = (v - vl) >> 7;
            hv |= (uint32_t)__half_as_ushort(__short2half_rn((short)vh)) << (16 * k);
            lv |= (uint32_t)__half_as_ushort(__short2half_rn((short)vl)) << (16 * k);
        }
        h[i] = hv;
        l[i] = lv;
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

__global__ void __launch_bounds__(TC_THREADS, 1)
k_init_tc(const __grid_constant__ LvlBatch B, const MatchConst mc, const __grid_constant__ TcPairs T,
          long long limit) {
    extern __shared__ __align__(1024) uint4 sm4[];
    const int dir = blockIdx.z, pair = blockIdx.y;
    const DirLvl& D = B.d[pair][dir];
    const int sg = mc.sigma, P = D.P, h = P / 2;
    const TcGeom g = tc_geom(D, sg);
    if ((int)blockIdx.x >= g.ctas || D.nx * D.ny == 0) return;
    const int mt = blockIdx.x % g.mtiles, band = blockIdx.x / g.mtiles;
    const int m0 = mt * TC_M, v0 = m0 / g.Wu, moff = m0 - v0 * g.Wu;
    const int nb = band * TC_NT * TC_N;
    const int ntile = min(TC_NT, g.ntiles - band * TC_NT);
    const int nsteps = T.n[dir];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // shared memory, in 16-byte units
    uint4* sQ = sm4 + TC_HDR;                          // centre table
    uint4* sS = sQ + TC_NT * TC_N;                     // K steps: a1, a2 - a1, b1, b2 - b1 (-1: zero)
    uint4* sA = sS + TC_MAXSTEP;                       // [part][phase][LA]
    uint4* sB = sA + 2 * g.phases * g.LA;              // [part][LB]
    uint4* sZ = sB + 2 * g.LB;                         // TC_N zero rows
    unsigned long long* sBest = reinterpret_cast<unsigned long long*>(sZ + TC_N);   // [2][TC_M]
    const uint32_t bar = smem_u32(sm4);
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(sm4) + 2;
    volatile int* s_abort = reinterpret_cast<volatile int*>(sm4) + 3;

    if (tid == 0) {
        tc_mbar_init(bar, 1);
        *s_abort = 0;
    }
    if (warp == 0) {                                   // the accumulators: 512 columns, all lanes
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                     ::"r"(smem_u32(s_tmem)), "r"(TC_TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }

    // reference phase slices: slice index k of phase (phi, psi) is phase pixel
    // f = v0 Wu + k, i.e. (u, v) = (f mod Wu, f div Wu); reads outside the
    // padded descriptor are clamped (only flattened seeds past the lattice
    // reach them)
    const int o = mc.c - h;
    const int rpitch = D.ref_pitch, tpitch = D.tgt_pitch;
#pragma unroll 4
    for (int e = tid; e < g.phases * g.LA; e += TC_THREADS) {
        const int ph = e / g.LA, k = e - ph * g.LA;
        const int f = v0 * g.Wu + k, v = f / g.Wu, u = f - v * g.Wu;
        const int X = clampi(sg * u + ph % sg + o, -BORD, D.rw + BORD - 1);
        const int Y = clampi(sg * v + ph / sg + o, -BORD, D.rh + BORD - 1);
        const uint4 w = __ldg(reinterpret_cast<const uint4*>(D.ref + (ptrdiff_t)Y * rpitch + 8 * X));
        uint4 hi, lo;
        tc_split(w, hi, lo);
        sA[e] = hi;
        sA[g.phases * g.LA + e] = lo;
    }
    // target band: staged pixel f = nb + k is (f mod Wt - P/2, f div Wt - P/2)
#pragma unroll 4
    for (int k = tid; k < g.LB; k += TC_THREADS) {
        const int f = nb + k, row = f / g.Wt, col = f - row * g.Wt;
        const int X = clampi(col - h, -BORD, D.tw + BORD - 1);
        const int Y = clampi(row - h, -BORD, D.th + BORD - 1);
        const uint4 w = __ldg(reinterpret_cast<const uint4*>(D.tgt + (ptrdiff_t)Y * tpitch + 8 * X));
        uint4 hi, lo;
        tc_split(w, hi, lo);
        sB[k] = hi;
        sB[g.LB + k] = lo;
    }
    for (int k = tid; k < TC_N; k += TC_THREADS) sZ[k] = make_uint4(0u, 0u, 0u, 0u);
    // centres of the band's columns: sum |b|^2 (INF: not a centre) and raster index
    for (int j = tid; j < TC_NT * TC_N; j += TC_THREADS) {
        const int n = nb + j, y = n / g.Wt, x = n - y * g.Wt;
        const bool in = x < D.tw && y < D.th;
        const unsigned long long sb = in ? D.sb2[(size_t)y * D.sbp + x] : INF;
        sQ[j] = make_uint4((uint32_t)sb, (uint32_t)(sb >> 32), (uint32_t)(y * D.tw + x), 0u);
    }
    // K steps: staged offsets (16-byte units) of both pixels in both operands
    for (int t = tid; t < nsteps; t += TC_THREADS) {
        const uint32_t c = T.pr[dir][t];
        const int p1 = c & 15, r1 = (c >> 4) & 15, p2 = (c >> 8) & 15, r2 = c >> 12;
        const int a1 = ((r1 % sg) * sg + p1 % sg) * g.LA + (r1 / sg) * g.Wu + p1 / sg;
        const bool z = p2 == 15;
        const int a2 = z ? a1 + 1 : ((r2 % sg) * sg + p2 % sg) * g.LA + (r2 / sg) * g.Wu + p2 / sg;
        const int b1 = r1 * g.Wt + p1;
        sS[t] = make_uint4((uint32_t)a1, (uint32_t)(a2 - a1), (uint32_t)b1,
                           z ? 0xffffffffu : (uint32_t)(r2 * g.Wt + p2 - b1));
    }
    // the staged operands are read by the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_tmem;

    // seed of this thread's accumulator lane
    const int quarter = warp & 3, half = warp >> 2;
    const int m = m0 + 32 * quarter + lane, si = m % g.Wu, sj = m / g.Wu;
    const bool seed_ok = si < D.nx && sj < D.ny;
    const unsigned long long sa =
        seed_ok ? D.sa2img[(size_t)(mc.c + sg * sj) * D.rw + (mc.c + sg * si)] : 0ull;
    unsigned long long best = INF;

    // M = 128, N = 160, fp16 A and B (K-major), fp32 accumulators
    const uint32_t idesc = (1u << 4) | ((uint32_t)(TC_N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
    const uint32_t aA = smem_u32(sA), aB = smem_u32(sB), aZ = smem_u32(sZ);
    int issued = 0;
    for (int k = 0; k < ntile; ++k) {
        if (tid == 0) {
            for (int t = 0; t < nsteps; ++t) {
                const uint4 s = sS[t];
                const uint32_t boff = (uint32_t)(k * TC_N) + s.z;
#pragma unroll
                for (int pa = 0; pa < 2; ++pa)
#pragma unroll
                    for (int pb = 0; pb < 2; ++pb) {
                        const uint32_t a = aA + 16u * ((uint32_t)(pa * g.phases * g.LA + moff) + s.x);
                        const uint32_t b = aB + 16u * ((uint32_t)(pb * g.LB) + boff);
                        const uint32_t blbo = s.w == 0xffffffffu ? aZ - b : 16u * s.w;
                        const uint32_t acc = (t > 0 || (pa == 1 && pb == 0)) ? 1u : 0u;
                        tc_mma(tmem + (uint32_t)((pa + pb) * TC_N), tc_desc(a, 16u * s.y),
                               tc_desc(b, blbo), idesc, acc);
                    }
            }
            tc_commit(bar);
        }
        issued = k + 1;
        __syncwarp();
        const bool ok = __all_sync(FULL, tc_mbar_wait(bar, (uint32_t)(k & 1), limit));
        tc_fence_after();
        if (!ok) {
            if (lane == 0) {
                atomicOr(B.err[pair], (unsigned)PGM_ERR_TIMEOUT);
                *s_abort = 1;
            }
        } else {
            // columns 80 half .. of the three accumulators, 16 at a time
            const uint32_t trow = tmem + ((uint32_t)(32 * quarter) << 16);
#pragma unroll 1
            for (int c0 = 80 * half; c0 < 80 * half + 80; c0 += 16) {
                uint32_t x0[16], x1[16], x2[16];
                tc_ld16(trow + (uint32_t)c0, x0);
                tc_ld16(trow + (uint32_t)(TC_N + c0), x1);
                tc_ld16(trow + (uint32_t)(2 * TC_N + c0), x2);
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const uint4 q = sQ[k * TC_N + c0 + j];
                    const unsigned long long sb = (unsigned long long)q.x | ((unsigned long long)q.y << 32);
                    if (sb == INF) continue;
                    const long long cross = ((long long)__float2int_rn(__uint_as_float(x0[j])) << 14) +
                                            ((long long)__float2int_rn(__uint_as_float(x1[j])) << 7) +
                                            (long long)__float2int_rn(__uint_as_float(x2[j]));
                    const unsigned long long key = (xcost(sa, sb, cross) << 24) | q.z;
                    best = key < best ? key : best;
                }
            }
        }
        tc_fence_before();
        __syncthreads();                               // accumulators free for the next tile
        tc_fence_after();
        if (*s_abort) break;
    }
    // the two column halves of a seed, then the bands of the seed
    sBest[half * TC_M + 32 * quarter + lane] = best;
    __syncthreads();
    if (tid < TC_M && !*s_abort) {
        const unsigned long long b0 = sBest[tid], b1 = sBest[TC_M + tid];
        const unsigned long long bb = b0 < b1 ? b0 : b1;
        const int mm = m0 + tid, i = mm % g.Wu, j = mm / g.Wu;
        if (i < D.nx && j < D.ny && bb != INF) atomicMin(D.cost + (size_t)j * D.nx + i, bb);
    }
    if (*s_abort && tid == 0 && issued > 0)            // let the issued MMAs finish
        (void)tc_mbar_wait(bar, (uint32_t)((issued - 1) & 1), TC_DRAIN_CYCLES);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n"
                     ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
    }
}

// every seed's result word starts at INF (no centre yet)
__global__ void k_init_tc_clear(const __grid_constant__ LvlBatch B) {
    const DirLvl& D = B.d[blockIdx.z][blockIdx.y];
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < D.nx * D.ny) D.cost[s] = INF;
}

// cost << 24 | q  ->  displacement, cost and flags of every seed
__global__ void k_init_tc_fin(const __grid_constant__ LvlBatch B, const MatchConst mc) {
    const int pair = blockIdx.z, dir = blockIdx.y;
    const DirLvl& D = B.d[pair][dir];
    const int ns = D.nx * D.ny, s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s == 0 && ns > 0)
        atomicAdd(B.evals[pair] + 4 + dir, (unsigned long long)ns * (unsigned long long)(D.tw * D.th));
    if (s >= ns) return;
    const unsigned long long k = D.cost[s];
    if (k == INF) {                                    // left unset (a wait ran out)
        D.u[s] = 0;
        D.flags[s] = 0;
        return;
    }
    const int q = (int)(k & 0xffffffull), si = s % D.nx, sj = s / D.nx;
    D.u[s] = pack_u(q % D.tw - (mc.c + mc.sigma * si), q / D.tw - (mc.c + mc.sigma * sj));
    D.cost[s] = k >> 24;
    D.flags[s] = F_VALID;
}

// The K steps of a P x P patch: pixels in raster order, each paired with the
// first later unpaired pixel that also lies later in the phase order (phase
// (r mod sigma) sigma + p mod sigma, then r div sigma, then p div sigma), so
// that both operands' second-pixel offsets are positive; else the zero block.
int tc_pairs(int P, int sigma, uint16_t* out) {
    bool used[TC_MAXP * TC_MAXP] = {};
    auto akey = [&](int i) {
        const int p = i % P, r = i / P;
        return (((r % sigma) * sigma + p % sigma) * 64 + r / sigma) * 64 + p / sigma;
    };
    int n = 0;
    for (int i = 0; i < P * P; ++i) {
        if (used[i]) continue;
        used[i] = true;
        int j = i + 1;
        while (j < P * P && (used[j] || akey(j) < akey(i))) ++j;
        if (j < P * P) {
            used[j] = true;
            out[n++] = (uint16_t)((i % P) | (i / P) << 4 | (j % P) << 8 | (j / P) << 12);
        } else {
            out[n++] = (uint16_t)((i % P) | (i / P) << 4 | 15 << 8 | 15 << 12);
        }
    }
    return n;
}

}  // namespace

// *handled = false (nothing launched) unless the batch is six-channel, squared
// L2, patches up to 15 x 15, and a CTA's staging fits in shared memory.
pgm_status launch_init_tc(const LvlBatch& B, const MatchConst& mc, int nch, bool* handled,
                          cudaStream_t st, int* nlaunch) {
    *handled = false;
    if (nch != 6 || mc.norm != PGM_L2SQ || mc.sigma < 1 || B.n < 1) return PGM_OK;
    int P[2] = {0, 0}, units = 0, ctas = 0, seeds = 0;
    for (int k = 0; k < B.n; ++k)
        for (int d = 0; d < 2; ++d) {
            const DirLvl& D = B.d[k][d];
            if (D.P < 1 || D.P > TC_MAXP || (P[d] && P[d] != D.P)) return PGM_OK;
            if ((long long)D.tw * D.th >= (1ll << 24) || !D.sa2img || !D.sb2) return PGM_OK;
            P[d] = D.P;
            const TcGeom g = tc_geom(D, mc.sigma);
            units = std::max(units, tc_units(g));
            ctas = std::max(ctas, g.ctas);
            seeds = std::max(seeds, D.nx * D.ny);
        }
    if (16L * units > 200L * 1024) return PGM_OK;
    TcPairs T;
    memset(&T, 0, sizeof(T));
    for (int d = 0; d < 2; ++d) T.n[d] = tc_pairs(P[d], mc.sigma, T.pr[d]);
    *handled = true;
    if (seeds == 0) return PGM_OK;
    if (pgm_status r = smem_opt_in((const void*)k_init_tc); r != PGM_OK) return r;
    const dim3 gs((seeds + 255) / 256, 2, B.n);
    k_init_tc_clear<<<gs, 256, 0, st>>>(B);
    k_init_tc<<<dim3(ctas, B.n, 2), TC_THREADS, 16 * units, st>>>(B, mc, T, wait_limit());
    k_init_tc_fin<<<gs, 256, 0, st>>>(B, mc);
    *nlaunch = 3;
    return launch_status("init (tensor cores): launch");
}

}  // namespace pgm
