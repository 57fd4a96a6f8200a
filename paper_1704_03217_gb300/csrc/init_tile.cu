// init_tile.cu -- exhaustive nearest-neighbour initialisation at the
// coarsest level for the squared-L2 cost: every seed starts from the target
// centre of least patch distance (Eq. 3) over the whole target image, ties to
// the smaller raster index (y, then x).
//
// D(s, q) = sum |a|^2 + sum |b|^2 - 2 <a, b>: the two sums come from the box
// filters of the same visit, the cross terms from dp2a products of the target
// words (two int16 values) with the seed's reference words in split-byte form
// (a = 128 a_h + a_l).  A CTA takes IN_SB seeds of one direction of one pair
// and every target centre.  The whole target image, with a border of P / 2
// replicated, and the seeds' reference patches sit in shared memory; a thread
// scores IN_PB centres against the IN_SB seeds at once (4 x 2 measured best
// of 2 x 4, 1 x 4, 1 x 8), each target word
// loaded once for all seeds and each reference word (a broadcast) once for
// all centres.  A patch row is summed in 32 bits (at most 48 words: below
// 2^31 for any descriptor value), the rows in 64 bits.
#include "match_common.cuh"

namespace pgm {
namespace {

constexpr int IN_SB = 2, IN_PB = 4, IN_THREADS = 256;

// shared words: target image with border, then IN_SB reference patches
__host__ __device__ inline int in_words(int nch, int P, int tw, int th) {
    const int wpp = nch / 2;
    return (tw + P - 1) * (th + P - 1) * wpp + IN_SB * P * P * wpp;
}

template <int NCH>
__global__ void __launch_bounds__(IN_THREADS) k_init_t(const __grid_constant__ LvlBatch B,
                                                       const MatchConst mc) {
    constexpr int WPP = NCH / 2;
    extern __shared__ __align__(16) uint32_t sm[];
    __shared__ unsigned long long s_cost[IN_THREADS / 32][IN_SB];
    __shared__ int s_q[IN_THREADS / 32][IN_SB];
    const int pair = blockIdx.z, dir = blockIdx.y;
    const DirLvl& D = B.d[pair][dir];
    const int ns = D.nx * D.ny, s0 = blockIdx.x * IN_SB;
    if (s0 >= ns) return;
    const int P = D.P, h = P / 2, sig = mc.sigma;
    const int tpw = D.tw + P - 1, tph = D.th + P - 1, tp = tpw * WPP, prw = P * WPP;
    const int rw = P * prw;                                // words of one reference patch
    uint32_t* sT = sm;
    uint32_t* sR = sm + tph * tp;

    const uint32_t* t32 = reinterpret_cast<const uint32_t*>(D.tgt);
    const int tpitch = D.tgt_pitch >> 1;
    for (int e = threadIdx.x; e < tph * tp; e += IN_THREADS) {
        const int r = e / tp, c = e - r * tp, px = c / WPP, wi = c - px * WPP;
        const int x = clampi(px - h, 0, D.tw - 1), y = clampi(r - h, 0, D.th - 1);
        sT[e] = __ldg(t32 + (size_t)y * tpitch + (size_t)x * px_words(NCH) + wi);
    }
    const int rpitch = D.ref_pitch >> 1;
    for (int e = threadIdx.x; e < IN_SB * rw; e += IN_THREADS) {
        const int k = e / rw, i = e - k * rw, row = i / prw, c = i - row * prw;
        const int px = c / WPP, wi = c - px * WPP;
        const int s = min(s0 + k, ns - 1);                 // a missing seed repeats the last
        const int si = s % D.nx, sj = s / D.nx;
        const int x = clampi(mc.c + sig * si + px - h, 0, D.rw - 1);
        const int y = clampi(mc.c + sig * sj + row - h, 0, D.rh - 1);
        sR[e] = __ldg(D.ref_split + (size_t)y * rpitch + (size_t)x * px_words(NCH) + wi);
    }
    __syncthreads();

    unsigned long long sa[IN_SB], bc[IN_SB];
    int bq[IN_SB];
#pragma unroll
    for (int k = 0; k < IN_SB; ++k) {
        const int s = min(s0 + k, ns - 1), si = s % D.nx, sj = s / D.nx;
        sa[k] = D.sa2img[(size_t)(mc.c + sig * sj) * D.rw + (mc.c + sig * si)];
        bc[k] = INF;
        bq[k] = 0;
    }
    const int nq = D.tw * D.th;
    for (int q0 = threadIdx.x; q0 < nq; q0 += IN_THREADS * IN_PB) {
        int base[IN_PB];
#pragma unroll
        for (int p = 0; p < IN_PB; ++p) {
            const int q = min(q0 + p * IN_THREADS, nq - 1);
            const int qx = q % D.tw, qy = q / D.tw;
            base[p] = qy * tp + qx * WPP;                  // patch corner in the staged image
        }
        long long acc[IN_PB][IN_SB];
#pragma unroll
        for (int p = 0; p < IN_PB; ++p)
#pragma unroll
            for (int k = 0; k < IN_SB; ++k) acc[p][k] = 0;
        for (int r = 0; r < P; ++r) {
            int lo[IN_PB][IN_SB], hi[IN_PB][IN_SB];
#pragma unroll
            for (int p = 0; p < IN_PB; ++p)
#pragma unroll
                for (int k = 0; k < IN_SB; ++k) { lo[p][k] = 0; hi[p][k] = 0; }
            const uint32_t* rrow = sR + r * prw;
#pragma unroll 3
            for (int c = 0; c < prw; ++c) {
                int tv[IN_PB];
#pragma unroll
                for (int p = 0; p < IN_PB; ++p) tv[p] = (int)sT[base[p] + r * tp + c];
#pragma unroll
                for (int k = 0; k < IN_SB; ++k) {
                    const int a = (int)rrow[k * rw + c];
#pragma unroll
                    for (int p = 0; p < IN_PB; ++p) {
                        lo[p][k] = __dp2a_lo(tv[p], a, lo[p][k]);
                        hi[p][k] = __dp2a_hi(tv[p], a, hi[p][k]);
                    }
                }
            }
#pragma unroll
            for (int p = 0; p < IN_PB; ++p)
#pragma unroll
                for (int k = 0; k < IN_SB; ++k)
                    acc[p][k] += (long long)hi[p][k] * 128 + (long long)lo[p][k];
        }
#pragma unroll
        for (int p = 0; p < IN_PB; ++p) {
            const int q = q0 + p * IN_THREADS;
            if (q >= nq) continue;
            const unsigned long long sb = D.sb2[(size_t)(q / D.tw) * D.sbp + q % D.tw];
#pragma unroll
            for (int k = 0; k < IN_SB; ++k) {
                const unsigned long long c = xcost(sa[k], sb, acc[p][k]);
                if (c < bc[k] || (c == bc[k] && q < bq[k])) { bc[k] = c; bq[k] = q; }
            }
        }
    }
    // least (cost, raster index) per seed over the CTA
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < IN_SB; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long c = __shfl_xor_sync(FULL, bc[k], o);
            const int q = __shfl_xor_sync(FULL, bq[k], o);
            if (c < bc[k] || (c == bc[k] && q < bq[k])) { bc[k] = c; bq[k] = q; }
        }
        if (lane == 0) { s_cost[warp][k] = bc[k]; s_q[warp][k] = bq[k]; }
    }
    __syncthreads();
    if (threadIdx.x < IN_SB && s0 + (int)threadIdx.x < ns) {
        const int k = threadIdx.x, s = s0 + k;
        unsigned long long c = s_cost[0][k];
        int q = s_q[0][k];
        for (int w = 1; w < IN_THREADS / 32; ++w)
            if (s_cost[w][k] < c || (s_cost[w][k] == c && s_q[w][k] < q)) { c = s_cost[w][k]; q = s_q[w][k]; }
        const int si = s % D.nx, sj = s / D.nx;
        D.u[s] = pack_u(q % D.tw - (mc.c + sig * si), q / D.tw - (mc.c + sig * sj));
        D.cost[s] = c;
        D.flags[s] = F_VALID;
    }
    if (threadIdx.x == 0) {
        const int nk = min(IN_SB, ns - s0);
        atomicAdd(B.evals[pair] + 4 + dir, (unsigned long long)nk * (unsigned long long)nq);
    }
}

template <int NCH>
pgm_status launch_in(const LvlBatch& B, const MatchConst& mc, int groups, int smem,
                     cudaStream_t st) {
    if (pgm_status r = smem_opt_in((const void*)k_init_t<NCH>); r != PGM_OK) return r;
    k_init_t<NCH><<<dim3(groups, 2, B.n), IN_THREADS, smem, st>>>(B, mc);
    return launch_status("init: launch");
}

// The same search for the direction descriptor on its bit-planes (every
// value a sign in {-1, 0, +1}): a 32-value word costs
// popc(nzA ^ nzB) + (popc(nzA & nzB & (sA ^ sB)) << f), f = 2 for the
// squared L2 cost and 1 for L1, exact in 32 bits.  A CTA takes IB_SB seeds;
// the target's padded planes (border replicated, so every centre inside the
// image reads without clamping) and the seeds' reference rows, shifted to
// start at bit 0, sit in shared memory.  A thread scores IN_PB centres
// against the seeds, each target row loaded once for all of them.
constexpr int IB_SB = 4;

template <int NCH>
__global__ void __launch_bounds__(IN_THREADS) k_init_b(const __grid_constant__ LvlBatch B,
                                                       const MatchConst mc) {
    constexpr int NR = NCH == 6 ? 3 : 1, NW = NR + 1;
    extern __shared__ __align__(16) uint32_t sm[];
    __shared__ unsigned s_cost[IN_THREADS / 32][IB_SB];
    __shared__ int s_q[IN_THREADS / 32][IB_SB];
    const int pair = blockIdx.z, dir = blockIdx.y;
    const DirLvl& D = B.d[pair][dir];
    const int ns = D.nx * D.ny, s0 = blockIdx.x * IB_SB;
    if (s0 >= ns) return;
    const int P = D.P, h = P / 2, sig = mc.sigma;
    const unsigned fac = mc.norm == PGM_L2SQ ? 2u : 1u;
    const int trow = D.tbit_row, tplane = trow * (D.th + 2 * BORD);
    uint32_t* sT = sm;                                   // nonzero rows, then sign rows
    uint32_t* sR = sm + 2 * tplane;                      // [seed][plane][row][NR]
    for (int e = threadIdx.x; e < 2 * tplane; e += IN_THREADS) sT[e] = __ldg(D.tgt_bits + e);
    const int rplane = D.rbit_row * (D.rh + 2 * BORD);
    for (int e = threadIdx.x; e < IB_SB * 2 * P; e += IN_THREADS) {
        const int k = e / (2 * P), pl = (e / P) & 1, r = e % P;
        const int s = min(s0 + k, ns - 1);                 // a missing seed repeats the last
        const int px = mc.c + sig * (s % D.nx), py = mc.c + sig * (s / D.nx);
        const int bit = (px - h + BORD) * NCH, sh = bit & 31;
        const uint32_t* row = D.ref_bits + pl * rplane + (size_t)(py - h + r + BORD) * D.rbit_row +
                              (bit >> 5);
        uint32_t v[NW];
#pragma unroll
        for (int i = 0; i < NW; ++i) v[i] = __ldg(row + i);
#pragma unroll
        for (int i = 0; i < NR; ++i) {
            const int nb = P * NCH - 32 * i;
            const uint32_t msk = nb <= 0 ? 0u : nb >= 32 ? 0xffffffffu : (1u << nb) - 1u;
            sR[((k * 2 + pl) * P + r) * NR + i] = __funnelshift_r(v[i], v[i + 1], sh) & msk;
        }
    }
    __syncthreads();
    unsigned bc[IB_SB];
    int bq[IB_SB];
#pragma unroll
    for (int k = 0; k < IB_SB; ++k) { bc[k] = 0xffffffffu; bq[k] = 0; }
    const int nq = D.tw * D.th;
    for (int q0 = threadIdx.x; q0 < nq; q0 += IN_THREADS * IN_PB) {
        int base[IN_PB], tsh[IN_PB];
        unsigned c[IN_PB][IB_SB];
#pragma unroll
        for (int p = 0; p < IN_PB; ++p) {
            const int q = min(q0 + p * IN_THREADS, nq - 1);
            const int qx = q % D.tw, qy = q / D.tw, bit = (qx - h + BORD) * NCH;
            base[p] = (qy - h + BORD) * trow + (bit >> 5);
            tsh[p] = bit & 31;
#pragma unroll
            for (int k = 0; k < IB_SB; ++k) c[p][k] = 0;
        }
        for (int r = 0; r < P; ++r) {
#pragma unroll
            for (int p = 0; p < IN_PB; ++p) {
                uint32_t vn[NW], vs[NW], tn[NR], ts[NR];
                const bool in = PGM_CHECK(base[p] >= 0 && base[p] + r * trow + NW <= tplane,
                                          B.err[pair]);
#pragma unroll
                for (int i = 0; i < NW; ++i) {
                    vn[i] = in ? sT[base[p] + r * trow + i] : 0u;
                    vs[i] = in ? sT[tplane + base[p] + r * trow + i] : 0u;
                }
#pragma unroll
                for (int i = 0; i < NR; ++i) {
                    tn[i] = __funnelshift_r(vn[i], vn[i + 1], tsh[p]);
                    ts[i] = __funnelshift_r(vs[i], vs[i + 1], tsh[p]);
                }
#pragma unroll
                for (int k = 0; k < IB_SB; ++k) {
                    const uint32_t* an = sR + ((k * 2) * P + r) * NR;
                    const uint32_t* as = sR + ((k * 2 + 1) * P + r) * NR;
#pragma unroll
                    for (int i = 0; i < NR; ++i) {
                        const uint32_t a = an[i];
                        const uint32_t msk = i < NR - 1 ? 0xffffffffu
                                             : (P * NCH - 32 * i >= 32 ? 0xffffffffu
                                                : (1u << (P * NCH - 32 * i)) - 1u);
                        c[p][k] += (unsigned)__popc((a ^ tn[i]) & msk) +
                                   ((unsigned)__popc(a & tn[i] & (as[i] ^ ts[i])) << fac);
                    }
                }
            }
        }
#pragma unroll
        for (int p = 0; p < IN_PB; ++p) {
            const int q = q0 + p * IN_THREADS;
            if (q >= nq) continue;
#pragma unroll
            for (int k = 0; k < IB_SB; ++k)
                if (c[p][k] < bc[k] || (c[p][k] == bc[k] && q < bq[k])) { bc[k] = c[p][k]; bq[k] = q; }
        }
    }
    // least (cost, raster index) per seed over the CTA
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < IB_SB; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned cc = __shfl_xor_sync(FULL, bc[k], o);
            const int q = __shfl_xor_sync(FULL, bq[k], o);
            if (cc < bc[k] || (cc == bc[k] && q < bq[k])) { bc[k] = cc; bq[k] = q; }
        }
        if (lane == 0) { s_cost[warp][k] = bc[k]; s_q[warp][k] = bq[k]; }
    }
    __syncthreads();
    if (threadIdx.x < IB_SB && s0 + (int)threadIdx.x < ns) {
        const int k = threadIdx.x, s = s0 + k;
        unsigned cc = s_cost[0][k];
        int q = s_q[0][k];
        for (int w = 1; w < IN_THREADS / 32; ++w)
            if (s_cost[w][k] < cc || (s_cost[w][k] == cc && s_q[w][k] < q)) { cc = s_cost[w][k]; q = s_q[w][k]; }
        const int si = s % D.nx, sj = s / D.nx;
        D.u[s] = pack_u(q % D.tw - (mc.c + sig * si), q / D.tw - (mc.c + sig * sj));
        D.cost[s] = cc;
        D.flags[s] = F_VALID;
    }
    if (threadIdx.x == 0) {
        const int nk = min(IB_SB, ns - s0);
        atomicAdd(B.evals[pair] + 4 + dir, (unsigned long long)nk * (unsigned long long)nq);
    }
}

template <int NCH>
pgm_status launch_ib(const LvlBatch& B, const MatchConst& mc, int groups, int smem,
                     cudaStream_t st) {
    if (pgm_status r = smem_opt_in((const void*)k_init_b<NCH>); r != PGM_OK) return r;
    k_init_b<NCH><<<dim3(groups, 2, B.n), IN_THREADS, smem, st>>>(B, mc);
    return launch_status("init: launch");
}

}  // namespace

// shared words of the bit-plane initialisation: the target's two padded
// planes and IB_SB seeds' reference rows
static int ib_words(const DirLvl& D) {
    return 2 * D.tbit_row * (D.th + 2 * BORD) + IB_SB * 2 * D.P * 3;
}

bool init_bits_fits(const LvlBatch& B) {
    for (int k = 0; k < B.n; ++k)
        for (int d = 0; d < 2; ++d) {
            const DirLvl& D = B.d[k][d];
            if (!D.ref_bits || !D.tgt_bits || D.rbit_row <= 0 || D.tbit_row <= 0 ||
                D.P > 2 * BORD + 1 || 4L * ib_words(D) > 200L * 1024)
                return false;
        }
    return true;
}

// *handled = false (nothing launched) when the cost is not squared L2 or a
// target image with its border does not fit in shared memory.
pgm_status launch_init_tile(const LvlBatch& B, const MatchConst& mc, int nch, bool* handled,
                            cudaStream_t st, int* nlaunch) {
    *handled = false;
    *nlaunch = 1;
    if (mc.descriptor == PGM_DIR && init_bits_fits(B)) {     // the bit-plane form, any norm
        int words = 0, seeds = 0;
        for (int k = 0; k < B.n; ++k)
            for (int d = 0; d < 2; ++d) {
                const DirLvl& D = B.d[k][d];
                const int w = ib_words(D);
                if (w > words) words = w;
                if (D.nx * D.ny > seeds) seeds = D.nx * D.ny;
            }
        {
            *handled = true;
            if (seeds == 0) return PGM_OK;
            const int groups = (seeds + IB_SB - 1) / IB_SB;
            return nch == 2 ? launch_ib<2>(B, mc, groups, 4 * words, st)
                            : launch_ib<6>(B, mc, groups, 4 * words, st);
        }
    }
    if (mc.norm != PGM_L2SQ) return PGM_OK;
    if (pgm_status r = launch_init_tc(B, mc, nch, handled, st, nlaunch); r != PGM_OK || *handled) return r;
    int words = 0, seeds = 0;
    for (int k = 0; k < B.n; ++k)
        for (int d = 0; d < 2; ++d) {
            const DirLvl& D = B.d[k][d];
            const int w = in_words(nch, D.P, D.tw, D.th);
            if (w > words) words = w;
            if (D.nx * D.ny > seeds) seeds = D.nx * D.ny;
        }
    if (4L * words > 200L * 1024) return PGM_OK;
    *handled = true;
    if (seeds == 0) return PGM_OK;
    const int groups = (seeds + IN_SB - 1) / IN_SB;
    return nch == 2 ? launch_in<2>(B, mc, groups, 4 * words, st)
                    : launch_in<6>(B, mc, groups, 4 * words, st);
}

}  // namespace pgm
