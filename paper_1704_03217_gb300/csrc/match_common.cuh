// match_common.cuh -- device helpers shared by the matching kernels.
#pragma once
#include "pgm_device.cuh"

namespace pgm {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr unsigned long long INF = ~0ull;

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }
__device__ __forceinline__ int lo16(uint32_t v) { return (int)(int16_t)(v & 0xffffu); }
__device__ __forceinline__ int hi16(uint32_t v) { return ((int)v) >> 16; }
__device__ __forceinline__ int32_t pack_u(int ux, int uy) {
    return (int32_t)(((uint32_t)ux & 0xffffu) | ((uint32_t)uy << 16));
}

// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of two 32x32->64 products,
// key bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// offset of the k-th limited random-search candidate (Eq. 5)
__device__ __forceinline__ int rs_off(uint32_t r, int k, int W, int mode) {
    if (mode == PGM_RS_SYMMETRIC) {
        int rho = max(1, W >> k);
        return (int)(((unsigned long long)r * (unsigned long long)(2 * rho + 1)) >> 32) - rho;
    }
    long long num = ((long long)r * 2 - 4294967295LL) * (long long)W;
    return (int)(num >> (32 + k));      // arithmetic shift = floor division by 2^(32+k)
}

__device__ __forceinline__ bool inside(const DirLvl& D, int qx, int qy) {
    return qx >= 0 && qy >= 0 && qx < D.tw && qy < D.th;
}

template <int MMAX>
struct XRef {
    int b[MMAX];      // signed bytes (a_l of word half 0, a_l half 1, a_h half 0, a_h half 1)
};

__device__ __forceinline__ int split_bytes(int a0, int a1) {
    const int l0 = ((a0 + 64) & 127) - 64, l1 = ((a1 + 64) & 127) - 64;
    const int h0 = (a0 - l0) >> 7, h1 = (a1 - l1) >> 7;
    return (int)((uint32_t)(l0 & 0xff) | ((uint32_t)(l1 & 0xff) << 8) |
                 ((uint32_t)(h0 & 0xff) << 16) | ((uint32_t)(h1 & 0xff) << 24));
}

__device__ __forceinline__ unsigned long long xcost(unsigned long long sa2, unsigned long long sb2,
                                                    long long cross) {
    return (unsigned long long)((long long)(sa2 + sb2) - 2 * cross);
}

}  // namespace
}  // namespace pgm
