// pyramid.cu -- gradient pyramid of one image on the GPU.
//
// Steps (one kernel each, all integer, all HBM/L2-streaming):
//   level 0: gray conversion (PGM-G/GD, Sec. III-F) or RGB de-interleave
//   levels 1..L-1: 5x5 binomial [1 4 6 4 1]^2 / 256 with decimation by 2 and
//            replicated border (Sec. III-D, downsample factor s = 1/2)
//   per level and direction: colour space of Table 2 (Sec. III-E): RGB,
//            CIELab or YCrCb, integer definitions
//   per level and direction: Sobel gradients Gx, Gy (Eq. 1-2), S = 3 or 5,
//            replicated border, int16, pixel-interleaved; for the direction
//            descriptor (Sec. III-F) their signs.
#include <string.h>

#include "match_common.cuh"

namespace pgm {
namespace {

__device__ __forceinline__ int gray_q14(int r, int g, int b) {
    // BT.601 luma weights 0.299, 0.587, 0.114 in Q14 (sum 16384)
    return (4899 * r + 9617 * g + 1868 * b + 8192) >> 14;
}

// Every kernel takes a batch of images (blockIdx.z); the grid covers the
// largest image and blocks outside an image's extent return.

// ---------------------------------------------------------------- level 0
// mode 0: gray input copied; mode 1: RGB -> gray; mode 2: RGB -> 3 planes.
// A thread makes 4 consecutive pixels (one 32-bit store per output plane;
// level rows are 16-byte aligned).
__global__ void k_level0(const __grid_constant__ PyrBatch B) {
    const PyrItem& it = B.it[blockIdx.z];
    const int x = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= it.sw || y >= it.sh) return;
    const uint8_t* src = it.src + (size_t)y * it.pitch;
    uint8_t* out = it.dst;
    const size_t o = (size_t)y * it.drow + x;
    const int n = it.sw - x < 4 ? it.sw - x : 4;
    uint32_t p0 = 0, p1 = 0, p2 = 0;
    for (int k = 0; k < n; ++k) {
        if (it.mode == 0) {
            p0 |= (uint32_t)src[x + k] << (8 * k);
        } else {
            const int r = src[3 * (x + k)], g = src[3 * (x + k) + 1], b = src[3 * (x + k) + 2];
            if (it.mode == 1) {
                p0 |= (uint32_t)gray_q14(r, g, b) << (8 * k);
            } else {
                p0 |= (uint32_t)r << (8 * k);
                p1 |= (uint32_t)g << (8 * k);
                p2 |= (uint32_t)b << (8 * k);
            }
        }
    }
    if (n == 4) {
        *reinterpret_cast<uint32_t*>(out + o) = p0;
        if (it.mode == 2) {
            *reinterpret_cast<uint32_t*>(out + it.dplane + o) = p1;
            *reinterpret_cast<uint32_t*>(out + 2 * it.dplane + o) = p2;
        }
    } else {
        for (int k = 0; k < n; ++k) {
            out[o + k] = (uint8_t)(p0 >> (8 * k));
            if (it.mode == 2) {
                out[it.dplane + o + k] = (uint8_t)(p1 >> (8 * k));
                out[2 * it.dplane + o + k] = (uint8_t)(p2 >> (8 * k));
            }
        }
    }
}

// ------------------------------------------------------- binomial down
// One output pixel per thread; blockIdx.z = image * C + channel.  The
// separable sums are exact integers, so summing rows first equals the 2D sum
// of the definition.
__global__ void k_down(const __grid_constant__ PyrBatch B, int C) {
    const PyrItem& it = B.it[blockIdx.z / C];
    const int ch = blockIdx.z % C;
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= it.dw || y >= it.dh) return;
    const uint8_t* src = it.src + ch * it.splane;
    const int k[5] = {1, 4, 6, 4, 1};
    int xs[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) xs[i] = clampi(2 * x + i - 2, 0, it.sw - 1);
    int acc = 0;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        const uint8_t* r = src + (size_t)clampi(2 * y + j - 2, 0, it.sh - 1) * it.srow;
        int s = 0;
#pragma unroll
        for (int i = 0; i < 5; ++i) s += k[i] * r[xs[i]];
        acc += k[j] * s;
    }
    it.dst[ch * it.dplane + (size_t)y * it.drow + x] = (uint8_t)((acc + 128) >> 8);
}

// ------------------------------------------------------- colour spaces
// Integer cube root of v <= 2^48: the floor of a float estimate, then one
// exact correction step each way.  The estimate 2^(log2(v) / 3) from the
// fast base-2 logarithm and exponential (each documented within 2 units in
// the last place here; log2(v) < 49) is within about 2e-6 of the root
// relatively, so for roots below 2^17 its integer part is off by at most
// one.  All 2^24 colours are checked against the oracle on the GPU.
__device__ __forceinline__ uint32_t icbrt48(unsigned long long v) {
    int c = v ? (int)exp2f(__log2f((float)v) * (1.0f / 3.0f)) : 0;
    const unsigned long long cc = (unsigned long long)(unsigned)c * (unsigned)c;
    if (c > 0 && cc * (unsigned)c > v) --c;
    const unsigned n = (unsigned)c + 1u;
    if ((unsigned long long)n * n * n <= v) ++c;
    return (uint32_t)c;
}

// CIELab companding function of t = T / (255 * 2^16), result scaled by 2^16.
__device__ __forceinline__ long long lab_f(long long T) {
    if (T * 24389 > 216LL * 255 * 65536) {               // t > (6/29)^3
        // t * 2^48 = floor(T 2^32 / 255) = T (2^32 - 1) / 255 + floor(T / 255)
        const uint32_t t32 = (uint32_t)T;                 // T < 2^24
        const unsigned long long V = (unsigned long long)t32 * 16843009ull + t32 / 255u;
        return (long long)icbrt48(V);
    }
    long long num = T * (841 * 29) + 4LL * 65536 * 108 * 255;          // t * 841/108 + 4/29
    return num / (108LL * 255 * 29);                                    // num > 0
}

__device__ __forceinline__ long long fdiv(long long a, long long b) {  // floor, b > 0
    long long q = a / b;
    return (a % b != 0 && a < 0) ? q - 1 : q;
}

__device__ __forceinline__ void to_lab(int r, int g, int b, int* o) {
    // D65 RGB -> XYZ / white, Q16 rows summing to 65536, linear RGB
    long long X = 28439LL * r + 24656LL * g + 12441LL * b;
    long long Y = 13937LL * r + 46869LL * g + 4730LL * b;
    long long Z = 1164LL * r + 7175LL * g + 57197LL * b;
    long long fx = lab_f(X), fy = lab_f(Y), fz = lab_f(Z);
    long long Ls = fdiv((116 * fy - 16 * 65536) * 255 + 3276800, 6553600);
    long long As = (500 * (fx - fy) + 128 * 65536 + 32768) >> 16;      // floor division
    long long Bs = (200 * (fy - fz) + 128 * 65536 + 32768) >> 16;
    o[0] = clampi((int)Ls, 0, 255);
    o[1] = clampi((int)As, 0, 255);
    o[2] = clampi((int)Bs, 0, 255);
}

__device__ __forceinline__ void to_ycrcb(int r, int g, int b, int* o) {
    int y = gray_q14(r, g, b);
    o[0] = y;
    o[1] = clampi(((r - y) * 11682 + (128 << 14) + 8192) >> 14, 0, 255);   // floor division
    o[2] = clampi(((b - y) * 9241 + (128 << 14) + 8192) >> 14, 0, 255);
}

__global__ void k_convert(const __grid_constant__ PyrBatch B) {
    const PyrItem& it = B.it[blockIdx.z];
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= it.sw || y >= it.sh) return;
    const size_t o = (size_t)y * it.srow + x, plane = it.splane;
    int r = it.src[o], g = it.src[plane + o], b = it.src[2 * plane + o];
    int v[3];
    if (it.mode == SP_LAB) to_lab(r, g, b, v); else to_ycrcb(r, g, b, v);
    it.dst[o] = (uint8_t)v[0];
    it.dst[plane + o] = (uint8_t)v[1];
    it.dst[2 * plane + o] = (uint8_t)v[2];
}

// ----------------------------------------------------------------- Sobel
// Gx = sum_j s_j sum_i d_i I(x+i, y+j); Gy with the roles of the axes swapped.
// A CTA of 32 x 8 threads makes a 32 x 16 block of one image (two rows per
// thread).  The (32 + S - 1) x (16 + S - 1) input pixels of every channel
// (border replicated) go to shared memory, as aligned 32-bit words for blocks
// away from the left and right borders; the horizontal passes (d and s along
// x, both within int16) are kept per input row as one packed word, and the
// vertical passes finish Gx and Gy (separable and exact in integers).  The
// output words (px_words per pixel: 3 data words and a zero word for colour,
// one word for gray) are staged in shared memory and leave as contiguous
// 16-byte stores, one tile row of each output array at a time.  A block at an
// image edge also writes the replicated border of BORD pixels next to it (a
// border pixel repeats the descriptor of the nearest image pixel, which the
// block holds), so every patch with its centre in the image can be read
// without clamping.
constexpr int SB_TW = 32, SB_TH = 16, SB_TY = 8, SB_XO = 4;   // SB_XO: staged columns left of x0
__device__ __forceinline__ int sb_d(int S, int i) {
    return S == 5 ? (i == 0 ? -1 : i == 1 ? -2 : i == 2 ? 0 : i == 3 ? 2 : 1) : (i - 1);
}
__device__ __forceinline__ int sb_s(int S, int i) {
    return S == 5 ? (i == 0 ? 1 : i == 1 ? 4 : i == 2 ? 6 : i == 3 ? 4 : 1) : (i == 1 ? 2 : 1);
}
template <int S, int C>
__global__ void __launch_bounds__(SB_TW * SB_TY) k_sobel(const __grid_constant__ PyrBatch B,
                                                         int dir_only) {
    constexpr int R = S / 2, IH = SB_TH + S - 1;
    constexpr int IWW = (SB_XO + SB_TW + R + 3) / 4;     // staged words per row (x0 - 4 .. )
    constexpr int IW = 4 * IWW, NT = SB_TW * SB_TY;
    constexpr int PXW = px_words(2 * C);                 // words per pixel in the output arrays
    constexpr int OW = SB_TW * PXW;                      // output words per tile row and array
    __shared__ __align__(16) uint8_t sI[C][IH][IW];      // column c holds x = x0 - SB_XO + c
    __shared__ uint32_t sH[C][IH][SB_TW];                // (sum d v) low 16, (sum s v) high 16
    __shared__ __align__(16) uint32_t sO[2][SB_TH][OW];  // descriptor words, split words
    const PyrItem& it = B.it[blockIdx.z];
    const int w = it.sw, h = it.sh, row = it.srow;
    const int x0 = blockIdx.x * SB_TW, y0 = blockIdx.y * SB_TH;
    if (x0 >= w || y0 >= h) return;                     // the whole block (uniform)
    const size_t plane = it.splane;
    const uint8_t* in = it.src;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * SB_TW + tx;
    if (x0 >= SB_XO && x0 + SB_TW + R <= w) {
        // interior in x: rows start 16-byte aligned and x0 - SB_XO is a
        // multiple of 4, so whole words are read; the words end inside the
        // padded row (x0 - 4 + IW <= row)
        for (int e = tid; e < C * IH * IWW; e += NT) {
            const int ch = e / (IH * IWW), rem = e - ch * (IH * IWW), r = rem / IWW, k = rem - r * IWW;
            const uint8_t* src = in + ch * plane + (size_t)clampi(y0 - R + r, 0, h - 1) * row;
            *reinterpret_cast<uint32_t*>(&sI[ch][r][4 * k]) =
                *reinterpret_cast<const uint32_t*>(src + x0 - SB_XO + 4 * k);
        }
    } else {
        for (int e = tid; e < C * IH * IW; e += NT) {
            const int ch = e / (IH * IW), rem = e - ch * (IH * IW), r = rem / IW, c = rem - r * IW;
            const uint8_t* src = in + ch * plane + (size_t)clampi(y0 - R + r, 0, h - 1) * row;
            sI[ch][r][c] = src[clampi(x0 - SB_XO + c, 0, w - 1)];
        }
    }
    __syncthreads();
    for (int r = ty; r < IH; r += SB_TY)
#pragma unroll
        for (int ch = 0; ch < C; ++ch) {
            int sd = 0, ss = 0;
#pragma unroll
            for (int i = 0; i < S; ++i) {
                const int v = sI[ch][r][SB_XO - R + tx + i];
                sd += sb_d(S, i) * v;
                ss += sb_s(S, i) * v;
            }
            sH[ch][r][tx] = (uint32_t)(uint16_t)sd | ((uint32_t)ss << 16);
        }
    __syncthreads();
    int g[2][2 * C];
#pragma unroll
    for (int ch = 0; ch < C; ++ch) {
        int gx0 = 0, gy0 = 0, gx1 = 0, gy1 = 0;
#pragma unroll
        for (int j = 0; j <= S; ++j) {                  // rows 2 ty .. 2 ty + S
            const uint32_t v = sH[ch][2 * ty + j][tx];
            const int sd = (int)(int16_t)(v & 0xffffu), ss = (int)(v >> 16);
            if (j < S) { gx0 += sb_s(S, j) * sd; gy0 += sb_d(S, j) * ss; }
            if (j > 0) { gx1 += sb_s(S, j - 1) * sd; gy1 += sb_d(S, j - 1) * ss; }
        }
        int gx[2] = {gx0, gx1}, gy[2] = {gy0, gy1};
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            int a = gx[k], b2 = gy[k];
            if (dir_only == 1) {                  // direction only: G ./ |G|
                a = (a > 0) - (a < 0);
                b2 = (b2 > 0) - (b2 < 0);
            } else if (dir_only == 2) {           // 8-sector angle as an integer unit vector
                const int ax = abs(a), ay = abs(b2);
                int cx, cy;
                if (a == 0 && b2 == 0) { cx = 0; cy = 0; }
                else if (408 * ay <= 169 * ax) { cx = a > 0 ? 64 : -64; cy = 0; }
                else if (408 * ax <= 169 * ay) { cx = 0; cy = b2 > 0 ? 64 : -64; }
                else { cx = a > 0 ? 45 : -45; cy = b2 > 0 ? 45 : -45; }
                a = cx; b2 = cy;
            }
            g[k][ch] = a;
            g[k][C + ch] = b2;
        }
    }
    // pixel-interleaved int16 as 32-bit words (2C is even), and the same
    // words with every value a split into signed bytes a = 128 a_h + a_l
    // (a_l in [-64, 63]) for the dp2a cross products
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int q = 0; q < PXW; ++q) {
            const bool dw = q < C;
            sO[0][2 * ty + k][tx * PXW + q] =
                dw ? (uint32_t)(uint16_t)g[k][2 * q] | ((uint32_t)(uint16_t)g[k][2 * q + 1] << 16) : 0u;
            sO[1][2 * ty + k][tx * PXW + q] = dw ? (uint32_t)split_bytes(g[k][2 * q], g[k][2 * q + 1]) : 0u;
        }
    __syncthreads();
    // dst and split point at pixel (0, 0) of padded arrays with rows of rw
    // words (a multiple of 4); pixel (x, y) starts at word y rw + x PXW, and
    // x0 PXW is a multiple of 32 words, so tile rows are 16-byte aligned
    const ptrdiff_t rw = (ptrdiff_t)(it.drow >> 1);
    uint32_t* const dst0 = reinterpret_cast<uint32_t*>(it.dst);
    uint32_t* const dst1 = it.split;
    // this block's output: its tile, widened by the border where it touches
    // an image edge
    const bool left = x0 == 0, right = x0 + SB_TW >= w, top = y0 == 0, bottom = y0 + SB_TH >= h;
    const int xa = left ? -BORD : x0, xb = right ? w + BORD : x0 + SB_TW;
    const int ya = top ? -BORD : y0, yb = bottom ? h + BORD : y0 + SB_TH;
    if (!(left || right || top || bottom)) {
        constexpr int NQ = OW / 4;
        for (int e = tid; e < 2 * SB_TH * NQ; e += NT) {
            const int a = e / (SB_TH * NQ), rem = e - a * (SB_TH * NQ), r = rem / NQ, q = rem - r * NQ;
            const uint4 v = *reinterpret_cast<const uint4*>(&sO[a][r][4 * q]);
            *reinterpret_cast<uint4*>((a ? dst1 : dst0) + (ptrdiff_t)(y0 + r) * rw +
                                      (ptrdiff_t)x0 * PXW + 4 * q) = v;
        }
    } else {
        // a border pixel takes the words of the nearest image pixel, which
        // lies in this tile; a warp walks one output row, a pixel per lane
        // (colour pixels as one 16-byte store)
        const int nx = xb - xa, nrow = yb - ya;
        for (int r = ty; r < 2 * nrow; r += SB_TY) {
            const int a = r >= nrow, y = ya + (a ? r - nrow : r);
            const int sy = clampi(y, 0, h - 1) - y0;
            uint32_t* const orow = (a ? dst1 : dst0) + (ptrdiff_t)y * rw;
            for (int i = tx; i < nx; i += SB_TW) {
                const int x = xa + i, sx = clampi(x, 0, w - 1) - x0;
                if constexpr (PXW == 4) {
                    *reinterpret_cast<uint4*>(orow + (ptrdiff_t)x * 4) =
                        *reinterpret_cast<const uint4*>(&sO[a][sy][sx * 4]);
                } else {
#pragma unroll
                    for (int q = 0; q < PXW; ++q) orow[(ptrdiff_t)x * PXW + q] = sO[a][sy][sx * PXW + q];
                }
            }
        }
    }
}

// ------------------------------------------------- direction bit-planes
// For the direction descriptor: word w of padded row yy of the nonzero and
// the sign bit-plane from the padded descriptor (bit b = x nch + c holds
// value c of padded pixel x; words past the row are zero).  One thread per
// word of one image (blockIdx.z).
template <int NCH>
__global__ void k_bits(const __grid_constant__ PyrBatch B) {
    constexpr int PXE = 2 * px_words(NCH);       // int16 elements per padded pixel
    const PyrItem& it = B.it[blockIdx.z];
    const int w = blockIdx.x * blockDim.x + threadIdx.x, yy = blockIdx.y * blockDim.y + threadIdx.y;
    const int pw = it.sw + 2 * BORD, ph = it.sh + 2 * BORD;
    if (w >= it.brow || yy >= ph) return;
    // padded pixel x of row yy: it.dst points at pixel (0, 0), rows drow int16
    const int16_t* row = reinterpret_cast<const int16_t*>(it.dst) + (ptrdiff_t)(yy - BORD) * it.drow -
                         (ptrdiff_t)BORD * PXE;
    uint32_t nz = 0, sg = 0;
    const int b0 = 32 * w, x0 = b0 / NCH, x1 = min((b0 + 31) / NCH, pw - 1);
    for (int x = x0; x <= x1; ++x) {           // whole pixels, one vector load each
        int v[NCH];
        if constexpr (NCH == 6) {
            const uint4 q = *reinterpret_cast<const uint4*>(row + (ptrdiff_t)x * PXE);
            v[0] = (int16_t)(q.x & 0xffff); v[1] = (int16_t)(q.x >> 16);
            v[2] = (int16_t)(q.y & 0xffff); v[3] = (int16_t)(q.y >> 16);
            v[4] = (int16_t)(q.z & 0xffff); v[5] = (int16_t)(q.z >> 16);
        } else {
            const uint32_t q = *reinterpret_cast<const uint32_t*>(row + (ptrdiff_t)x * PXE);
            v[0] = (int16_t)(q & 0xffff); v[1] = (int16_t)(q >> 16);
        }
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            const int k = x * NCH + c - b0;
            if (k < 0 || k >= 32) continue;
            nz |= (uint32_t)(v[c] != 0) << k;
            sg |= (uint32_t)(v[c] < 0) << k;
        }
    }
    it.bits[(size_t)yy * it.brow + w] = nz;
    it.bits[(size_t)(ph + yy) * it.brow + w] = sg;
}

}  // namespace

// One launch per step of the pyramid for a whole batch of images (all with
// the same parameters; sizes may differ).
pgm_status launch_pyramid_batch(const pgm_params* p, int n, const PyrPlan* plans,
                                const uint8_t* const* imgs, const int* cs, const size_t* pitches,
                                uint8_t* const* pyrs, cudaStream_t st) {
    static thread_local PyrBatch B;
    const PyrPlan& p0 = plans[0];
    const int L = p0.L, C = p0.C, nsch = p0.nsch;
    dim3 blk(32, 8);
    auto grid = [&](int w, int h, int z) { return dim3((w + 31) / 32, (h + 7) / 8, z); };
    const int dir_only = p->descriptor;      // 0 full, 1 signs, 2 sectors
    for (int base = 0; base < n; base += PYR_MAXB) {
        const int m = n - base < PYR_MAXB ? n - base : PYR_MAXB;
        int nlaunch = L + nsch * L * (dir_only == 1 ? 2 : 1);
        for (int s = 0; s < nsch; ++s)
            for (int l = 0; l < L; ++l)
                nlaunch += p0.space[s][l] == SP_LAB || p0.space[s][l] == SP_YCRCB;
        KScope ks(PGM_K_PYRAMID, st, nlaunch);
        // level 0
        int mw = 0, mh = 0;
        memset(&B, 0, sizeof(B));
        B.n = m;
        for (int k = 0; k < m; ++k) {
            const PyrPlan& pp = plans[base + k];
            PyrItem& it = B.it[k];
            it.src = imgs[base + k]; it.pitch = pitches[base + k];
            it.sw = pp.W[0]; it.sh = pp.H[0];
            it.dst = pyrs[base + k] + pp.img_off[0]; it.drow = pp.img_row[0];
            it.dplane = pp.img_plane[0];
            it.mode = cs[base + k] == 1 ? 0 : (C == 1 ? 1 : 2);
            mw = pp.W[0] > mw ? pp.W[0] : mw; mh = pp.H[0] > mh ? pp.H[0] : mh;
        }
        k_level0<<<grid((mw + 3) / 4, mh, m), blk, 0, st>>>(B);
        for (int l = 1; l < L; ++l) {
            mw = mh = 0;
            for (int k = 0; k < m; ++k) {
                const PyrPlan& pp = plans[base + k];
                const uint8_t* pyr = pyrs[base + k];
                PyrItem& it = B.it[k];
                it.src = pyr + pp.img_off[l - 1]; it.sw = pp.W[l - 1]; it.sh = pp.H[l - 1];
                it.srow = pp.img_row[l - 1]; it.splane = pp.img_plane[l - 1];
                it.dst = pyrs[base + k] + pp.img_off[l]; it.dw = pp.W[l]; it.dh = pp.H[l];
                it.drow = pp.img_row[l]; it.dplane = pp.img_plane[l];
                mw = pp.W[l] > mw ? pp.W[l] : mw; mh = pp.H[l] > mh ? pp.H[l] : mh;
            }
            k_down<<<grid(mw, mh, m * C), blk, 0, st>>>(B, C);
        }
        for (int s = 0; s < nsch; ++s)
            for (int l = 0; l < L; ++l) {
                const int sp = p0.space[s][l];
                mw = mh = 0;
                for (int k = 0; k < m; ++k) {
                    const PyrPlan& pp = plans[base + k];
                    mw = pp.W[l] > mw ? pp.W[l] : mw; mh = pp.H[l] > mh ? pp.H[l] : mh;
                }
                if (sp == SP_LAB || sp == SP_YCRCB) {
                    for (int k = 0; k < m; ++k) {
                        const PyrPlan& pp = plans[base + k];
                        PyrItem& it = B.it[k];
                        it.src = pyrs[base + k] + pp.img_off[l]; it.sw = pp.W[l]; it.sh = pp.H[l];
                        it.srow = pp.img_row[l]; it.splane = pp.img_plane[l];
                        it.dst = pyrs[base + k] + pp.cimg_off[s][l];
                        it.mode = sp;
                    }
                    k_convert<<<grid(mw, mh, m), blk, 0, st>>>(B);
                }
                for (int k = 0; k < m; ++k) {
                    const PyrPlan& pp = plans[base + k];
                    PyrItem& it = B.it[k];
                    it.src = pyrs[base + k] + pp.cimg_off[s][l]; it.sw = pp.W[l]; it.sh = pp.H[l];
                    it.srow = pp.img_row[l]; it.splane = pp.img_plane[l];
                    it.dst = pyrs[base + k] + pp.desc_off[s][l]; it.drow = pp.desc_row[l];
                    it.split = reinterpret_cast<uint32_t*>(pyrs[base + k] + pp.split_off[s][l]);
                }
                dim3 g((mw + SB_TW - 1) / SB_TW, (mh + SB_TH - 1) / SB_TH, m);
                const dim3 sblk(SB_TW, SB_TY);
                if (p->sobel == 5) {
                    if (C == 1) k_sobel<5, 1><<<g, sblk, 0, st>>>(B, dir_only);
                    else k_sobel<5, 3><<<g, sblk, 0, st>>>(B, dir_only);
                } else {
                    if (C == 1) k_sobel<3, 1><<<g, sblk, 0, st>>>(B, dir_only);
                    else k_sobel<3, 3><<<g, sblk, 0, st>>>(B, dir_only);
                }
                if (dir_only == 1) {                   // the sign codes as bit-planes
                    int mb = 0;
                    for (int k = 0; k < m; ++k) {
                        const PyrPlan& pp = plans[base + k];
                        PyrItem& it = B.it[k];
                        it.bits = reinterpret_cast<uint32_t*>(pyrs[base + k] + pp.bits_off[s][l]);
                        it.brow = pp.bit_row[l];
                        mb = pp.bit_row[l] > mb ? pp.bit_row[l] : mb;
                    }
                    const dim3 gb((mb + 31) / 32, (mh + 2 * BORD + 7) / 8, m);
                    if (C == 3) k_bits<6><<<gb, dim3(32, 8), 0, st>>>(B);
                    else k_bits<2><<<gb, dim3(32, 8), 0, st>>>(B);
                }
            }
        if (pgm_status r = launch_status("pyramid: launch"); r != PGM_OK) return r;
    }
    return PGM_OK;
}

}  // namespace pgm
