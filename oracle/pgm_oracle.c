/*
 * pgm_oracle.c -- plain, slow, single-threaded CPU oracle for Pyramidal
 * Gradient Matching (Li, arXiv 1704.03217).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, by the smoke check and by
 * the benchmark's CPU-baseline leg, never by the product path.  It shares no
 * code with the CUDA library.
 *
 * The code follows the paper's steps in the paper's order, with no blocking,
 * fusion or reordering.  Places where the paper is silent follow the written
 * readings R1..R20 of the design notes; each place names its reading.
 *
 * Parity status: every step is pinned by tests/test_oracle_*.py (closed
 * forms, invariants, brute force, published known-answer vectors), except the
 * end-to-end field of a full pyramid on a natural image, which no published
 * value fixes -- its pins are the invariants (bias, identity, integer
 * translation, fixed point) and the per-step brute-force checks.
 */
#include "pgm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define MAXL 16
#define INF_COST UINT64_MAX

/* ------------------------------------------------------------------ */
/* small helpers                                                      */
/* ------------------------------------------------------------------ */
static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* floor(a / b) for b > 0 */
static int64_t floordiv(int64_t a, int64_t b) {
    int64_t q = a / b;
    if ((a % b != 0) && (a < 0)) q -= 1;
    return q;
}

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11 "Parallel random    */
/* numbers: as easy as 1, 2, 3"), written from the published definition. */
/* The paper only asks for random offsets R_i (Sec. III-B, Eq. 5);      */
/* reading R11 fixes this counter-based stream.                         */
/* ------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * c0;
        uint64_t p1 = (uint64_t)M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------ */
/* Colour spaces (Sec. III-E, Table 2; Sec. III-F gray).  The paper     */
/* gives no formulas: readings R2 (gray, YCrCb) and R3 (CIELab).        */
/* ------------------------------------------------------------------ */
static int gray_of(int r, int g, int b) {             /* R2, BT.601 in Q14 */
    return (4899 * r + 9617 * g + 1868 * b + 8192) >> 14;
}

/* largest c with c^3 <= v, by bisection (v < 2^63) */
uint32_t orc_icbrt(uint64_t v) {
    uint64_t lo = 0, hi = 2097152; /* 2^21: hi^3 = 2^63 > v */
    while (hi - lo > 1) {
        uint64_t mid = (lo + hi) / 2;
        if (mid * mid * mid <= v) lo = mid; else hi = mid;
    }
    return (uint32_t)lo;
}

/* f(t) of CIELab scaled by 2^16, for t = T / (255 * 2^16) (R3) */
static int64_t lab_f16(int64_t T) {
    /* knee: t > (6/29)^3 = 216/24389 */
    if (T * 24389 > (int64_t)216 * 255 * 65536) {
        uint64_t V = ((uint64_t)T << 32) / 255u;     /* t * 2^48 */
        return (int64_t)orc_icbrt(V);                /* cbrt(t) * 2^16 */
    }
    /* f = t * 841/108 + 4/29 */
    int64_t num = T * 841 * 29 + (int64_t)4 * 65536 * 108 * 255;
    int64_t den = (int64_t)108 * 255 * 29;
    return floordiv(num, den);
}

static void lab_of(int r, int g, int b, uint8_t out[3]) {
    /* rows of the D65 RGB->XYZ matrix divided by the white point, Q16,
     * each row summing to 65536 (R3; no sRGB companding) */
    int64_t TX = (int64_t)28439 * r + 24656 * g + 12441 * b;
    int64_t TY = (int64_t)13937 * r + 46869 * g + 4730 * b;
    int64_t TZ = (int64_t)1164 * r + 7175 * g + 57197 * b;
    int64_t fx = lab_f16(TX), fy = lab_f16(TY), fz = lab_f16(TZ);
    /* L* = 116 f(Y) - 16, scaled to 0..255 with round half up */
    int64_t L = floordiv((116 * fy - 16 * 65536) * 255 + 3276800, 6553600);
    int64_t A = floordiv(500 * (fx - fy) + 128 * 65536 + 32768, 65536);
    int64_t B = floordiv(200 * (fy - fz) + 128 * 65536 + 32768, 65536);
    out[0] = (uint8_t)clampi((int)L, 0, 255);
    out[1] = (uint8_t)clampi((int)A, 0, 255);
    out[2] = (uint8_t)clampi((int)B, 0, 255);
}

static void ycrcb_of(int r, int g, int b, uint8_t out[3]) { /* R2 */
    int y = gray_of(r, g, b);
    int64_t cr = floordiv((int64_t)(r - y) * 11682 + (128 << 14) + 8192, 16384);
    int64_t cb = floordiv((int64_t)(b - y) * 9241 + (128 << 14) + 8192, 16384);
    out[0] = (uint8_t)y;
    out[1] = (uint8_t)clampi((int)cr, 0, 255);
    out[2] = (uint8_t)clampi((int)cb, 0, 255);
}

void orc_convert(int space, const uint8_t* rgb, int64_t n, uint8_t* out) {
    for (int64_t i = 0; i < n; ++i) {
        int r = rgb[3 * i], g = rgb[3 * i + 1], b = rgb[3 * i + 2];
        switch (space) {
        case ORC_SP_GRAY: out[i] = (uint8_t)gray_of(r, g, b); break;
        case ORC_SP_RGB: out[3 * i] = r; out[3 * i + 1] = g; out[3 * i + 2] = b; break;
        case ORC_SP_LAB: lab_of(r, g, b, out + 3 * i); break;
        default: ycrcb_of(r, g, b, out + 3 * i); break;
        }
    }
}

/* ------------------------------------------------------------------ */
/* Image pyramid, s = 1/2 (Sec. III-D; filter by reading R1):           */
/*   I^{l+1}(x,y) = (sum_{i,j} k_i k_j I^l(2x+i, 2y+j) + 128) >> 8      */
/*   k = [1 4 6 4 1], i,j in -2..2, replicated border,                  */
/*   W_{l+1} = ceil(W_l / 2).                                           */
/* ------------------------------------------------------------------ */
void orc_pyr_down(const uint8_t* in, int w, int h, uint8_t* out) {
    static const int k[5] = {1, 4, 6, 4, 1};
    int w2 = (w + 1) / 2, h2 = (h + 1) / 2;
    for (int y = 0; y < h2; ++y)
        for (int x = 0; x < w2; ++x) {
            int s = 0;
            for (int j = -2; j <= 2; ++j)
                for (int i = -2; i <= 2; ++i) {
                    int xx = clampi(2 * x + i, 0, w - 1), yy = clampi(2 * y + j, 0, h - 1);
                    s += k[i + 2] * k[j + 2] * in[yy * w + xx];
                }
            out[y * w2 + x] = (uint8_t)((s + 128) >> 8);
        }
}

/* ------------------------------------------------------------------ */
/* Sobel gradients, Eq. 1-2 (Sec. III-A); kernel by reading R4:         */
/*   Gx(x,y) = sum_j s_j sum_i d_i I(x+i, y+j), Gy with d along y,      */
/*   S=5: d=[-1 -2 0 2 1], s=[1 4 6 4 1]; S=3: d=[-1 0 1], s=[1 2 1];   */
/*   replicated border.                                                 */
/* ------------------------------------------------------------------ */
void orc_sobel(const uint8_t* in, int w, int h, int S, int16_t* gx, int16_t* gy) {
    static const int d5[5] = {-1, -2, 0, 2, 1}, s5[5] = {1, 4, 6, 4, 1};
    static const int d3[3] = {-1, 0, 1}, s3[3] = {1, 2, 1};
    const int* d = S == 5 ? d5 : d3;
    const int* s = S == 5 ? s5 : s3;
    int R = S / 2;
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            int sx = 0, sy = 0;
            for (int j = -R; j <= R; ++j)
                for (int i = -R; i <= R; ++i) {
                    int v = in[clampi(y + j, 0, h - 1) * w + clampi(x + i, 0, w - 1)];
                    sx += s[j + R] * d[i + R] * v;   /* derivative along x */
                    sy += d[j + R] * s[i + R] * v;   /* derivative along y */
                }
            gx[y * w + x] = (int16_t)sx;
            gy[y * w + x] = (int16_t)sy;
        }
}

/* Uniform 8-sector angle descriptor (an extension beyond the paper's two
 * descriptors): the angle of (gx, gy) is binned into 8 sectors of 45 degrees
 * centred on the axes and diagonals, by integer comparisons of |gx| and |gy|
 * against tan(22.5 deg) ~ 169/408 (boundaries go to the axis sectors); the
 * sector is coded as the integer unit vector 64 (cos, sin) of its centre,
 * (45, 45) on the diagonals; a zero gradient is (0, 0).  The squared L2 cost of
 * Eq. 3 then grows with the circular distance between sectors. */
void orc_sector(int gx, int gy, int16_t out[2]) {
    static const int16_t code[8][2] = {{64, 0}, {45, 45}, {0, 64}, {-45, 45},
                                       {-64, 0}, {-45, -45}, {0, -64}, {45, -45}};
    int ax = gx < 0 ? -gx : gx, ay = gy < 0 ? -gy : gy, s;
    if (gx == 0 && gy == 0) { out[0] = 0; out[1] = 0; return; }
    if (408 * ay <= 169 * ax) s = gx > 0 ? 0 : 4;
    else if (408 * ax <= 169 * ay) s = gy > 0 ? 2 : 6;
    else if (gx > 0) s = gy > 0 ? 1 : 7;
    else s = gy > 0 ? 3 : 5;
    out[0] = code[s][0]; out[1] = code[s][1];
}

/* ------------------------------------------------------------------ */
/* Patch distance D_r, Eq. 3 (Sec. III-B): the sum over the patch of the */
/* squared L2 norm of the gradient-vector difference (norm = 0), or the  */
/* L1 norm (norm = 1, reading R6).  Patch offsets -floor(P/2) ..        */
/* P-1-floor(P/2) (reading R7); patch pixels outside an image take the  */
/* nearest border pixel of that image.  Planar descriptors [nch][h][w]. */
/* ------------------------------------------------------------------ */
uint64_t orc_patch_dist(const int16_t* A, int wa, int ha, const int16_t* B, int wb, int hb,
                        int nch, int ax, int ay, int bx, int by, int P, int norm) {
    int lo = -(P / 2), hi = P - 1 - P / 2;
    uint64_t sum = 0;
    for (int oy = lo; oy <= hi; ++oy)
        for (int ox = lo; ox <= hi; ++ox) {
            int xa = clampi(ax + ox, 0, wa - 1), ya = clampi(ay + oy, 0, ha - 1);
            int xb = clampi(bx + ox, 0, wb - 1), yb = clampi(by + oy, 0, hb - 1);
            for (int c = 0; c < nch; ++c) {
                int64_t d = (int64_t)A[(int64_t)c * wa * ha + (int64_t)ya * wa + xa]
                          - (int64_t)B[(int64_t)c * wb * hb + (int64_t)yb * wb + xb];
                sum += (uint64_t)(norm == 0 ? d * d : (d < 0 ? -d : d));
            }
        }
    return sum;
}

/* Limited random-search offset for the k-th candidate (Eq. 5, reading R11).
 * mode 0: uniform on [-rho_k, rho_k], rho_k = max(1, floor(W / 2^k)).
 * mode 1: the literal floor(R W / 2^k) with R = (2r - (2^32-1)) / 2^32. */
int32_t orc_rs_offset(uint32_t r, int k, int W, int mode) {
    if (mode == 0) {
        int64_t rho = W >> k;
        if (rho < 1) rho = 1;
        return (int32_t)((((uint64_t)r * (uint64_t)(2 * rho + 1)) >> 32) - (uint64_t)rho);
    }
    int64_t num = ((int64_t)2 * r - (int64_t)4294967295LL) * (int64_t)W;
    return (int32_t)floordiv(num, (int64_t)1 << (32 + k));
}

/* ------------------------------------------------------------------ */
/* gradient pyramid                                                   */
/* ------------------------------------------------------------------ */
struct orc_pyr {
    orc_params prm;
    int L, C, nsch;
    int W[MAXL], H[MAXL];
    uint8_t* img[MAXL];          /* [C][H][W] */
    uint8_t* cimg[2][MAXL];      /* [C][H][W] */
    int16_t* desc[2][MAXL];      /* [2C][H][W] */
};

/* colour space of a level in a scheme (Table 2; reading R1 cycles it with
 * period 3 for L > 3).  Scheme 0 serves the forward field, scheme 1 the
 * backward field. */
static int space_of(const orc_params* p, int scheme, int level) {
    static const int fwd[3] = {ORC_SP_RGB, ORC_SP_LAB, ORC_SP_YCRCB};
    static const int bwd[3] = {ORC_SP_LAB, ORC_SP_YCRCB, ORC_SP_RGB};
    if (p->color == 0) return ORC_SP_GRAY;
    if (p->cs_sched != 0) return ORC_SP_RGB;
    return scheme == 0 ? fwd[level % 3] : bwd[level % 3];
}

orc_pyr* orc_pyr_build(const orc_params* p, const uint8_t* img, int w, int h, int c) {
    if (w < 1 || h < 1 || (c != 1 && c != 3) || p->levels < 1 || p->levels > MAXL) return NULL;
    if (p->color == 1 && c != 3) return NULL;
    orc_pyr* py = (orc_pyr*)calloc(1, sizeof(orc_pyr));
    py->prm = *p;
    py->L = p->levels;
    py->C = p->color == 1 ? 3 : 1;
    py->nsch = (p->color == 1 && p->cs_sched == 0) ? 2 : 1;
    int C = py->C;
    /* level 0: gray conversion for PGM-G/GD (Sec. III-F), else RGB planes */
    py->W[0] = w; py->H[0] = h;
    py->img[0] = (uint8_t*)malloc((size_t)C * w * h);
    for (int64_t i = 0; i < (int64_t)w * h; ++i) {
        if (C == 1) {
            py->img[0][i] = c == 1 ? img[i] : (uint8_t)gray_of(img[3 * i], img[3 * i + 1], img[3 * i + 2]);
        } else {
            for (int ch = 0; ch < 3; ++ch) py->img[0][(int64_t)ch * w * h + i] = img[3 * i + ch];
        }
    }
    for (int l = 1; l < py->L; ++l) {
        int pw = py->W[l - 1], ph = py->H[l - 1];
        py->W[l] = (pw + 1) / 2; py->H[l] = (ph + 1) / 2;
        int64_t n = (int64_t)py->W[l] * py->H[l];
        py->img[l] = (uint8_t*)malloc((size_t)C * n);
        for (int ch = 0; ch < C; ++ch)
            orc_pyr_down(py->img[l - 1] + (int64_t)ch * pw * ph, pw, ph, py->img[l] + ch * n);
    }
    for (int s = 0; s < py->nsch; ++s)
        for (int l = 0; l < py->L; ++l) {
            int W = py->W[l], H = py->H[l];
            int64_t n = (int64_t)W * H;
            uint8_t* ci = (uint8_t*)malloc((size_t)C * n);
            int sp = space_of(p, s, l);
            if (C == 1) {
                memcpy(ci, py->img[l], n);
            } else {
                uint8_t* rgb = (uint8_t*)malloc(3 * n);
                uint8_t* cv = (uint8_t*)malloc(3 * n);
                for (int64_t i = 0; i < n; ++i)
                    for (int ch = 0; ch < 3; ++ch) rgb[3 * i + ch] = py->img[l][ch * n + i];
                orc_convert(sp, rgb, n, cv);
                for (int64_t i = 0; i < n; ++i)
                    for (int ch = 0; ch < 3; ++ch) ci[ch * n + i] = cv[3 * i + ch];
                free(rgb); free(cv);
            }
            py->cimg[s][l] = ci;
            int16_t* d = (int16_t*)malloc(sizeof(int16_t) * 2 * C * n);
            for (int ch = 0; ch < C; ++ch)
                orc_sobel(ci + ch * n, W, H, p->sobel, d + ch * n, d + (C + ch) * n);
            if (p->descriptor == 1) {      /* direction only, Sec. III-F: G ./ |G| */
                for (int64_t i = 0; i < 2 * C * n; ++i)
                    d[i] = (int16_t)(d[i] > 0 ? 1 : (d[i] < 0 ? -1 : 0));   /* R5: 0/0 := 0 */
            } else if (p->descriptor == 2) {   /* 8-sector angle per colour channel */
                for (int ch = 0; ch < C; ++ch)
                    for (int64_t i = 0; i < n; ++i) {
                        int16_t v[2];
                        orc_sector(d[ch * n + i], d[(C + ch) * n + i], v);
                        d[ch * n + i] = v[0];
                        d[(C + ch) * n + i] = v[1];
                    }
            }
            py->desc[s][l] = d;
        }
    return py;
}

void orc_pyr_free(orc_pyr* py) {
    if (!py) return;
    for (int l = 0; l < py->L; ++l) {
        free(py->img[l]);
        for (int s = 0; s < 2; ++s) { free(py->cimg[s][l]); free(py->desc[s][l]); }
    }
    free(py);
}
int orc_pyr_levels(const orc_pyr* py) { return py->L; }
int orc_pyr_schemes(const orc_pyr* py) { return py->nsch; }
int orc_pyr_channels(const orc_pyr* py) { return py->C; }
void orc_pyr_dims(const orc_pyr* py, int level, int* w, int* h) { *w = py->W[level]; *h = py->H[level]; }
const uint8_t* orc_pyr_image(const orc_pyr* py, int level) { return py->img[level]; }
const uint8_t* orc_pyr_cimage(const orc_pyr* py, int s, int level) { return py->cimg[s][level]; }
const int16_t* orc_pyr_desc(const orc_pyr* py, int s, int level) { return py->desc[s][level]; }

/* ------------------------------------------------------------------ */
/* correspondence fields on the seed lattice (reading R8)              */
/* ------------------------------------------------------------------ */
typedef struct {
    int nx, ny;
    int32_t *ux, *uy;       /* displacement u = F(p) - p, level pixels */
    uint8_t *valid;         /* 0: uninitialized (Sec. III-B)           */
    uint64_t* cost;         /* D(p, p+u) of the current u              */
    uint8_t *outl, *oinit;  /* O^l and "O^l is initialized" (Eq. 6)    */
} field_t;

struct orc_match {
    orc_params prm;
    const orc_pyr *p1, *p2;
    int L, nvis_run;
    int vis_level[4 * MAXL + 8];
    int64_t evals;
    uint64_t stream_id;
    field_t f[MAXL][2];     /* [level][dir]: dir 0 forward (I1 -> I2), 1 backward */
};

static int lattice_n(int Wl, int sigma) {
    int c = sigma / 2;
    return (Wl - 1 - c) >= 0 ? (Wl - 1 - c) / sigma + 1 : 0;
}

/* image dims of the reference and target images of a direction */
static void dir_images(const orc_match* m, int l, int dir, int* wr, int* hr, int* wt, int* ht,
                       const int16_t** R, const int16_t** T) {
    const orc_pyr* ref = dir == 0 ? m->p1 : m->p2;
    const orc_pyr* tgt = dir == 0 ? m->p2 : m->p1;
    int s = dir < ref->nsch ? dir : ref->nsch - 1;
    *wr = ref->W[l]; *hr = ref->H[l]; *wt = tgt->W[l]; *ht = tgt->H[l];
    *R = ref->desc[s][l]; *T = tgt->desc[s][l];
}

static uint64_t dist(orc_match* m, int l, int dir, int px, int py, int qx, int qy) {
    int wr, hr, wt, ht; const int16_t *R, *T;
    dir_images(m, l, dir, &wr, &hr, &wt, &ht, &R, &T);
    int P = dir == 0 ? m->prm.patch_fwd : m->prm.patch_bwd;
    m->evals++;
    return orc_patch_dist(R, wr, hr, T, wt, ht, 2 * m->p1->C, px, py, qx, qy, P, m->prm.norm);
}

static int inside_target(orc_match* m, int l, int dir, int qx, int qy) {
    const orc_pyr* tgt = dir == 0 ? m->p2 : m->p1;
    return qx >= 0 && qy >= 0 && qx < tgt->W[l] && qy < tgt->H[l];
}

/* KD-tree initialisation of F^m (Sec. III-D) read as the exact nearest
 * neighbour it approximates (reading R9): every target pixel is tried in
 * raster order and only a strictly lower cost replaces the best, so ties go
 * to the smaller target y, then the smaller target x. */
static void init_exhaustive(orc_match* m, int l, int dir) {
    field_t* F = &m->f[l][dir];
    const orc_pyr* tgt = dir == 0 ? m->p2 : m->p1;
    int sig = m->prm.seed_stride, c = sig / 2;
    for (int j = 0; j < F->ny; ++j)
        for (int i = 0; i < F->nx; ++i) {
            int px = c + sig * i, py = c + sig * j, s = j * F->nx + i;
            uint64_t best = INF_COST; int bx = 0, by = 0;
            for (int qy = 0; qy < tgt->H[l]; ++qy)
                for (int qx = 0; qx < tgt->W[l]; ++qx) {
                    uint64_t d = dist(m, l, dir, px, py, qx, qy);
                    if (d < best) { best = d; bx = qx; by = qy; }
                }
            F->ux[s] = bx - px; F->uy[s] = by - py; F->valid[s] = 1; F->cost[s] = best;
            F->outl[s] = 0; F->oinit[s] = 0;
        }
}

/* cost of each initialised seed's current u at the start of a visit; a
 * seed whose match centre falls outside the target becomes uninitialised
 * (reading R10) */
static void cost_fill(orc_match* m, int l, int dir) {
    field_t* F = &m->f[l][dir];
    int sig = m->prm.seed_stride, c = sig / 2;
    for (int j = 0; j < F->ny; ++j)
        for (int i = 0; i < F->nx; ++i) {
            int s = j * F->nx + i;
            if (!F->valid[s]) continue;
            int px = c + sig * i, py = c + sig * j;
            int qx = px + F->ux[s], qy = py + F->uy[s];
            if (!inside_target(m, l, dir, qx, qy)) { F->valid[s] = 0; continue; }
            F->cost[s] = dist(m, l, dir, px, py, qx, qy);
        }
}

/* propagation direction of iteration t (Sec. III-B, the FlowFields order):
 * (dx_x, dy_y) = (+,+), (-,-), (-,+), (+,-) */
static const int DIR_SX[4] = {1, -1, -1, 1};
static const int DIR_SY[4] = {1, -1, 1, -1};

/* One seed's update: propagation (Eq. 4) then limited random search (Eq. 5),
 * in the candidate order of reading R11; a candidate replaces the best only
 * on a strictly lower cost. */
static void update_seed(orc_match* m, int l, int dir, int visit, int t, int i, int j) {
    field_t* F = &m->f[l][dir];
    int sig = m->prm.seed_stride, c = sig / 2;
    int s = j * F->nx + i;
    int px = c + sig * i, py = c + sig * j;
    int sx = DIR_SX[t & 3], sy = DIR_SY[t & 3];
    int have = F->valid[s];
    int32_t bux = F->ux[s], buy = F->uy[s];
    uint64_t bc = have ? F->cost[s] : INF_COST;

    /* Eq. 4: Omega = {F(p), F(p - dx) + dx, F(p - dy) + dy}; in displacement
     * form the neighbour's candidate is the neighbour's u */
    int nbi[2] = {i - sx, i}, nbj[2] = {j, j - sy};
    for (int k = 0; k < 2; ++k) {
        int ni = nbi[k], nj = nbj[k];
        if (ni < 0 || nj < 0 || ni >= F->nx || nj >= F->ny) continue;
        int ns = nj * F->nx + ni;
        if (!F->valid[ns]) continue;                 /* uninitialized: ignored */
        int32_t cx = F->ux[ns], cy = F->uy[ns];
        if (!inside_target(m, l, dir, px + cx, py + cy)) continue;
        uint64_t d = dist(m, l, dir, px, py, px + cx, py + cy);
        if (d < bc) { bc = d; bux = cx; buy = cy; have = 1; }
    }
    /* PGM-C3/G3 (Sec. IV): at full resolution, random search only at the
     * points of a grid of spacing rs_grid */
    int g = m->prm.rs_grid;
    int search = !(l == 0 && g > 0 && !(px % g == g / 2 && py % g == g / 2));
    if (have && search) {
        /* Eq. 5: Psi = {F(p)} u {F(p) + floor(R_i W / 2^i)}, i = 0..floor(log2 W),
         * all around the post-propagation F(p) */
        int K = 0;
        for (int w = m->prm.rs_W; w >= 1; w >>= 1) K++;
        int32_t u0x = bux, u0y = buy;
        uint32_t key[2] = {(uint32_t)m->prm.philox_key, (uint32_t)(m->prm.philox_key >> 32)};
        uint32_t r[4] = {0, 0, 0, 0};
        for (int k = 0; k < K; ++k) {
            if ((k & 1) == 0) {
                uint32_t ctr[4] = {(uint32_t)s,
                                   ((uint32_t)visit << 16) | ((uint32_t)dir << 15) | (uint32_t)t,
                                   ((uint32_t)l << 16) | (uint32_t)(k / 2),
                                   (uint32_t)m->stream_id};
                orc_philox4x32_10(ctr, key, r);
            }
            int32_t dx = orc_rs_offset(r[2 * (k & 1)], k, m->prm.rs_W, m->prm.rs_mode);
            int32_t dy = orc_rs_offset(r[2 * (k & 1) + 1], k, m->prm.rs_W, m->prm.rs_mode);
            int32_t cx = u0x + dx, cy = u0y + dy;
            if (!inside_target(m, l, dir, px + cx, py + cy)) continue;
            uint64_t d = dist(m, l, dir, px, py, px + cx, py + cy);
            if (d < bc) { bc = d; bux = cx; buy = cy; }
        }
    }
    if (have) { F->ux[s] = bux; F->uy[s] = buy; F->valid[s] = 1; F->cost[s] = bc; }
}

/* Step 1, basic gradient matching: T iterations of propagation + search.
 * Checkerboard: within an iteration all seeds of colour (i+j) even update
 * from the current field, then all seeds of colour odd (a seed's lattice
 * neighbours all have the other colour, so the order inside a colour does not
 * matter).  Sequential: the paper's in-place scan, rows in the order of dy and
 * columns in the order of dx. */
static void basic_matching(orc_match* m, int l, int visit, int T, int schedule) {
    for (int t = 0; t < T; ++t) {
        if (schedule == ORC_SCHED_CHECKERBOARD) {
            for (int colour = 0; colour < 2; ++colour)
                for (int dir = 0; dir < 2; ++dir) {
                    field_t* F = &m->f[l][dir];
                    for (int j = 0; j < F->ny; ++j)
                        for (int i = 0; i < F->nx; ++i)
                            if (((i + j) & 1) == colour) update_seed(m, l, dir, visit, t, i, j);
                }
        } else {
            int sx = DIR_SX[t & 3], sy = DIR_SY[t & 3];
            for (int dir = 0; dir < 2; ++dir) {
                field_t* F = &m->f[l][dir];
                for (int jj = 0; jj < F->ny; ++jj) {
                    int j = sy > 0 ? jj : F->ny - 1 - jj;
                    for (int ii = 0; ii < F->nx; ++ii) {
                        int i = sx > 0 ? ii : F->nx - 1 - ii;
                        update_seed(m, l, dir, visit, t, i, j);
                    }
                }
            }
        }
    }
}

/* Steps 2-3: forward-backward consistency C^l (reading R13) and the
 * outlier-record update of Eq. 6, read as "outlier when either is yes"
 * (reading R12). */
static void consistency_update(orc_match* m, int l) {
    int sig = m->prm.seed_stride, c = sig / 2;
    uint8_t* C[2];
    for (int dir = 0; dir < 2; ++dir) {
        field_t* F = &m->f[l][dir];
        field_t* G = &m->f[l][1 - dir];
        C[dir] = (uint8_t*)malloc((size_t)F->nx * F->ny + 1);
        for (int j = 0; j < F->ny; ++j)
            for (int i = 0; i < F->nx; ++i) {
                int s = j * F->nx + i;
                int out = 1;
                if (F->valid[s] && G->nx > 0 && G->ny > 0) {
                    int qx = c + sig * i + F->ux[s], qy = c + sig * j + F->uy[s];
                    int gi = clampi((int)floordiv(qx - c + sig / 2, sig), 0, G->nx - 1);
                    int gj = clampi((int)floordiv(qy - c + sig / 2, sig), 0, G->ny - 1);
                    int gs = gj * G->nx + gi;
                    if (G->valid[gs]) {
                        int64_t ex = F->ux[s] + G->ux[gs], ey = F->uy[s] + G->uy[gs];
                        out = (ex * ex + ey * ey) > m->prm.tau2;
                    }
                }
                C[dir][s] = (uint8_t)out;
            }
    }
    for (int dir = 0; dir < 2; ++dir) {
        field_t* F = &m->f[l][dir];
        for (int s = 0; s < F->nx * F->ny; ++s)
            F->outl[s] = F->oinit[s] ? (uint8_t)(F->outl[s] | C[dir][s]) : C[dir][s];
        free(C[dir]);
    }
}

/* Steps 4-5 for one target cell: correspondence-field propagation (Eq. 7)
 * and outlier-record propagation (Eq. 8) in displacement form (reading R14).
 * The n source cells are aleph (children for k = j+1, the parent for
 * k = j-1); aleph' keeps those with O^j = no (or, with prop_all, every
 * initialised one -- the "propagate both" ablation of Table 1).
 *   up:   u^k = mean of aleph' u, halved, rounded half away from zero
 *   down: u^k = 2 u^j(parent)
 * Outputs: out[0..1] = u^k, out[2] = initialised, out[3] = O^k. */
void orc_xfer_cell(int up, int n, const int32_t* ux, const int32_t* uy, const uint8_t* valid,
                   const uint8_t* outl, int prop_all, int32_t out[4]) {
    int64_t sx = 0, sy = 0;
    int cnt = 0, n_inl = 0;
    for (int a = 0; a < n; ++a) {
        int inl = !outl[a];
        n_inl += inl;
        if (inl || (prop_all && valid[a])) { sx += ux[a]; sy += uy[a]; cnt++; }
    }
    out[0] = out[1] = 0;
    if (cnt > 0) {
        if (up) {
            int64_t dd = 2 * (int64_t)cnt;
            int64_t ax = sx < 0 ? -sx : sx, ay = sy < 0 ? -sy : sy;
            int64_t rx = (ax + cnt) / dd, ry = (ay + cnt) / dd;
            out[0] = (int32_t)(sx < 0 ? -rx : rx);
            out[1] = (int32_t)(sy < 0 ? -ry : ry);
        } else {
            out[0] = (int32_t)(2 * sx); out[1] = (int32_t)(2 * sy);
        }
    }
    out[2] = cnt > 0;
    out[3] = n_inl == 0;            /* Eq. 8: yes iff aleph' (inliers) is empty */
}

/* Steps 4-5 over a whole level, both directions: from level j to k = j +- 1
 * on lattice indices (reading R8).  with_o = 0 is the single blue arrow of
 * Fig. 5 (field only; O^k uninitialised). */
static void transfer(orc_match* m, int j, int k, int with_o) {
    int prop_all = (m->prm.ablation >> 1) & 1;
    for (int dir = 0; dir < 2; ++dir) {
        field_t* S = &m->f[j][dir];
        field_t* D = &m->f[k][dir];
        for (int y = 0; y < D->ny; ++y)
            for (int x = 0; x < D->nx; ++x) {
                int d = y * D->nx + x;
                int32_t ux[4], uy[4]; uint8_t va[4], ol[4];
                int n = 0;
                if (k == j + 1) {
                    /* aleph = children {2x, 2x+1} x {2y, 2y+1} on the finer lattice */
                    for (int b = 0; b < 2; ++b)
                        for (int a = 0; a < 2; ++a) {
                            int cx = 2 * x + a, cy = 2 * y + b;
                            if (cx >= S->nx || cy >= S->ny) continue;
                            int cs = cy * S->nx + cx;
                            ux[n] = S->ux[cs]; uy[n] = S->uy[cs];
                            va[n] = S->valid[cs]; ol[n] = S->outl[cs]; n++;
                        }
                } else if (S->nx > 0 && S->ny > 0) {
                    /* aleph = {parent (floor(x/2), floor(y/2))}, clamped to the coarser lattice */
                    int cx = x / 2, cy = y / 2;
                    if (cx > S->nx - 1) cx = S->nx - 1;
                    if (cy > S->ny - 1) cy = S->ny - 1;
                    int cs = cy * S->nx + cx;
                    ux[0] = S->ux[cs]; uy[0] = S->uy[cs]; va[0] = S->valid[cs]; ol[0] = S->outl[cs];
                    n = 1;
                }
                int32_t out[4];
                orc_xfer_cell(k == j + 1, n, ux, uy, va, ol, prop_all, out);
                D->ux[d] = out[0]; D->uy[d] = out[1];
                D->valid[d] = (uint8_t)out[2];
                D->cost[d] = INF_COST;
                if (with_o) { D->outl[d] = (uint8_t)out[3]; D->oinit[d] = 1; }
                else { D->outl[d] = 0; D->oinit[d] = 0; }
            }
    }
}

/* the visit schedule of Fig. 5 for general L (reading R15): m = L-1; m (init),
 * then [m-1, m] x N (field + record), then m-1 (field only), then m-2 .. 0 */
static int build_schedule(const orc_params* p, int* lv, int* xfer_o) {
    int L = p->levels, m = L - 1, N = p->refine_rounds;
    if (p->ablation & 1) N = 0;
    int n = 0;
    lv[n] = m; xfer_o[n] = 0; n++;
    if (m == 0) return n;
    for (int r = 0; r < N; ++r) {
        lv[n] = m - 1; xfer_o[n] = 1; n++;
        lv[n] = m; xfer_o[n] = 1; n++;
    }
    lv[n] = m - 1; xfer_o[n] = 0; n++;
    for (int l = m - 2; l >= 0; --l) { lv[n] = l; xfer_o[n] = 1; n++; }
    if (p->ablation & 4)
        for (int v = 0; v < n; ++v) xfer_o[v] = 0;
    return n;
}

orc_match* orc_match_run(const orc_params* p, const orc_pyr* p1, const orc_pyr* p2,
                         int schedule, uint64_t stream_id) {
    if (!p1 || !p2 || p1->L != p->levels || p2->L != p->levels || p1->C != p2->C) return NULL;
    if (p->seed_stride < 1 || p->patch_fwd < 1 || p->patch_bwd < 1 || p->rs_W < 1) return NULL;
    orc_match* m = (orc_match*)calloc(1, sizeof(orc_match));
    m->prm = *p; m->p1 = p1; m->p2 = p2; m->L = p->levels; m->stream_id = stream_id;
    for (int l = 0; l < m->L; ++l)
        for (int dir = 0; dir < 2; ++dir) {
            const orc_pyr* ref = dir == 0 ? p1 : p2;
            field_t* F = &m->f[l][dir];
            F->nx = lattice_n(ref->W[l], p->seed_stride);
            F->ny = lattice_n(ref->H[l], p->seed_stride);
            size_t n = (size_t)F->nx * F->ny + 1;
            F->ux = (int32_t*)calloc(n, 4); F->uy = (int32_t*)calloc(n, 4);
            F->valid = (uint8_t*)calloc(n, 1); F->cost = (uint64_t*)calloc(n, 8);
            F->outl = (uint8_t*)calloc(n, 1); F->oinit = (uint8_t*)calloc(n, 1);
            for (size_t s = 0; s < n; ++s) F->cost[s] = INF_COST;
        }
    int lv[4 * MAXL + 8], xo[4 * MAXL + 8];
    int nv = build_schedule(p, lv, xo);
    if (p->max_visits > 0 && p->max_visits < nv) nv = p->max_visits;
    for (int v = 0; v < nv; ++v) {
        int l = lv[v];
        m->vis_level[v] = l;
        if (v == 0) { init_exhaustive(m, l, 0); init_exhaustive(m, l, 1); }
        else transfer(m, lv[v - 1], l, xo[v]);
        cost_fill(m, l, 0); cost_fill(m, l, 1);
        int T = p->iters_level[l] >= 0 ? p->iters_level[l] : l == 0 ? p->iters_fine : p->iters_coarse;
        basic_matching(m, l, v, T, schedule);
        consistency_update(m, l);
    }
    m->nvis_run = nv;
    return m;
}

void orc_match_free(orc_match* m) {
    if (!m) return;
    for (int l = 0; l < m->L; ++l)
        for (int d = 0; d < 2; ++d) {
            field_t* F = &m->f[l][d];
            free(F->ux); free(F->uy); free(F->valid); free(F->cost); free(F->outl); free(F->oinit);
        }
    free(m);
}
int orc_match_visits(const orc_match* m) { return m->nvis_run; }
int orc_match_visit_level(const orc_match* m, int v) { return m->vis_level[v]; }
int64_t orc_match_evals(const orc_match* m) { return m->evals; }
void orc_field_dims(const orc_match* m, int level, int dir, int* nx, int* ny) {
    *nx = m->f[level][dir].nx; *ny = m->f[level][dir].ny;
}
void orc_field_get(const orc_match* m, int level, int dir, int32_t* ux, int32_t* uy,
                   uint8_t* valid, uint64_t* cost, uint8_t* outl, uint8_t* oinit) {
    const field_t* F = &m->f[level][dir];
    size_t n = (size_t)F->nx * F->ny;
    if (ux) memcpy(ux, F->ux, n * 4);
    if (uy) memcpy(uy, F->uy, n * 4);
    if (valid) memcpy(valid, F->valid, n);
    if (cost) memcpy(cost, F->cost, n * 8);
    if (outl) memcpy(outl, F->outl, n);
    if (oinit) memcpy(oinit, F->oinit, n);
}

/* Region removal (Sec. III-E, reading R16) on a level-0 forward field given
 * as arrays (nx x ny seeds, raster order), then the grid export of Sec.
 * III-G (reading R17).  Inlier seeds (valid, O = no) that are 4-neighbours on
 * the lattice join a region iff their displacements differ by less than
 * sqrt(region_dmax2); regions with fewer than min_region seeds are removed.
 * Regions are found by breadth-first search. */
int64_t orc_filter_arrays(const orc_params* p, int nx, int ny, const int32_t* ux,
                          const int32_t* uy, const uint8_t* valid, const uint8_t* outl,
                          int32_t* rows, int64_t max_rows, uint8_t* keep_out) {
    int n = nx * ny;
    int sig = p->seed_stride, c = sig / 2;
    int* comp = (int*)malloc(sizeof(int) * (n + 1));
    int* queue = (int*)malloc(sizeof(int) * (n + 1));
    int* size = (int*)calloc((size_t)n + 1, sizeof(int));
    for (int s = 0; s < n; ++s) comp[s] = -1;
    int ncomp = 0;
    for (int s0 = 0; s0 < n; ++s0) {
        if (comp[s0] >= 0 || outl[s0] || !valid[s0]) continue;
        int head = 0, tail = 0;
        queue[tail++] = s0; comp[s0] = ncomp;
        while (head < tail) {
            int s = queue[head++];
            int i = s % nx, j = s / nx;
            int ni[4] = {i - 1, i + 1, i, i}, nj[4] = {j, j, j - 1, j + 1};
            for (int k = 0; k < 4; ++k) {
                if (ni[k] < 0 || nj[k] < 0 || ni[k] >= nx || nj[k] >= ny) continue;
                int t = nj[k] * nx + ni[k];
                if (comp[t] >= 0 || outl[t] || !valid[t]) continue;
                int64_t dx = ux[s] - ux[t], dy = uy[s] - uy[t];
                if (dx * dx + dy * dy >= p->region_dmax2) continue;
                comp[t] = ncomp; queue[tail++] = t;
            }
        }
        size[ncomp] = tail;
        ncomp++;
    }
    int64_t cnt = 0;
    for (int s = 0; s < n; ++s) {
        int keep = comp[s] >= 0 && size[comp[s]] >= p->min_region;
        if (keep_out) keep_out[s] = (uint8_t)keep;
        if (!keep) continue;
        if (cnt < max_rows && rows) {
            int i = s % nx, j = s / nx;
            int x = c + sig * i, y = c + sig * j;
            rows[4 * cnt + 0] = x; rows[4 * cnt + 1] = y;
            rows[4 * cnt + 2] = x + ux[s]; rows[4 * cnt + 3] = y + uy[s];
        }
        cnt++;
    }
    free(comp); free(queue); free(size);
    return cnt;
}

/* The same on the level-0 forward field of a match. */
int64_t orc_filter(const orc_params* p, const orc_match* m, int32_t* rows, int64_t max_rows,
                   uint8_t* keep_out) {
    const field_t* F = &m->f[0][0];
    return orc_filter_arrays(p, F->nx, F->ny, F->ux, F->uy, F->valid, F->outl, rows, max_rows,
                             keep_out);
}

/* ------------------------------------------------------------------------
 * Sparse-to-dense interpolation (Sec. III-G).  The paper hands its grid-3
 * matches to EpicFlow (edge-aware geodesic distance on a learned edge map,
 * then Nadaraya-Watson (NW) or locally-weighted affine (LA) interpolation,
 * LA when the matches exceed 2.2 % of the image).  Here the edge map is the
 * L1 magnitude of the level-0 gradient descriptor (R23), the neighbours of a
 * pixel are its K geodesically nearest matches (R24) and the weights are
 * exp(-d / lambda) (R25).
 * ---------------------------------------------------------------------- */

/* R23: step cost of a pixel */
void orc_interp_cost(const int16_t* desc, int nch, int w, int h, int shift, uint32_t* cost) {
    for (int64_t p = 0; p < (int64_t)w * h; ++p) {
        int64_t s = 0;
        for (int c = 0; c < nch; ++c) {
            int v = desc[(int64_t)c * w * h + p];
            s += v < 0 ? -v : v;
        }
        cost[p] = 1u + (uint32_t)(s >> shift);
    }
}

/* binary min-heap of (key, pixel) */
typedef struct { uint64_t key; int64_t px; } orc_hent;
typedef struct { orc_hent* a; int64_t n, cap; } orc_heap;

static int heap_push(orc_heap* H, uint64_t key, int64_t px) {
    if (H->n == H->cap) {
        int64_t cap = H->cap ? 2 * H->cap : 1024;
        orc_hent* a = (orc_hent*)realloc(H->a, (size_t)cap * sizeof(orc_hent));
        if (!a) return -1;
        H->a = a;
        H->cap = cap;
    }
    int64_t i = H->n++;
    while (i > 0) {
        int64_t up = (i - 1) / 2;
        if (H->a[up].key < key || (H->a[up].key == key && H->a[up].px <= px)) break;
        H->a[i] = H->a[up];
        i = up;
    }
    H->a[i].key = key;
    H->a[i].px = px;
    return 0;
}

static orc_hent heap_pop(orc_heap* H) {
    orc_hent top = H->a[0], last = H->a[--H->n];
    int64_t i = 0;
    for (;;) {
        int64_t c = 2 * i + 1;
        if (c >= H->n) break;
        if (c + 1 < H->n && (H->a[c + 1].key < H->a[c].key ||
                             (H->a[c + 1].key == H->a[c].key && H->a[c + 1].px < H->a[c].px)))
            ++c;
        if (last.key < H->a[c].key || (last.key == H->a[c].key && last.px <= H->a[c].px)) break;
        H->a[i] = H->a[c];
        i = c;
    }
    H->a[i] = last;
    return top;
}

/* R24: Dijkstra from every match at once, where a pixel is settled once per
 * label, at most K times: entries leave the heap in (distance, label) order,
 * so each pixel receives its labels in that order and keeps the first K
 * distinct ones.  (If label i is among the K nearest of pixel p, it is among
 * the K nearest of every pixel on a shortest path from match i to p, so the
 * truncation loses nothing.) */
int orc_interp_knn(int w, int h, const uint32_t* cost, const int32_t* sx, const int32_t* sy,
                   int64_t n, int K, uint64_t* keys) {
    const int64_t N = (int64_t)w * h;
    int* cnt = (int*)calloc((size_t)N, sizeof(int));
    orc_heap H = {NULL, 0, 0};
    if (!cnt) return -1;
    for (int64_t p = 0; p < N * K; ++p) keys[p] = UINT64_MAX;
    int rc = 0;
    for (int64_t i = 0; i < n && rc == 0; ++i)
        if (sx[i] >= 0 && sy[i] >= 0 && sx[i] < w && sy[i] < h)
            rc = heap_push(&H, (uint64_t)i, (int64_t)sy[i] * w + sx[i]);
    int64_t* first = (int64_t*)malloc((size_t)N * sizeof(int64_t));  /* a position given twice */
    if (!first) rc = -1;
    for (int64_t p = 0; p < N && first; ++p) first[p] = -1;
    for (int64_t i = 0; i < n && first; ++i)
        if (sx[i] >= 0 && sy[i] >= 0 && sx[i] < w && sy[i] < h) {
            const int64_t p = (int64_t)sy[i] * w + sx[i];
            if (first[p] < 0) first[p] = i;
        }
    while (rc == 0 && H.n > 0) {
        const orc_hent e = heap_pop(&H);
        const uint64_t d = e.key >> 32;
        const int64_t lab = (int64_t)(e.key & 0xffffffffu), p = e.px;
        if (d == 0 && first[p] != lab) continue;           /* duplicate position */
        if (cnt[p] >= K) continue;
        int seen = 0;
        for (int k = 0; k < cnt[p]; ++k)
            if ((int64_t)(keys[p * K + k] & 0xffffffffu) == lab) seen = 1;
        if (seen) continue;
        keys[p * K + cnt[p]++] = e.key;
        const int x = (int)(p % w), y = (int)(p / w);
        const int nx[4] = {x - 1, x + 1, x, x}, ny[4] = {y, y, y - 1, y + 1};
        for (int k = 0; k < 4 && rc == 0; ++k) {
            if (nx[k] < 0 || ny[k] < 0 || nx[k] >= w || ny[k] >= h) continue;
            const int64_t q = (int64_t)ny[k] * w + nx[k];
            if (cnt[q] >= K) continue;
            const uint64_t dq = d + cost[p] + cost[q];
            if (dq >= 0xffffffffull) continue;               /* beyond the distance range */
            rc = heap_push(&H, dq << 32 | (uint64_t)lab, q);
        }
    }
    free(H.a);
    free(cnt);
    free(first);
    return rc;
}

/* R25: NW average, or the weighted affine fit (Cramer's rule on the 3 x 3
 * normal equations in coordinates relative to the pixel, whose constant
 * term is the value at the pixel).  The weights are taken relative to the
 * nearest match's (exp(-(d - d0) / lambda), the same fit and average); the
 * fit counts as degenerate when det M <= 1e-6 (sum of weights)^3. */
void orc_interp_flow(int w, int h, int K, const uint64_t* keys, const int32_t* sx,
                     const int32_t* sy, const int32_t* fx, const int32_t* fy, double lambda,
                     int use_la, double* flow) {
    for (int64_t p = 0; p < (int64_t)w * h; ++p) {
        const int x = (int)(p % w), y = (int)(p / w);
        double sw = 0, nwx = 0, nwy = 0;
        double M[3][3] = {{0}}, bx[3] = {0}, by[3] = {0};
        const uint64_t d0 = keys[p * K] >> 32;          /* weights relative to the nearest */
        for (int k = 0; k < K; ++k) {
            const uint64_t key = keys[p * K + k];
            if (key == UINT64_MAX) break;
            const int64_t i = (int64_t)(key & 0xffffffffu);
            const double wgt = exp(-(double)((key >> 32) - d0) / lambda);
            const double v[3] = {(double)(sx[i] - x), (double)(sy[i] - y), 1.0};
            sw += wgt;
            nwx += wgt * fx[i];
            nwy += wgt * fy[i];
            for (int a = 0; a < 3; ++a) {
                for (int b = 0; b < 3; ++b) M[a][b] += wgt * v[a] * v[b];
                bx[a] += wgt * fx[i] * v[a];
                by[a] += wgt * fy[i] * v[a];
            }
        }
        double ox = 0, oy = 0;
        if (sw > 0) {
            ox = nwx / sw;
            oy = nwy / sw;
            if (use_la) {
                const double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                                   M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                                   M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
                if (det > 1e-6 * sw * sw * sw) {
                    /* constant term: the determinant with column 3 replaced by b */
                    const double dx = M[0][0] * (M[1][1] * bx[2] - bx[1] * M[2][1]) -
                                      M[0][1] * (M[1][0] * bx[2] - bx[1] * M[2][0]) +
                                      bx[0] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
                    const double dy = M[0][0] * (M[1][1] * by[2] - by[1] * M[2][1]) -
                                      M[0][1] * (M[1][0] * by[2] - by[1] * M[2][0]) +
                                      by[0] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
                    ox = dx / det;
                    oy = dy / det;
                }
            }
        }
        flow[2 * p] = ox;
        flow[2 * p + 1] = oy;
    }
}
