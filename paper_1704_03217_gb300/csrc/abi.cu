// abi.cu -- the extern "C" entry points of libpgm: argument checks, buffer
// layouts (plans), the visit schedule of Fig. 5 and the launch sequence.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <utility>
#include <vector>

#include "pgm_device.cuh"

namespace pgm {

// ------------------------------------------------------ launch accounting
static std::atomic<long long> g_launches{0};

// kernels whose shared-memory limit is raised on a device (smem_opt_in)
static std::mutex g_optin_mu;
static std::vector<std::pair<const void*, int>> g_optin;
pgm_status smem_opt_in(const void* kern) {
    int dev = 0;
    PGM_TRY(cudaGetDevice(&dev), "shared-memory opt-in: cudaGetDevice");
    std::lock_guard<std::mutex> lock(g_optin_mu);
    for (const auto& e : g_optin)
        if (e.first == kern && e.second == dev) return PGM_OK;
    int max_optin = 0;
    PGM_TRY(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev),
            "shared-memory opt-in: device limit");
    cudaFuncAttributes fa;
    PGM_TRY(cudaFuncGetAttributes(&fa, kern), "shared-memory opt-in: kernel attributes");
    // the kernel's static shared memory counts against the same limit
    const int dyn = max_optin - (int)fa.sharedSizeBytes;
    PGM_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn),
            "shared-memory opt-in: set");
    g_optin.emplace_back(kern, dev);
    return PGM_OK;
}

// the CUDA call behind the last PGM_ERR_CUDA of each host thread
static thread_local char g_detail[192];
pgm_status cuda_fail(const char* site, cudaError_t e) {
    snprintf(g_detail, sizeof(g_detail), "%s: %s (%d): %s", site, cudaGetErrorName(e), (int)e,
             cudaGetErrorString(e));
    (void)cudaGetLastError();     // reported by the status: not left for the caller's next check
    return PGM_ERR_CUDA;
}

// ------------------------------------------- host-side fault injection
// pgm_inject_launch_failure: a countdown over the launch steps of the
// matching schedule, process-wide; the step that takes it from 1 to 0 fails.
static std::atomic<int> g_fail_step{0};
static bool fault_due() {
    int v = g_fail_step.load(std::memory_order_relaxed);
    while (v > 0 && !g_fail_step.compare_exchange_weak(v, v - 1, std::memory_order_relaxed)) {
    }
    return v == 1;
}
static pgm_status injected_fail(const char* site) {
    snprintf(g_detail, sizeof(g_detail), "%s: injected launch failure", site);
    return PGM_ERR_CUDA;
}

// ------------------------------------------------------------ tuning knobs
static std::atomic<int> g_slack{2}, g_chunk{MAXB}, g_tile_w{8};
Tuning tuning() { return Tuning{g_slack.load(), g_chunk.load(), g_tile_w.load()}; }

// bounded device waits (the search kernel's mbarrier waits), in SM cycles
constexpr long long WAIT_DEFAULT = 1ll << 31;        // about 1 s at 2 GHz
static std::atomic<long long> g_wait{WAIT_DEFAULT};
long long wait_limit() { return g_wait.load(); }
bool pdl_enabled() {
    static const bool on = [] {
        const char* e = getenv("PGM_PDL");
        return !(e && e[0] == '0');
    }();
    return on;
}

namespace {
struct ProfEvent { int cls; int n; cudaEvent_t a, b; };
struct ProfState {
    bool on = false;
    std::vector<ProfEvent> open;          // recorded, not yet read
    std::vector<cudaEvent_t> pool;
    double ms[PGM_K_COUNT] = {0};
    long long launches[PGM_K_COUNT] = {0};
};
thread_local ProfState g_prof;

cudaEvent_t take_event() {
    if (!g_prof.pool.empty()) {
        cudaEvent_t e = g_prof.pool.back();
        g_prof.pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}
}  // namespace

KScope::KScope(int c, cudaStream_t s, int nl) : cls(c), st(s), n(nl), slot(-1) {
    if (!g_prof.on) return;
    cudaEvent_t a = take_event(), b = take_event();
    if (!a || !b) return;
    cudaEventRecord(a, st);
    g_prof.open.push_back({cls, n, a, b});
    slot = (int)g_prof.open.size() - 1;
}

KScope::~KScope() {
    g_launches.fetch_add(n, std::memory_order_relaxed);
    if (slot >= 0 && slot < (int)g_prof.open.size()) {
        g_prof.open[slot].n = n;              // the launcher may have changed the count
        cudaEventRecord(g_prof.open[slot].b, st);
    }
}

pgm_status check_params(const pgm_params* p) {
    if (!p) return PGM_ERR_ARG;
    if (p->levels < 1 || p->levels > MAXL) return PGM_ERR_ARG;
    if (p->seed_stride < 1 || p->seed_stride > 64) return PGM_ERR_ARG;
    if (p->patch_fwd < 1 || p->patch_bwd < 1) return PGM_ERR_ARG;
    if (p->patch_fwd > MAXP || p->patch_bwd > MAXP) return PGM_ERR_UNSUPPORTED;
    if (p->sobel != 3 && p->sobel != 5) return PGM_ERR_ARG;
    if (p->color != PGM_GRAY && p->color != PGM_RGB) return PGM_ERR_ARG;
    if (p->descriptor != PGM_FULL && p->descriptor != PGM_DIR && p->descriptor != PGM_SECTOR)
        return PGM_ERR_ARG;
    if (p->cs_sched != PGM_CS_PAPER && p->cs_sched != PGM_CS_PLAIN) return PGM_ERR_ARG;
    if (p->norm != PGM_L2SQ && p->norm != PGM_L1) return PGM_ERR_ARG;
    if (p->iters_coarse < 0 || p->iters_fine < 0 || p->iters_coarse > 32767 ||
        p->iters_fine > 32767) return PGM_ERR_ARG;
    for (int l = 0; l < 12; ++l)
        if (p->iters_level[l] < -1 || p->iters_level[l] > 32767) return PGM_ERR_ARG;
    if (p->refine_rounds < 0 || p->refine_rounds > 64) return PGM_ERR_ARG;
    if (p->rs_W < 1 || p->rs_W > (1 << 14)) return PGM_ERR_ARG;
    if (p->rs_mode != PGM_RS_SYMMETRIC && p->rs_mode != PGM_RS_PAPER_FLOOR) return PGM_ERR_ARG;
    if (p->tau2 < 0 || p->min_region < 0 || p->region_dmax2 < 0 || p->max_visits < 0)
        return PGM_ERR_ARG;
    if (p->ablation < 0 || p->ablation > 7 || p->rs_grid < 0 || p->rs_grid > 64)
        return PGM_ERR_ARG;
    return PGM_OK;
}

// Table 2 read with period 3 for deeper pyramids; scheme 0 forward, 1 backward
static int space_of(const pgm_params* p, int scheme, int level) {
    if (p->color == PGM_GRAY) return SP_GRAY;
    if (p->cs_sched == PGM_CS_PLAIN) return SP_RGB;
    static const int fwd[3] = {SP_RGB, SP_LAB, SP_YCRCB};
    static const int bwd[3] = {SP_LAB, SP_YCRCB, SP_RGB};
    return scheme == 0 ? fwd[level % 3] : bwd[level % 3];
}

bool make_pyr_plan(const pgm_params* p, int w, int h, PyrPlan* pp) {
    if (check_params(p) != PGM_OK || w < 1 || h < 1 || w > 32767 || h > 32767) return false;
    memset(pp, 0, sizeof(*pp));
    pp->L = p->levels;
    pp->C = p->color == PGM_RGB ? 3 : 1;
    pp->nch = 2 * pp->C;
    pp->nsch = (p->color == PGM_RGB && p->cs_sched == PGM_CS_PAPER) ? 2 : 1;
    pp->pxw = px_words(pp->nch);
    size_t off = 0;
    for (int l = 0; l < pp->L; ++l) {
        pp->W[l] = l == 0 ? w : (pp->W[l - 1] + 1) / 2;
        pp->H[l] = l == 0 ? h : (pp->H[l - 1] + 1) / 2;
        pp->img_row[l] = (int)align_up(pp->W[l], 16);
        pp->img_plane[l] = (size_t)pp->img_row[l] * pp->H[l];
        pp->img_off[l] = off;
        off = align_up(off + pp->img_plane[l] * pp->C, 256);
        // padded row: W + 2 BORD pixels of 2 pxw int16 values, 16-byte multiple
        pp->desc_row[l] = (int)align_up((size_t)(pp->W[l] + 2 * BORD) * 2 * pp->pxw, 8);
    }
    for (int s = 0; s < pp->nsch; ++s)
        for (int l = 0; l < pp->L; ++l) {
            int sp = space_of(p, s, l);
            pp->space[s][l] = sp;
            if (sp == SP_LAB || sp == SP_YCRCB) {
                pp->cimg_off[s][l] = off;
                off = align_up(off + pp->img_plane[l] * pp->C, 256);
            } else {
                pp->cimg_off[s][l] = pp->img_off[l];
            }
            // the padded arrays; pixel (0, 0) sits BORD rows and BORD pixels in
            const size_t arr = (size_t)pp->desc_row[l] * (pp->H[l] + 2 * BORD) * 2;
            const size_t inner = ((size_t)BORD * pp->desc_row[l] + (size_t)BORD * 2 * pp->pxw) * 2;
            pp->desc_pad_off[s][l] = off;
            pp->desc_off[s][l] = off + inner;
            off = align_up(off + arr, 256);
            pp->split_pad_off[s][l] = off;
            pp->split_off[s][l] = off + inner;
            off = align_up(off + arr, 256);
            if (p->descriptor == PGM_DIR) {      // bit-planes of the sign codes
                const int rowbits = (pp->W[l] + 2 * BORD) * pp->nch;
                pp->bit_row[l] = (int)align_up((size_t)(rowbits + 31) / 32 + 4, 4);
                pp->bits_off[s][l] = off;
                off = align_up(off + 2 * 4 * (size_t)pp->bit_row[l] * (pp->H[l] + 2 * BORD), 256);
            }
        }
    for (int s = pp->nsch; s < 2; ++s)
        for (int l = 0; l < pp->L; ++l) {
            pp->space[s][l] = pp->space[0][l];
            pp->cimg_off[s][l] = pp->cimg_off[0][l];
            pp->desc_off[s][l] = pp->desc_off[0][l];
            pp->split_off[s][l] = pp->split_off[0][l];
            pp->desc_pad_off[s][l] = pp->desc_pad_off[0][l];
            pp->split_pad_off[s][l] = pp->split_pad_off[0][l];
            pp->bits_off[s][l] = pp->bits_off[0][l];
        }
    pp->bytes = off + 256;     // tail slack: vector loads never leave the buffer
    return true;
}

bool make_ws_plan(const pgm_params* p, int w1, int h1, int w2, int h2, WsPlan* wp) {
    PyrPlan a, b;
    if (!make_pyr_plan(p, w1, h1, &a) || !make_pyr_plan(p, w2, h2, &b)) return false;
    memset(wp, 0, sizeof(*wp));
    wp->L = p->levels;
    size_t off = 256;          // [0, 256): status word
    wp->off_err = 0;
    for (int l = 0; l < wp->L; ++l)
        for (int d = 0; d < 2; ++d) {
            const PyrPlan& r = d == 0 ? a : b;
            int nx = lattice_n(r.W[l], p->seed_stride), ny = lattice_n(r.H[l], p->seed_stride);
            wp->nx[l][d] = nx; wp->ny[l][d] = ny;
            size_t n = (size_t)nx * ny;
            wp->off_u[l][d] = off;     off = align_up(off + 4 * n, 256);
            wp->off_cost[l][d] = off;  off = align_up(off + 8 * n, 256);
            wp->off_flags[l][d] = off; off = align_up(off + n, 256);
            wp->off_sa2[l][d] = off;   off = align_up(off + 8 * n, 256);
            const PyrPlan& t = d == 0 ? b : a;       // target image of this direction
            wp->sbp[l][d] = (t.W[l] + 1) & ~1;         // even: 16-byte rows for tensor copies
            wp->off_sb2[l][d] = off;
            off = align_up(off + 8 * (size_t)wp->sbp[l][d] * t.H[l], 256);
            wp->off_sa2img[l][d] = off;
            off = align_up(off + 8 * (size_t)r.W[l] * r.H[l], 256);
        }
    size_t n0 = (size_t)wp->nx[0][0] * wp->ny[0][0];
    wp->nblk0 = (int)((n0 + 255) / 256);
    wp->off_label = off; off = align_up(off + 4 * n0, 256);
    wp->off_size = off;  off = align_up(off + 4 * n0, 256);
    wp->off_bsum = off;  off = align_up(off + 4 * (size_t)wp->nblk0 + 4, 256);
    wp->bytes = off;
    return true;
}

// Fig. 5 for general L (m = L-1): m (init); [m-1, m] x N with field and
// outlier record; m-1 with the field only; then m-2 .. 0 with both.
void make_schedule(const pgm_params* p, Schedule* s) {
    const int m = p->levels - 1;
    const int N = (p->ablation & PGM_ABL_NO_REFINE) ? 0 : p->refine_rounds;
    int n = 0;
    s->level[n] = m; s->with_o[n] = 0; ++n;
    if (m > 0) {
        for (int r = 0; r < N; ++r) {
            s->level[n] = m - 1; s->with_o[n] = 1; ++n;
            s->level[n] = m; s->with_o[n] = 1; ++n;
        }
        s->level[n] = m - 1; s->with_o[n] = 0; ++n;
        for (int l = m - 2; l >= 0; --l) { s->level[n] = l; s->with_o[n] = 1; ++n; }
    }
    if (p->ablation & PGM_ABL_NO_OUTLIER_PROP)
        for (int v = 0; v < n; ++v) s->with_o[v] = 0;
    if (p->max_visits > 0 && p->max_visits < n) n = p->max_visits;
    s->n = n;
}

namespace {

struct PairCtx {
    PyrPlan a, b;
    WsPlan w;
    const uint8_t* pyr1; const uint8_t* pyr2;
    uint8_t* ws;
    uint32_t stream_id;
};

void fill_dir(const pgm_params* p, const PairCtx& c, int l, int d, DirLvl* D) {
    const PyrPlan& R = d == 0 ? c.a : c.b;     // reference image's pyramid
    const PyrPlan& T = d == 0 ? c.b : c.a;
    const uint8_t* rp = d == 0 ? c.pyr1 : c.pyr2;
    const uint8_t* tp = d == 0 ? c.pyr2 : c.pyr1;
    int s = d < R.nsch ? d : R.nsch - 1;
    D->ref = reinterpret_cast<const int16_t*>(rp + R.desc_off[s][l]);
    D->ref_split = reinterpret_cast<const uint32_t*>(rp + R.split_off[s][l]);
    D->tgt = reinterpret_cast<const int16_t*>(tp + T.desc_off[s][l]);
    D->ref_pitch = R.desc_row[l]; D->tgt_pitch = T.desc_row[l];
    D->rw = R.W[l]; D->rh = R.H[l]; D->tw = T.W[l]; D->th = T.H[l];
    D->nx = c.w.nx[l][d]; D->ny = c.w.ny[l][d];
    D->onx = c.w.nx[l][1 - d]; D->ony = c.w.ny[l][1 - d];
    D->P = d == 0 ? p->patch_fwd : p->patch_bwd;
    D->sbp = c.w.sbp[l][d];
    D->u = reinterpret_cast<int32_t*>(c.ws + c.w.off_u[l][d]);
    D->cost = reinterpret_cast<unsigned long long*>(c.ws + c.w.off_cost[l][d]);
    D->flags = c.ws + c.w.off_flags[l][d];
    D->ou = reinterpret_cast<const int32_t*>(c.ws + c.w.off_u[l][1 - d]);
    D->oflags = c.ws + c.w.off_flags[l][1 - d];
    D->sa2 = reinterpret_cast<unsigned long long*>(c.ws + c.w.off_sa2[l][d]);
    D->sb2 = reinterpret_cast<unsigned long long*>(c.ws + c.w.off_sb2[l][d]);
    D->sa2img = reinterpret_cast<unsigned long long*>(c.ws + c.w.off_sa2img[l][d]);
    D->rbit_row = R.bit_row[l];
    D->tbit_row = T.bit_row[l];
    D->ref_bits = R.bit_row[l] ? reinterpret_cast<const uint32_t*>(rp + R.bits_off[s][l]) : nullptr;
    D->tgt_bits = T.bit_row[l] ? reinterpret_cast<const uint32_t*>(tp + T.bits_off[s][l]) : nullptr;
}

// Auxiliary streams with their fork and join events, one set per (device,
// caller stream) of each host thread, so that calls on different caller
// streams never wait on each other's forked work.  Created on first use and
// kept (the library allocates no device memory for them); with AUX_MAX sets
// in use a call on a new caller stream does not fork (*out = null).
struct Aux {
    bool used = false;
    int dev = -1;
    cudaStream_t key = nullptr;      // the caller's stream
    cudaStream_t s = nullptr;        // box filters of the finer levels
    cudaStream_t s2 = nullptr;       // backward-direction search phases
    cudaEvent_t fork = nullptr, sfork = nullptr, sjoin = nullptr;
    cudaEvent_t lvl[MAXL] = {};
};
constexpr int AUX_MAX = 32;
static thread_local Aux g_aux[AUX_MAX];

static pgm_status aux_get(cudaStream_t st, Aux** out) {
    *out = nullptr;
    int dev = 0;
    PGM_TRY(cudaGetDevice(&dev), "aux streams: cudaGetDevice");
    for (int i = 0; i < AUX_MAX; ++i)
        if (g_aux[i].used && g_aux[i].dev == dev && g_aux[i].key == st) {
            *out = &g_aux[i];
            return PGM_OK;
        }
    for (int i = 0; i < AUX_MAX; ++i) {
        if (g_aux[i].used) continue;
        Aux a;
        a.dev = dev;
        a.key = st;
        PGM_TRY(cudaStreamCreateWithFlags(&a.s, cudaStreamNonBlocking), "aux streams: create");
        PGM_TRY(cudaStreamCreateWithFlags(&a.s2, cudaStreamNonBlocking), "aux streams: create");
        PGM_TRY(cudaEventCreateWithFlags(&a.fork, cudaEventDisableTiming), "aux streams: event");
        PGM_TRY(cudaEventCreateWithFlags(&a.sfork, cudaEventDisableTiming), "aux streams: event");
        PGM_TRY(cudaEventCreateWithFlags(&a.sjoin, cudaEventDisableTiming), "aux streams: event");
        for (int l = 0; l < MAXL; ++l)
            PGM_TRY(cudaEventCreateWithFlags(&a.lvl[l], cudaEventDisableTiming), "aux streams: event");
        a.used = true;
        g_aux[i] = a;
        *out = &g_aux[i];
        return PGM_OK;
    }
    return PGM_OK;
}

// What a call has forked onto its auxiliary streams and not yet joined back
// to the caller's stream.
struct Forks {
    Aux* aux = nullptr;
    bool s_forked = false;       // aux->s waits on this call's work
    bool box_open[MAXL] = {};    // box sums of level l pending on aux->s
    bool s2_open = false;        // backward search phases pending on aux->s2
};

pgm_status run_batch_forked(const pgm_params* p, PairCtx* ctx, int n, cudaStream_t st,
                            Forks& fk) {
    Schedule sch;
    make_schedule(p, &sch);
    const int nch = ctx[0].a.nch;
    const int maxP = p->patch_fwd > p->patch_bwd ? p->patch_fwd : p->patch_bwd;
    MatchConst mc;
    memset(&mc, 0, sizeof(mc));
    mc.sigma = p->seed_stride; mc.c = p->seed_stride / 2;
    mc.norm = p->norm; mc.rs_W = p->rs_W; mc.rs_mode = p->rs_mode; mc.K = rs_count(p->rs_W);
    mc.key0 = (uint32_t)(p->philox_key & 0xffffffffu); mc.key1 = (uint32_t)(p->philox_key >> 32);
    mc.tau2 = p->tau2;
    mc.rs_grid = p->rs_grid;
    mc.slack = tuning().slack;
    mc.tile_w = tuning().tile_w;
    mc.descriptor = p->descriptor;
    static thread_local LvlBatch B;       // ~8 KB: kept off the stack
    static thread_local XferBatch X;
    for (int k = 0; k < n; ++k)           // reset the status word and the evaluation counters
        PGM_TRY(cudaMemsetAsync(ctx[k].ws, 0, PGM_WS_EVALS_OFFSET + 8 * PGM_WS_EVALS_COUNT, st),
                "match: zero the status word and counters");
    // per level and direction: box sums of |G|^2 over the target and the
    // reference patches.  The coarsest level's come first on the caller's
    // stream; the finer levels' are forked onto an auxiliary stream, where
    // they overlap the initialisation and the coarse visits, and each is
    // joined back before the first visit at its level (the kernel time
    // profile keeps them on the caller's stream).
    Aux*& aux = fk.aux;
    bool aux_tried = false, forked = false;
    if (p->norm == PGM_L2SQ) {
        bool needed[MAXL] = {false};
        for (int v = 0; v < sch.n; ++v) needed[sch.level[v]] = true;
        const int l0 = sch.level[0];
        for (int l = p->levels - 1; l >= 0; --l) {
            if (!needed[l]) continue;
            if (l != l0 && !aux_tried && !g_prof.on) {
                aux_tried = true;
                pgm_status r = aux_get(st, &aux);
                if (r != PGM_OK) return r;
            }
            if (l != l0 && aux && !forked) {
                PGM_TRY(cudaEventRecord(aux->fork, st), "match: fork box sums");
                PGM_TRY(cudaStreamWaitEvent(aux->s, aux->fork, 0), "match: fork box sums");
                forked = true;
                fk.s_forked = true;
            }
            memset(&B, 0, sizeof(B));
            B.n = n; B.level = l;
            int max_px = 0;
            for (int k = 0; k < n; ++k)
                for (int d = 0; d < 2; ++d) {
                    fill_dir(p, ctx[k], l, d, &B.d[k][d]);
                    int np = B.d[k][d].tw * B.d[k][d].th;
                    if (np > max_px) max_px = np;
                    np = B.d[k][d].rw * B.d[k][d].rh;
                    if (np > max_px) max_px = np;
                }
            // the direction descriptor's bit-plane kernels need no box sums;
            // only a level whose search (or, at the coarsest, initialisation)
            // falls back to the int16 kernels does
            if (p->descriptor == PGM_DIR && pm_tile_fits(B, mc, nch) &&
                (l != l0 || init_bits_fits(B)))
                continue;
            const bool on_aux = l != l0 && aux;
            if (fault_due()) return injected_fail("match: box sums");
            pgm_status r = launch_box(B, nch, max_px, on_aux ? aux->s : st);
            if (r != PGM_OK) return r;
            if (on_aux) {
                PGM_TRY(cudaEventRecord(aux->lvl[l], aux->s), "match: box sums done");
                fk.box_open[l] = true;
            }
        }
    }
    for (int v = 0; v < sch.n; ++v) {
        const int l = sch.level[v];
        char rname[16];
        snprintf(rname, sizeof(rname), "level %d", l);
        Range visit_range(rname);
        if (fk.box_open[l]) {
            PGM_TRY(cudaStreamWaitEvent(st, aux->lvl[l], 0), "match: join box sums");
            fk.box_open[l] = false;
        }
        memset(&B, 0, sizeof(B));
        B.n = n; B.level = l; B.visit = v;
        int max_seeds = 0, max_half = 0;
        for (int k = 0; k < n; ++k) {
            for (int d = 0; d < 2; ++d) {
                fill_dir(p, ctx[k], l, d, &B.d[k][d]);
                int ns = B.d[k][d].nx * B.d[k][d].ny;
                int nh = ((B.d[k][d].nx + 1) / 2) * B.d[k][d].ny;
                if (ns > max_seeds) max_seeds = ns;
                if (nh > max_half) max_half = nh;
            }
            B.stream_id[k] = ctx[k].stream_id;
            B.evals[k] = reinterpret_cast<unsigned long long*>(ctx[k].ws + PGM_WS_EVALS_OFFSET);
            B.err[k] = reinterpret_cast<uint32_t*>(ctx[k].ws + ctx[k].w.off_err);
        }
        pgm_status r;
        if (fault_due()) return injected_fail(v == 0 ? "match: initialisation" : "match: transfer");
        if (v == 0) {
            r = launch_init(B, mc, nch, maxP, max_seeds, st);
        } else {
            const int src = sch.level[v - 1];
            memset(&X, 0, sizeof(X));
            X.n = n; X.up = l == src + 1; X.with_o = sch.with_o[v];
            X.prop_all = (p->ablation & PGM_ABL_PROPAGATE_ALL) ? 1 : 0;
            for (int k = 0; k < n; ++k)
                for (int d = 0; d < 2; ++d) {
                    const WsPlan& w = ctx[k].w;
                    XferDir& T = X.d[k][d];
                    T.su = reinterpret_cast<const int32_t*>(ctx[k].ws + w.off_u[src][d]);
                    T.sflags = ctx[k].ws + w.off_flags[src][d];
                    T.snx = w.nx[src][d]; T.sny = w.ny[src][d];
                    T.du = reinterpret_cast<int32_t*>(ctx[k].ws + w.off_u[l][d]);
                    T.dcost = reinterpret_cast<unsigned long long*>(ctx[k].ws + w.off_cost[l][d]);
                    T.dflags = ctx[k].ws + w.off_flags[l][d];
                    T.dnx = w.nx[l][d]; T.dny = w.ny[l][d];
                }
            r = launch_transfer(X, max_seeds, st);
        }
        if (r != PGM_OK) return r;
        // the cost refresh of the visit: by the search kernel's first
        // iteration when the tile kernel takes the batch, else on its own
        const int T = iters_at(p, l);
        const bool fused = T > 0 && pm_tile_fits(B, mc, nch);
        if (!fused) {
            if (fault_due()) return injected_fail("match: cost refresh");
            r = launch_cost_fill(B, mc, nch, maxP, max_seeds, st);
            if (r != PGM_OK) return r;
        }
        // the two directions search independently until the consistency
        // check: when each phase is one launch per direction, the backward
        // ones go on an auxiliary stream and overlap the forward ones (the
        // kernel time profile keeps them on the caller's stream)
        cudaStream_t st2 = nullptr;
        if (fused && !g_prof.on && pm_tile_split(B, mc, nch)) {
            if (!aux_tried) {
                aux_tried = true;
                r = aux_get(st, &aux);
                if (r != PGM_OK) return r;
            }
            if (aux) {
                PGM_TRY(cudaEventRecord(aux->sfork, st), "match: fork backward search");
                PGM_TRY(cudaStreamWaitEvent(aux->s2, aux->sfork, 0), "match: fork backward search");
                st2 = aux->s2;
                fk.s2_open = true;
            }
        }
        for (int t = 0; t < T; ++t)
            for (int col = 0; col < 2; ++col) {
                mc.t = t; mc.colour = col; mc.refresh = fused && t == 0;
                if (fault_due()) return injected_fail("match: search phase");
                r = launch_pm_phase(B, mc, nch, maxP, max_half, st, st2);
                if (r != PGM_OK) return r;
            }
        if (st2) {
            PGM_TRY(cudaEventRecord(aux->sjoin, st2), "match: join backward search");
            PGM_TRY(cudaStreamWaitEvent(st, aux->sjoin, 0), "match: join backward search");
            fk.s2_open = false;
        }
        mc.t = 0; mc.colour = 0; mc.refresh = 0;
        if (fault_due()) return injected_fail("match: consistency");
        r = launch_consist(B, mc, max_seeds, st);
        if (r != PGM_OK) return r;
    }
    return PGM_OK;
}

// The whole schedule on a batch.  A call that fails part-way may leave work
// forked onto the auxiliary streams; it is joined back to `st` before the
// call returns, so that none of it runs unordered after the caller's stream
// (where it could write into a workspace the caller has already released)
// and a stream capture stays joined.  On success every fork is already
// joined and nothing is added.
pgm_status run_batch(const pgm_params* p, PairCtx* ctx, int n, cudaStream_t st) {
    Forks fk;
    const pgm_status r = run_batch_forked(p, ctx, n, st, fk);
    bool box = fk.s_forked && r != PGM_OK;
    for (int l = 0; l < MAXL; ++l) box = box || fk.box_open[l];
    if (fk.aux && box) {
        cudaEventRecord(fk.aux->fork, fk.aux->s);
        cudaStreamWaitEvent(st, fk.aux->fork, 0);
    }
    if (fk.aux && fk.s2_open) {
        cudaEventRecord(fk.aux->sjoin, fk.aux->s2);
        cudaStreamWaitEvent(st, fk.aux->sjoin, 0);
    }
    if (r != PGM_OK) (void)cudaGetLastError();    // the status already reports the failure
    return r;
}

pgm_status prepare_pair(const pgm_params* p, const void* pyr1, const void* pyr2, int w1, int h1,
                        int w2, int h2, uint64_t sid, void* ws, size_t ws_bytes, PairCtx* c) {
    if (!pyr1 || !pyr2 || !ws) return PGM_ERR_ARG;
    if (w1 < 1 || h1 < 1 || w2 < 1 || h2 < 1 || w1 > 32767 || h1 > 32767 || w2 > 32767 ||
        h2 > 32767) return PGM_ERR_SIZE;
    if (!make_pyr_plan(p, w1, h1, &c->a) || !make_pyr_plan(p, w2, h2, &c->b) ||
        !make_ws_plan(p, w1, h1, w2, h2, &c->w)) return PGM_ERR_ARG;
    if (ws_bytes < c->w.bytes) return PGM_ERR_WORKSPACE;
    if (((uintptr_t)pyr1 | (uintptr_t)pyr2 | (uintptr_t)ws) & 255u) return PGM_ERR_ARG;
    for (int l = 0; l < p->levels; ++l)
        for (int d = 0; d < 2; ++d)
            if (c->w.nx[l][d] < 1 || c->w.ny[l][d] < 1) return PGM_ERR_SIZE;
    const int m = p->levels - 1;
    // exhaustive init: target raster index and cost are packed into 24 + 40 bits
    if ((long long)c->a.W[m] * c->a.H[m] >= (1LL << 24) ||
        (long long)c->b.W[m] * c->b.H[m] >= (1LL << 24)) return PGM_ERR_UNSUPPORTED;
    c->pyr1 = static_cast<const uint8_t*>(pyr1);
    c->pyr2 = static_cast<const uint8_t*>(pyr2);
    c->ws = static_cast<uint8_t*>(ws);
    c->stream_id = (uint32_t)sid;
    return PGM_OK;
}

}  // namespace
}  // namespace pgm

using namespace pgm;

extern "C" {

void pgm_default_params(pgm_params* p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->levels = 3; p->seed_stride = 3; p->patch_fwd = 15; p->patch_bwd = 11; p->sobel = 5;
    p->color = PGM_RGB; p->descriptor = PGM_FULL; p->cs_sched = PGM_CS_PAPER; p->norm = PGM_L2SQ;
    p->iters_coarse = 4; p->iters_fine = 6; p->refine_rounds = 2; p->rs_W = 2;
    for (int l = 0; l < 12; ++l) p->iters_level[l] = -1;
    p->rs_mode = PGM_RS_SYMMETRIC; p->tau2 = 1; p->min_region = 9; p->region_dmax2 = 144;
    p->max_visits = 0; p->ablation = 0; p->rs_grid = 0;
    p->philox_key = 0x5EED5EED1234ABCDull;
}

const char* pgm_status_string(pgm_status s) {
    switch (s) {
    case PGM_OK: return "ok";
    case PGM_ERR_ARG: return "invalid argument";
    case PGM_ERR_SIZE: return "image too small for the pyramid or seed lattice";
    case PGM_ERR_WORKSPACE: return "buffer smaller than required";
    case PGM_ERR_CUDA: return "CUDA error";
    case PGM_ERR_TIMEOUT: return "device wait timed out";
    case PGM_ERR_DEVICE_BOUNDS: return "device-side bounds check failed";
    case PGM_ERR_UNSUPPORTED: return "outside the library's limits";
    }
    return "unknown status";
}

size_t pgm_pyramid_bytes(const pgm_params* p, int w, int h) {
    PyrPlan pp;
    return make_pyr_plan(p, w, h, &pp) ? pp.bytes : 0;
}

pgm_status pgm_build_pyramid(const pgm_params* p, const uint8_t* d_img, int w, int h, int c,
                             size_t pitch, void* d_pyr, size_t pyr_bytes, void* stream) {
    pgm_status r = check_params(p);
    if (r != PGM_OK) return r;
    if (!d_img || !d_pyr || (c != 1 && c != 3) || (p->color == PGM_RGB && c != 3))
        return PGM_ERR_ARG;
    if (w < 1 || h < 1 || w > 32767 || h > 32767) return PGM_ERR_SIZE;
    if (pitch < (size_t)w * c || ((uintptr_t)d_pyr & 255u)) return PGM_ERR_ARG;
    PyrPlan pp;
    if (!make_pyr_plan(p, w, h, &pp)) return PGM_ERR_ARG;
    if (pyr_bytes < pp.bytes) return PGM_ERR_WORKSPACE;
    uint8_t* pyr = static_cast<uint8_t*>(d_pyr);
    Range range("pgm_build_pyramid");
    return launch_pyramid_batch(p, 1, &pp, &d_img, &c, &pitch, &pyr,
                                static_cast<cudaStream_t>(stream));
}

pgm_status pgm_build_pyramid_batch(const pgm_params* p, int n, const uint8_t* const* d_imgs,
                                   const int32_t* dims, const size_t* pitches,
                                   void* const* d_pyrs, const size_t* pyr_bytes, void* stream) {
    pgm_status r = check_params(p);
    if (r != PGM_OK) return r;
    if (n < 0 || (n > 0 && (!d_imgs || !dims || !pitches || !d_pyrs || !pyr_bytes)))
        return PGM_ERR_ARG;
    if (n == 0) return PGM_OK;
    static thread_local PyrPlan plans[PYR_MAXB];
    static thread_local int cs[PYR_MAXB];
    static thread_local uint8_t* pyrs[PYR_MAXB];
    for (int base = 0; base < n; base += PYR_MAXB) {
        const int m = n - base < PYR_MAXB ? n - base : PYR_MAXB;
        for (int k = 0; k < m; ++k) {          // every image is checked before any launch
            const int i = base + k;
            const int w = dims[3 * i], h = dims[3 * i + 1], c = dims[3 * i + 2];
            if (!d_imgs[i] || !d_pyrs[i] || (c != 1 && c != 3) || (p->color == PGM_RGB && c != 3))
                return PGM_ERR_ARG;
            if (w < 1 || h < 1 || w > 32767 || h > 32767) return PGM_ERR_SIZE;
            if (pitches[i] < (size_t)w * c || ((uintptr_t)d_pyrs[i] & 255u)) return PGM_ERR_ARG;
            if (!make_pyr_plan(p, w, h, &plans[k])) return PGM_ERR_ARG;
            if (pyr_bytes[i] < plans[k].bytes) return PGM_ERR_WORKSPACE;
        }
    }
    Range range("pgm_build_pyramid");
    for (int base = 0; base < n; base += PYR_MAXB) {
        const int m = n - base < PYR_MAXB ? n - base : PYR_MAXB;
        for (int k = 0; k < m; ++k) {
            const int i = base + k;
            make_pyr_plan(p, dims[3 * i], dims[3 * i + 1], &plans[k]);
            cs[k] = dims[3 * i + 2];
            pyrs[k] = static_cast<uint8_t*>(d_pyrs[i]);
        }
        r = launch_pyramid_batch(p, m, plans, d_imgs + base, cs, pitches + base, pyrs,
                                 static_cast<cudaStream_t>(stream));
        if (r != PGM_OK) return r;
    }
    return PGM_OK;
}

pgm_status pgm_pyramid_desc_layout(const pgm_params* p, int w, int h, int scheme, int level,
                                   size_t* offset_bytes, int* lw, int* lh, int* nch,
                                   int* row_elems, int* px_elems, int* border) {
    PyrPlan pp;
    if (!make_pyr_plan(p, w, h, &pp) || scheme < 0 || scheme > 1 || level < 0 ||
        level >= pp.L || !offset_bytes || !lw || !lh || !nch || !row_elems || !px_elems ||
        !border) return PGM_ERR_ARG;
    *offset_bytes = pp.desc_off[scheme][level];
    *lw = pp.W[level]; *lh = pp.H[level]; *nch = pp.nch; *row_elems = pp.desc_row[level];
    *px_elems = 2 * pp.pxw;
    *border = BORD;
    return PGM_OK;
}

pgm_status pgm_pyramid_image_layout(const pgm_params* p, int w, int h, int scheme, int level,
                                    size_t* offset_bytes, int* lw, int* lh, int* channels,
                                    int* row_bytes, size_t* plane_bytes) {
    PyrPlan pp;
    if (!make_pyr_plan(p, w, h, &pp) || scheme < 0 || scheme > 1 || level < 0 ||
        level >= pp.L || !offset_bytes || !lw || !lh || !channels || !row_bytes || !plane_bytes)
        return PGM_ERR_ARG;
    *offset_bytes = pp.cimg_off[scheme][level];
    *lw = pp.W[level]; *lh = pp.H[level]; *channels = pp.C;
    *row_bytes = pp.img_row[level]; *plane_bytes = pp.img_plane[level];
    return PGM_OK;
}

size_t pgm_match_workspace_bytes(const pgm_params* p, int w1, int h1, int w2, int h2) {
    WsPlan wp;
    return make_ws_plan(p, w1, h1, w2, h2, &wp) ? wp.bytes : 0;
}

pgm_status pgm_match(const pgm_params* p, const void* d_pyr1, const void* d_pyr2, int w1, int h1,
                     int w2, int h2, uint64_t stream_id, void* d_ws, size_t ws_bytes,
                     void* stream) {
    pgm_status r = check_params(p);
    if (r != PGM_OK) return r;
    static thread_local PairCtx c;
    r = prepare_pair(p, d_pyr1, d_pyr2, w1, h1, w2, h2, stream_id, d_ws, ws_bytes, &c);
    if (r != PGM_OK) return r;
    Range range("pgm_match");
    return run_batch(p, &c, 1, static_cast<cudaStream_t>(stream));
}

pgm_status pgm_match_batch(const pgm_params* p, int n, const void* const* d_pyr1,
                           const void* const* d_pyr2, const int32_t* dims,
                           const uint64_t* stream_ids, void* const* d_ws,
                           const size_t* ws_bytes, void* stream) {
    pgm_status r = check_params(p);
    if (r != PGM_OK) return r;
    if (n < 0 || (n > 0 && (!d_pyr1 || !d_pyr2 || !dims || !stream_ids || !d_ws || !ws_bytes)))
        return PGM_ERR_ARG;
    static thread_local PairCtx ctx[MAXB];
    const int chunk = tuning().chunk;
    for (int base = 0; base < n; base += chunk) {     // validate everything first
        int m = n - base < chunk ? n - base : chunk;
        for (int k = 0; k < m; ++k) {
            int i = base + k;
            r = prepare_pair(p, d_pyr1[i], d_pyr2[i], dims[4 * i], dims[4 * i + 1],
                             dims[4 * i + 2], dims[4 * i + 3], stream_ids[i], d_ws[i],
                             ws_bytes[i], &ctx[k]);
            if (r != PGM_OK) return r;
        }
    }
    Range range("pgm_match");
    for (int base = 0; base < n; base += chunk) {
        int m = n - base < chunk ? n - base : chunk;
        for (int k = 0; k < m; ++k) {
            int i = base + k;
            prepare_pair(p, d_pyr1[i], d_pyr2[i], dims[4 * i], dims[4 * i + 1], dims[4 * i + 2],
                         dims[4 * i + 3], stream_ids[i], d_ws[i], ws_bytes[i], &ctx[k]);
        }
        r = run_batch(p, ctx, m, static_cast<cudaStream_t>(stream));
        if (r != PGM_OK) return r;
    }
    return PGM_OK;
}

pgm_status pgm_field_layout(const pgm_params* p, int w1, int h1, int w2, int h2, int level,
                            int dir, int* nx, int* ny, size_t* off_u, size_t* off_cost,
                            size_t* off_flags) {
    WsPlan wp;
    if (!make_ws_plan(p, w1, h1, w2, h2, &wp) || level < 0 || level >= wp.L || dir < 0 ||
        dir > 1 || !nx || !ny || !off_u || !off_cost || !off_flags) return PGM_ERR_ARG;
    *nx = wp.nx[level][dir]; *ny = wp.ny[level][dir];
    *off_u = wp.off_u[level][dir]; *off_cost = wp.off_cost[level][dir];
    *off_flags = wp.off_flags[level][dir];
    return PGM_OK;
}

pgm_status pgm_filter(const pgm_params* p, int w1, int h1, int w2, int h2, void* d_ws,
                      size_t ws_bytes, int32_t* d_matches, int64_t max_matches,
                      int32_t* d_count, uint8_t* d_keep, void* stream) {
    pgm_status r = check_params(p);
    if (r != PGM_OK) return r;
    if (!d_ws || !d_count || max_matches < 0 || (max_matches > 0 && !d_matches))
        return PGM_ERR_ARG;
    if (((uintptr_t)d_matches) & 15u) return PGM_ERR_ARG;
    WsPlan wp;
    if (!make_ws_plan(p, w1, h1, w2, h2, &wp)) return PGM_ERR_ARG;
    if (ws_bytes < wp.bytes) return PGM_ERR_WORKSPACE;
    Range range("pgm_filter");
    return launch_filter(p, wp, static_cast<uint8_t*>(d_ws), d_matches, max_matches, d_count,
                         d_keep, static_cast<cudaStream_t>(stream));
}

pgm_status pgm_filter_batch(const pgm_params* p, int n, const int32_t* dims, void* const* d_ws,
                            const size_t* ws_bytes, int32_t* const* d_matches,
                            const int64_t* max_matches, int32_t* const* d_counts, void* stream) {
    pgm_status r = check_params(p);
    if (r != PGM_OK) return r;
    if (n < 0 || (n > 0 && (!dims || !d_ws || !ws_bytes || !d_matches || !max_matches ||
                            !d_counts)))
        return PGM_ERR_ARG;
    static thread_local FiltBatch F;
    static thread_local WsPlan wp;
    for (int i = 0; i < n; ++i) {               // every pair is checked before any launch
        if (!d_ws[i] || !d_counts[i] || max_matches[i] < 0 ||
            (max_matches[i] > 0 && !d_matches[i]) || (((uintptr_t)d_matches[i]) & 15u))
            return PGM_ERR_ARG;
        if (!make_ws_plan(p, dims[4 * i], dims[4 * i + 1], dims[4 * i + 2], dims[4 * i + 3], &wp))
            return PGM_ERR_ARG;
        if (ws_bytes[i] < wp.bytes) return PGM_ERR_WORKSPACE;
    }
    filter_consts(p, &F);
    Range range("pgm_filter");
    for (int base = 0; base < n; base += MAXB) {
        const int m = n - base < MAXB ? n - base : MAXB;
        F.n = m;
        int max_seeds = 0;
        for (int k = 0; k < m; ++k) {
            const int i = base + k;
            make_ws_plan(p, dims[4 * i], dims[4 * i + 1], dims[4 * i + 2], dims[4 * i + 3], &wp);
            filter_item(wp, static_cast<uint8_t*>(d_ws[i]), d_matches[i], max_matches[i],
                        d_counts[i], nullptr, &F.it[k]);
            const int ns = F.it[k].nx * F.it[k].ny;
            if (ns > max_seeds) max_seeds = ns;
        }
        r = launch_filter_batch(p, F, max_seeds, static_cast<cudaStream_t>(stream));
        if (r != PGM_OK) return r;
    }
    return PGM_OK;
}

pgm_status pgm_sync_status(const pgm_params* p, int w1, int h1, int w2, int h2, void* d_ws,
                           size_t ws_bytes, void* stream) {
    pgm_status r = check_params(p);
    if (r != PGM_OK) return r;
    WsPlan wp;
    if (!d_ws || !make_ws_plan(p, w1, h1, w2, h2, &wp)) return PGM_ERR_ARG;
    if (ws_bytes < wp.bytes) return PGM_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint32_t word = 0;
    PGM_TRY(cudaMemcpyAsync(&word, static_cast<uint8_t*>(d_ws) + wp.off_err, 4,
                            cudaMemcpyDeviceToHost, st), "sync_status: read the status word");
    PGM_TRY(cudaStreamSynchronize(st), "sync_status: synchronize");
    if (word != 0) {
        PGM_TRY(cudaMemsetAsync(static_cast<uint8_t*>(d_ws) + wp.off_err, 0, 4, st),
                "sync_status: clear the status word");
        return (pgm_status)word;
    }
    return PGM_OK;
}

pgm_status pgm_set_tuning(const pgm_tuning* t) {
    if (!t) { g_slack = 2; g_chunk = MAXB; g_tile_w = 8; return PGM_OK; }
    if (t->window_slack < 0 || t->window_slack > 32 || t->pairs_per_launch < 1 ||
        t->pairs_per_launch > MAXB || (t->tile_w != 4 && t->tile_w != 8 && t->tile_w != 16))
        return PGM_ERR_ARG;
    g_slack = t->window_slack;
    g_chunk = t->pairs_per_launch;
    g_tile_w = t->tile_w;
    return PGM_OK;
}

pgm_status pgm_inject_launch_failure(int steps) {
    if (steps < 0) return PGM_ERR_ARG;
    g_fail_step.store(steps, std::memory_order_relaxed);
    return PGM_OK;
}

pgm_status pgm_set_wait_limit(int64_t cycles) {
    if (cycles < 0) return PGM_ERR_ARG;
    g_wait = cycles == 0 ? WAIT_DEFAULT : (long long)cycles;
    return PGM_OK;
}

pgm_status pgm_get_tuning(pgm_tuning* t) {
    if (!t) return PGM_ERR_ARG;
    t->window_slack = g_slack;
    t->pairs_per_launch = g_chunk;
    t->tile_w = g_tile_w;
    return PGM_OK;
}

int64_t pgm_launch_count(void) { return (int64_t)g_launches.load(); }

const char* pgm_error_detail(void) { return g_detail; }

int pgm_checked_build(void) {
#ifdef PGM_CHECKED
    return 1;
#else
    return 0;
#endif
}

pgm_status pgm_profile_enable(int on) {
    if (on) {
        for (auto& e : g_prof.open) { g_prof.pool.push_back(e.a); g_prof.pool.push_back(e.b); }
        g_prof.open.clear();
        for (int k = 0; k < PGM_K_COUNT; ++k) { g_prof.ms[k] = 0; g_prof.launches[k] = 0; }
        cudaEvent_t probe = take_event();
        if (!probe) return cuda_fail("profile: event create", cudaErrorMemoryAllocation);
        g_prof.pool.push_back(probe);
    }
    g_prof.on = on != 0;
    return PGM_OK;
}

pgm_status pgm_profile_read(double* ms, int64_t* launches) {
    for (auto& e : g_prof.open) {
        PGM_TRY(cudaEventSynchronize(e.b), "profile: event synchronize");
        float t = 0.f;
        PGM_TRY(cudaEventElapsedTime(&t, e.a, e.b), "profile: elapsed time");
        g_prof.ms[e.cls] += t;
        g_prof.launches[e.cls] += e.n;
        g_prof.pool.push_back(e.a);
        g_prof.pool.push_back(e.b);
    }
    g_prof.open.clear();
    for (int k = 0; k < PGM_K_COUNT; ++k) {
        if (ms) ms[k] = g_prof.ms[k];
        if (launches) launches[k] = g_prof.launches[k];
    }
    return PGM_OK;
}

int64_t pgm_nominal_evals(const pgm_params* p, int w1, int h1, int w2, int h2) {
    WsPlan wp;
    if (!make_ws_plan(p, w1, h1, w2, h2, &wp)) return -1;
    Schedule sch;
    make_schedule(p, &sch);
    const int64_t per_it = 2 + rs_count(p->rs_W);
    int64_t total = 0;
    for (int v = 0; v < sch.n; ++v) {
        const int l = sch.level[v];
        const int64_t T = iters_at(p, l);
        for (int d = 0; d < 2; ++d) {
            const int64_t ns = (int64_t)wp.nx[l][d] * wp.ny[l][d];
            int64_t searching = ns;            // seeds that run the random search
            if (l == 0 && p->rs_grid > 0) {
                const int g = p->rs_grid, c = p->seed_stride / 2;
                int64_t gx = 0, gy = 0;
                for (int i = 0; i < wp.nx[l][d]; ++i) gx += (c + p->seed_stride * i) % g == g / 2;
                for (int j = 0; j < wp.ny[l][d]; ++j) gy += (c + p->seed_stride * j) % g == g / 2;
                searching = gx * gy;
            }
            total += ns * (1 + 2 * T) + searching * T * (per_it - 2);
        }
    }
    return total;
}

}  // extern "C"
