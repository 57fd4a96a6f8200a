// pgm_device.cuh -- internal declarations shared by the CUDA translation
// units of libpgm (host plans, kernel argument blocks, launchers).
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/pgm.h"

namespace pgm {

constexpr int MAXL = 12;         // pyramid levels supported
constexpr int MAXB = 32;         // pairs per batched launch
constexpr int MAXP = 16;         // largest patch side
constexpr int MAXVIS = 4 * MAXL + 2 * 64 + 4;
// Descriptor arrays carry a replicated border of BORD pixels on every side,
// so that any patch (P <= MAXP) whose centre lies inside the image can be
// read without clamping.  A colour pixel takes 4 words (6 int16 values and
// one zero word, 16 bytes), a gray pixel 1 word.
constexpr int BORD = MAXP / 2;
__host__ __device__ constexpr int px_words(int nch) { return nch == 2 ? 1 : 4; }

// seed flag bits
constexpr uint8_t F_VALID = 1;   // field initialised at this seed
constexpr uint8_t F_OUTL = 2;    // outlier record O^l = yes
constexpr uint8_t F_OINIT = 4;   // O^l came with a red arrow (Eq. 6 "initialized")

enum Space { SP_GRAY = 0, SP_RGB = 1, SP_LAB = 2, SP_YCRCB = 3 };

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// ---------------------------------------------------------------- plans
struct PyrPlan {
    int L, C, nsch, nch;
    int W[MAXL], H[MAXL];
    size_t img_off[MAXL];        // level image, C planes of uint8
    int img_row[MAXL];           // bytes per row
    size_t img_plane[MAXL];      // bytes per plane
    int space[2][MAXL];
    size_t cimg_off[2][MAXL];    // colour-converted image (aliases img if identity)
    size_t desc_off[2][MAXL];    // int16 descriptors, pixel-interleaved: pixel (0, 0)
    size_t split_off[2][MAXL];   // same words with each value split into two signed bytes
    size_t desc_pad_off[2][MAXL];    // start of the padded arrays (pixel (-BORD, -BORD))
    size_t split_pad_off[2][MAXL];
    int desc_row[MAXL];          // int16 elements per padded row (also 16-bit halves of a split row)
    int pxw;                     // 32-bit words per pixel (px_words)
    // direction descriptor only: two bit-planes per scheme and level (nonzero,
    // then sign), rows of bit_row words covering the padded row of the
    // descriptor, bit (x + BORD) * nch + c of row y + BORD for value c of
    // pixel (x, y); the sign plane follows the nonzero plane's H + 2 BORD rows
    size_t bits_off[2][MAXL];
    int bit_row[MAXL];           // words per bit-plane row (a multiple of 4), 0: no planes
    size_t bytes;
};

struct WsPlan {
    int L;
    int nx[MAXL][2], ny[MAXL][2];
    size_t off_u[MAXL][2], off_cost[MAXL][2], off_flags[MAXL][2];
    size_t off_sa2[MAXL][2];     // per seed: sum of |G|^2 over its reference patch
    size_t off_sb2[MAXL][2];     // per target pixel: sum of |G|^2 over the patch there
    int sbp[MAXL][2];            // row pitch (elements, even) of the target sums
    size_t off_sa2img[MAXL][2];  // per reference pixel: sum of |G|^2 over the patch there
    size_t off_err;              // uint32 device status word
    size_t off_label, off_size, off_bsum;   // filter scratch (level-0 forward lattice)
    int nblk0;                   // blocks of the level-0 forward lattice scan
    size_t bytes;
};

struct Schedule {
    int n;
    int level[MAXVIS];
    int with_o[MAXVIS];          // transfer into this visit carries O (Eq. 8)
};

// Programmatic dependent launch along the matching loop (search phases,
// consistency, transfer): a kernel launched with launch_pdl may start while
// the previous kernel of its stream is still running; it runs its prologue
// (shared memory and barrier set-up), then pdl_wait() blocks until that kernel
// has completed and its writes are visible, before any global memory access.
// pdl_trigger() lets the next kernel start early.  Without the launch
// attribute both are no-ops.  PGM_PDL=0 in the environment turns the
// attribute off (same results).
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_trigger() {
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
#endif
bool pdl_enabled();
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = pdl_enabled() ? 1 : 0;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<Args&&>(args)...);
}

// Record, for this host thread, which CUDA call failed and how
// (pgm_error_detail), and return PGM_ERR_CUDA.
pgm_status cuda_fail(const char* site, cudaError_t e);
// The status after kernel launches: PGM_OK, or PGM_ERR_CUDA recorded at site.
inline pgm_status launch_status(const char* site) {
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PGM_OK : cuda_fail(site, e);
}
#define PGM_TRY(call, site)                                         \
    do {                                                            \
        const cudaError_t pgm_e_ = (call);                          \
        if (pgm_e_ != cudaSuccess) return ::pgm::cuda_fail(site, pgm_e_); \
    } while (0)

// Allow kernel `kern` the device's largest dynamic shared memory per block.
// The limit is an attribute of the kernel on the current device, shared by
// every host thread, so it is raised once per (kernel, device) to the
// maximum (a launch still uses only what it asks for) and never lowered.
pgm_status smem_opt_in(const void* kern);

pgm_status check_params(const pgm_params* p);
bool make_pyr_plan(const pgm_params* p, int w, int h, PyrPlan* pp);
bool make_ws_plan(const pgm_params* p, int w1, int h1, int w2, int h2, WsPlan* wp);
void make_schedule(const pgm_params* p, Schedule* s);
inline int lattice_n(int W, int sigma) {
    int c = sigma / 2;
    return (W - 1 - c) >= 0 ? (W - 1 - c) / sigma + 1 : 0;
}
// iterations of a visit at level l: the per-level count when set, else
// iters_fine at level 0 and iters_coarse above
inline int iters_at(const pgm_params* p, int l) {
    return p->iters_level[l] >= 0 ? p->iters_level[l] : l == 0 ? p->iters_fine : p->iters_coarse;
}
inline int rs_count(int W) { int K = 0; for (int w = W; w >= 1; w >>= 1) ++K; return K; }

// ------------------------------------------------------- kernel blocks
// One direction of one pair at one level.
struct DirLvl {
    const int16_t* ref;          // descriptor of the reference image (this dir), pixel (0, 0)
    const int16_t* tgt;          // descriptor of the target image, pixel (0, 0)
    const uint32_t* ref_split;   // reference descriptor in split-byte form, pixel (0, 0)
    int32_t ref_pitch, tgt_pitch;// int16 elements per (padded) row
    int32_t rw, rh, tw, th;      // reference / target image size
    int32_t nx, ny;              // lattice of this direction (on the reference)
    int32_t onx, ony;            // lattice of the other direction
    int32_t P;                   // patch side
    int32_t sbp;                 // row pitch (elements) of sb2
    int32_t* u;                  // packed displacement (ux low 16, uy high 16)
    unsigned long long* cost;
    uint8_t* flags;
    const int32_t* ou;           // other direction: displacement
    const uint8_t* oflags;       //                  flags
    unsigned long long* sa2;     // per seed: sum over the reference patch of |G|^2
    unsigned long long* sb2;     // per target pixel (row pitch sbp): same over the target patch
    unsigned long long* sa2img;  // per reference pixel (row pitch rw): sum over its patch
    const uint32_t* ref_bits;    // direction descriptor: bit-planes of the reference (padded row 0)
    const uint32_t* tgt_bits;    //                       ... of the target
    int32_t rbit_row, tbit_row;  // words per bit-plane row (0: no planes)
};

struct LvlBatch {
    int32_t n;                   // pairs in this launch
    int32_t level, visit, pad;
    DirLvl d[MAXB][2];
    uint32_t stream_id[MAXB];
    unsigned long long* evals[MAXB];       // workspace header counters (include/pgm.h)
    uint32_t* err[MAXB];                   // workspace status words (pgm_sync_status)
};

// One direction of one pair for the transfer between levels.
struct XferDir {
    const int32_t* su; const uint8_t* sflags; int32_t snx, sny;
    int32_t* du; unsigned long long* dcost; uint8_t* dflags; int32_t dnx, dny;
};
struct XferBatch {
    int32_t n, up, with_o, prop_all;
    XferDir d[MAXB][2];
};

struct MatchConst {              // scalars common to one launch
    int32_t sigma, c;            // lattice stride and offset
    int32_t norm, rs_W, rs_mode, K;
    uint32_t key0, key1;
    int32_t t, colour, tau2, rs_grid;   // rs_grid > 0: level-0 search on that grid only
    int32_t slack;                      // tuning: target-window margin of the tile kernels
    int32_t refresh;                    // search phase also scores the current matches first
    int32_t cost_only;                  // score the current matches only (a visit without iterations)
    int32_t descriptor;                 // PGM_FULL, PGM_DIR (bit-plane search), PGM_SECTOR
    int32_t tile_w;                     // tuning: seeds per search-tile row (64 per tile)
};

// result-invariant tuning knobs (pgm_set_tuning)
struct Tuning { int slack; int chunk; int tile_w; };
Tuning tuning();

// Device index checks of the checked build (-DPGM_CHECKED, libpgm_checked.so):
// a check that fails records PGM_ERR_DEVICE_BOUNDS in the status word errp
// and evaluates to false, so the caller skips the access.  In the regular
// build a check is the constant true.
#ifdef PGM_CHECKED
#define PGM_CHECK(cond, errp) \
    ((cond) ? true : (atomicOr((errp), (unsigned)PGM_ERR_DEVICE_BOUNDS), false))
#else
#define PGM_CHECK(cond, errp) true
#endif

// A host-side NVTX push/pop range: names the entry point and, inside
// pgm_match, the visit's level on a profiler's timeline (and lets a profiler
// select the kernels of one level).  Costs a pointer test when no tool is
// attached.
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

// Brackets the launches of one kernel class: counts them and, while
// pgm_profile_enable(1) is on for this thread, records an event pair.
struct KScope {
    KScope(int cls, cudaStream_t st, int nlaunch = 1);
    ~KScope();
    int cls; cudaStream_t st; int n; int slot;
};

// ------------------------------------------------------------ launchers
// pyramid.cu
constexpr int PYR_MAXB = 64;      // images per pyramid launch
struct PyrItem {                  // one image in one pyramid launch
    const uint8_t* src;
    uint8_t* dst;
    uint32_t* split;              // Sobel: split-byte copy of the descriptor (pixel (0, 0))
    int sw, sh, srow;             // source level size and row bytes
    int dw, dh, drow;             // destination level size and row bytes / int16 elements
                                  // (Sobel: dst, split point at pixel (0, 0) of padded arrays)
    size_t splane, dplane;        // plane strides
    size_t pitch;                 // level 0: input row bytes
    int mode;                     // level 0: input mode; colour conversion: target space
    int pad;
    uint32_t* bits;               // Sobel, direction descriptor: bit-planes (padded row 0)
    int brow;                     // words per bit-plane row
    int pad2;
};
struct PyrBatch { int n; int pad; PyrItem it[PYR_MAXB]; };
pgm_status launch_pyramid_batch(const pgm_params* p, int n, const PyrPlan* plans,
                                const uint8_t* const* imgs, const int* cs, const size_t* pitches,
                                uint8_t* const* pyrs, cudaStream_t st);
// match.cu
pgm_status launch_init(const LvlBatch& B, const MatchConst& mc, int nch, int maxP,
                       int max_seeds, cudaStream_t st);
pgm_status launch_cost_fill(const LvlBatch& B, const MatchConst& mc, int nch, int maxP,
                            int max_seeds, cudaStream_t st);
// st2 (may be null): the stream of the backward direction when pm_tile_split
// says the phase runs one launch per direction
pgm_status launch_pm_phase(const LvlBatch& B, const MatchConst& mc, int nch, int maxP,
                           int max_seeds, cudaStream_t st, cudaStream_t st2);
pgm_status launch_consist(const LvlBatch& B, const MatchConst& mc, int max_seeds,
                          cudaStream_t st);
pgm_status launch_transfer(const XferBatch& X, int max_seeds, cudaStream_t st);
pgm_status launch_box(const LvlBatch& B, int nch, int max_pixels, cudaStream_t st);
// pm_row.cu (search and cost refresh on staged tiles) and init_tile.cu:
// exhaustive init, squared L2, target image staged in shared memory;
// *handled = false when it does not apply (the caller uses the direct kernel)
// (*nlaunch: the kernels launched)
pgm_status launch_init_tile(const LvlBatch& B, const MatchConst& mc, int nch, bool* handled,
                            cudaStream_t st, int* nlaunch);
// init_tc.cu: the same initialisation on the tensor cores (six channels,
// squared L2, patches up to 15 x 15); *handled = false when it does not apply
pgm_status launch_init_tc(const LvlBatch& B, const MatchConst& mc, int nch, bool* handled,
                          cudaStream_t st, int* nlaunch);
// true when the tile search kernel takes this batch (it then also does the
// cost refresh of a visit's first iteration, MatchConst::refresh)
bool pm_tile_fits(const LvlBatch& B, const MatchConst& mc, int nch);
// init_tile.cu: the bit-plane initialisation takes this batch (planes present,
// staged target fits in shared memory)
bool init_bits_fits(const LvlBatch& B);
// true when the tile search kernel takes this batch with one launch per
// direction (phases larger than one tile per resident CTA)
bool pm_tile_split(const LvlBatch& B, const MatchConst& mc, int nch);
pgm_status launch_pm_tile(const LvlBatch& B, const MatchConst& mc, int nch, int maxP, int* nlaunch,
                          bool* handled, cudaStream_t st, cudaStream_t st2);
pgm_status launch_cost_tile(const LvlBatch& B, const MatchConst& mc, int nch, bool* handled,
                            cudaStream_t st);
// filter.cu
struct FiltItem {                 // the level-0 forward field of one pair
    const uint8_t* flags;
    const int32_t* u;
    int* label; int* size; int* bsum;   // scratch
    int nx, ny;
    int32_t* rows;
    long long max_rows;
    int32_t* count;
    uint8_t* keep;                // optional
};
struct FiltBatch {
    int n, sigma, c, dmax2, min_region, pad;
    FiltItem it[MAXB];
};
pgm_status launch_filter_batch(const pgm_params* p, const FiltBatch& F, int max_seeds,
                               cudaStream_t st);
void filter_item(const WsPlan& wp, uint8_t* d_ws, int32_t* d_matches, int64_t max_matches,
                 int32_t* d_count, uint8_t* d_keep, FiltItem* it);
void filter_consts(const pgm_params* p, FiltBatch* F);
pgm_status launch_filter_ptrs(const pgm_params* p, int nx, int ny, const int32_t* u,
                              const uint8_t* flags, int* label, int* size, int* bsum,
                              int32_t* d_matches, int64_t max_matches, int32_t* d_count,
                              cudaStream_t st);
pgm_status launch_filter(const pgm_params* p, const WsPlan& wp, uint8_t* d_ws,
                         int32_t* d_matches, int64_t max_matches, int32_t* d_count,
                         uint8_t* d_keep, cudaStream_t st);

}  // namespace pgm
