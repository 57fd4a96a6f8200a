/*
 * pgm.h -- C ABI of the GB300 (sm_103a) hot path of Pyramidal Gradient
 * Matching (Li, "Pyramidal Gradient Matching for Optical Flow Estimation",
 * arXiv 1704.03217).
 *
 * Problem statement (Sec. III): given two images I1, I2, build their
 * gradient pyramids (Sec. III-A Eq. 1-2, Sec. III-D, Table 2), compute a
 * forward field F: I1 -> I2 and a backward field I2 -> I1 on a regular seed
 * lattice by coarse-to-fine limited PatchMatch (Sec. III-B Eq. 3-5, Sec. III-D
 * Eq. 6-8, Fig. 5), filter outliers by forward-backward consistency and small
 * region removal (Sec. III-E), and export the surviving matches
 * (Sec. III-G).
 *
 * Conventions (all entry points):
 *  - The caller owns every buffer; the library allocates no memory.  "d_"
 *    pointers are device pointers of the current CUDA device; others are
 *    host pointers.
 *  - Work is enqueued asynchronously on `stream` (a cudaStream_t; NULL is
 *    the legacy default stream).  The returned status covers argument checks
 *    and launch errors only; device-side failures are recorded in the
 *    workspace's error word and reported by pgm_sync_status().
 *  - pgm_match and pgm_match_batch fork part of their work onto two streams
 *    of the library's own: the box sums of the finer levels and the
 *    backward direction's search phases.  The pair of streams belongs to
 *    the caller's `stream` (created on first use, per host thread and
 *    device, up to 32 caller streams per thread; calls on further streams
 *    do not fork).  Each fork starts from an event recorded on `stream` and
 *    is joined back to `stream` by an event wait before the call returns,
 *    so all of the call's work stays ordered on `stream` and is captured
 *    with it into a CUDA graph.
 *  - Nothing throws across the ABI.  Calls on different workspaces may run
 *    concurrently from different host threads.
 *  - Results are a deterministic function of (params, images, stream_id):
 *    all arithmetic is integer and the random search draws from a
 *    counter-based generator (Philox4x32-10) keyed by params.philox_key.
 */
#ifndef PGM_H
#define PGM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PGM_OK = 0,
    PGM_ERR_ARG = 1,           /* NULL pointer, bad enum value, bad parameter */
    PGM_ERR_SIZE = 2,          /* image too small for the pyramid / lattice   */
    PGM_ERR_WORKSPACE = 3,     /* buffer smaller than the *_bytes query       */
    PGM_ERR_CUDA = 4,          /* a CUDA launch or API call failed            */
    PGM_ERR_TIMEOUT = 5,       /* a bounded device wait ran out               */
    PGM_ERR_DEVICE_BOUNDS = 6, /* a device-side index check failed            */
    PGM_ERR_UNSUPPORTED = 7    /* valid but outside the library's limits      */
} pgm_status;

enum { PGM_GRAY = 0, PGM_RGB = 1 };                 /* params.color           */
enum { PGM_FULL = 0, PGM_DIR = 1, PGM_SECTOR = 2 }; /* params.descriptor      */
enum { PGM_CS_PAPER = 0, PGM_CS_PLAIN = 1 };        /* params.cs_sched        */
enum { PGM_L2SQ = 0, PGM_L1 = 1 };                  /* params.norm            */
enum { PGM_RS_SYMMETRIC = 0, PGM_RS_PAPER_FLOOR = 1 }; /* params.rs_mode      */
enum { PGM_ABL_NO_REFINE = 1, PGM_ABL_PROPAGATE_ALL = 2, PGM_ABL_NO_OUTLIER_PROP = 4 };

/* Method parameters.  Defaults (pgm_default_params) are the paper's
 * (Sec. IV: W=2, S=5, L=3, s=1/2, N=2, m=L-1, 4 iterations per level and 6 at
 * full resolution; Sec. III-E: r=7 forward, r=5 backward, regions < 9
 * removed, motion difference < 12 px), on a seed lattice of stride 3. */
typedef struct {
    int32_t levels;        /* L, 1..12 pyramid levels, downsample 1/2      */
    int32_t seed_stride;   /* sigma >= 1: lattice stride in level pixels,
                              seeds at c + sigma*i with c = sigma/2         */
    int32_t patch_fwd;     /* patch side P (1..16) of the forward field    */
    int32_t patch_bwd;     /* patch side P (1..16) of the backward field   */
    int32_t sobel;         /* S in {3, 5} (Eq. 1)                          */
    int32_t color;         /* PGM_GRAY (PGM-G/GD) or PGM_RGB (PGM-C/CD)    */
    int32_t descriptor;    /* PGM_FULL gradient, PGM_DIR (G ./ |G|) or
                              PGM_SECTOR (uniform 8-sector angle, coded as
                              integer unit vectors; beyond the paper)      */
    int32_t cs_sched;      /* PGM_CS_PAPER: Table 2 colour spaces per level
                              and direction; PGM_CS_PLAIN: RGB throughout  */
    int32_t norm;          /* PGM_L2SQ (Eq. 3) or PGM_L1                   */
    int32_t iters_coarse;  /* propagation+search iterations at levels > 0  */
    int32_t iters_fine;    /* ... at level 0                               */
    int32_t refine_rounds; /* N, rounds of refinement between m and m-1    */
    int32_t rs_W;          /* W >= 1, limited random-search radius (Eq. 5) */
    int32_t rs_mode;       /* PGM_RS_SYMMETRIC or PGM_RS_PAPER_FLOOR       */
    int32_t tau2;          /* consistency threshold |u_f + u_b|^2 <= tau2  */
    int32_t min_region;    /* regions with fewer seeds are removed         */
    int32_t region_dmax2;  /* 4-neighbours join a region iff |du|^2 < this */
    int32_t max_visits;    /* 0: whole schedule; k > 0: stop after k visits */
    int32_t ablation;      /* PGM_ABL_* bits (Table 1 rows)                */
    int32_t rs_grid;       /* 0: random search at every seed; g > 0: at
                              level 0 only at seeds whose pixel x and y are
                              both == g/2 (mod g) (PGM-C3/G3: g = 3)       */
    uint64_t philox_key;   /* key of the random-search stream              */
    int32_t iters_level[12]; /* per-level iteration counts: entry l >= 0
                              replaces iters_coarse / iters_fine at level l;
                              -1 (the default) keeps them; at most 32767   */
} pgm_params;

/* Fill *p with the defaults above.  Never fails for a non-NULL p. */
void pgm_default_params(pgm_params* p);

/* Static description of a status code. */
const char* pgm_status_string(pgm_status s);

/* For the last PGM_ERR_CUDA returned to the calling host thread: the library
 * step and the CUDA error behind it ("" if there was none).  The text stays
 * valid until the thread's next failing call.  Never fails. */
const char* pgm_error_detail(void);

/* ------------------------------------------------------------------ */
/* Gradient pyramid (Sec. III-A Eq. 1-2, Sec. III-D, Sec. III-E Table 2) */
/* ------------------------------------------------------------------ */

/* Bytes of the pyramid buffer of one w x h image (0 on invalid input).
 * The layout depends only on (params, w, h). */
size_t pgm_pyramid_bytes(const pgm_params* p, int w, int h);

/* Build the gradient pyramid of one image.
 *   d_img: w x h pixels, c = 1 (gray) or 3 (interleaved RGB) uint8 channels,
 *          rows `pitch` bytes apart (pitch >= w*c).
 *   d_pyr: device buffer of at least pgm_pyramid_bytes(p, w, h) bytes,
 *          256-byte aligned; overwritten.
 * Levels: I^{l+1} = 5-tap binomial of I^l decimated by 2 (W_{l+1} =
 * ceil(W_l/2)); PGM_GRAY converts RGB to gray first; PGM_RGB converts each
 * level to the colour space of Table 2 for the forward and the backward
 * direction; then Sobel gradients (int16) and, for PGM_DIR, their signs.
 * Errors: PGM_ERR_ARG (NULL, c not 1/3, PGM_RGB with c = 1, bad params),
 * PGM_ERR_WORKSPACE (pyr_bytes too small), PGM_ERR_CUDA. */
pgm_status pgm_build_pyramid(const pgm_params* p, const uint8_t* d_img, int w, int h, int c,
                             size_t pitch, void* d_pyr, size_t pyr_bytes, void* stream);

/* Build the pyramids of n images (same params, sizes may differ) in shared
 * launches: one launch per pyramid step for the whole batch.  Host arrays of
 * length n: d_imgs[i]; dims[3*i..3*i+2] = (w, h, c); pitches[i] (bytes);
 * d_pyrs[i] (256-byte aligned); pyr_bytes[i].  Each result equals
 * pgm_build_pyramid on that image alone.  Every image is checked before any
 * launch; errors as pgm_build_pyramid. */
pgm_status pgm_build_pyramid_batch(const pgm_params* p, int n, const uint8_t* const* d_imgs,
                                   const int32_t* dims, const size_t* pitches,
                                   void* const* d_pyrs, const size_t* pyr_bytes, void* stream);

/* Where one level's descriptor lives inside a pyramid buffer (for tests and
 * tools): int16 values, pixel-interleaved, `nch` = 2C channels per pixel in
 * the order Gx of each colour channel, then Gy of each, pixels `px_elems`
 * int16 apart (8 for 6 channels, the last two zero; 2 for 2 channels), rows
 * `row_elems` int16 apart.  offset_bytes locates pixel (0, 0); the array has
 * a border of `border` pixels on every side that repeats the nearest image
 * pixel (Sec. III-B patches read outside the image take the border value).
 * scheme 0 serves the forward field, 1 the backward field (equal to 0 unless
 * PGM_RGB with PGM_CS_PAPER). */
pgm_status pgm_pyramid_desc_layout(const pgm_params* p, int w, int h, int scheme, int level,
                                   size_t* offset_bytes, int* lw, int* lh, int* nch,
                                   int* row_elems, int* px_elems, int* border);
/* Where one level's colour-converted uint8 image lives: C planes of lh rows,
 * rows `row_bytes` apart, planes `plane_bytes` apart. */
pgm_status pgm_pyramid_image_layout(const pgm_params* p, int w, int h, int scheme, int level,
                                    size_t* offset_bytes, int* lw, int* lh, int* channels,
                                    int* row_bytes, size_t* plane_bytes);

/* ------------------------------------------------------------------ */
/* Pyramidal matching (Sec. III-B Eq. 3-5, Sec. III-D Eq. 6-8, Fig. 5)  */
/* ------------------------------------------------------------------ */

/* Bytes of the match workspace for a w1 x h1 -> w2 x h2 pair (0 on
 * invalid input). */
size_t pgm_match_workspace_bytes(const pgm_params* p, int w1, int h1, int w2, int h2);

/* Run the whole coarse-to-fine schedule on one pair.
 *   d_pyr1, d_pyr2: pyramids of I1 (w1 x h1) and I2 (w2 x h2) built with
 *                   the same params.
 *   stream_id:      low 32 bits enter the random-search counter, so that
 *                   different pairs draw independent numbers.
 *   d_ws:           >= pgm_match_workspace_bytes, 256-byte aligned; it
 *                   receives the fields of every level and both directions
 *                   and must be kept for pgm_filter / pgm_field_layout.  Its
 *                   contents on entry do not matter: the call first clears
 *                   the status word and the evaluation counters, so
 *                   pgm_sync_status then reports this call's device-side
 *                   failures.
 * Schedule (m = L-1): exhaustive nearest-neighbour init at m, then
 * [m-1, m] x N with field and outlier record, then m-1 with the field only,
 * then m-2 .. 0.  Each visit: cost of the current field, `iters` iterations
 * of propagation + limited random search (checkerboard order), consistency
 * check, outlier-record update, then the transfer to the next level.
 * Errors: PGM_ERR_ARG, PGM_ERR_SIZE (a level has no seed), PGM_ERR_WORKSPACE,
 * PGM_ERR_UNSUPPORTED (patch > 16, coarsest level over 2^24 pixels),
 * PGM_ERR_CUDA. */
pgm_status pgm_match(const pgm_params* p, const void* d_pyr1, const void* d_pyr2,
                     int w1, int h1, int w2, int h2, uint64_t stream_id,
                     void* d_ws, size_t ws_bytes, void* stream);

/* Run pgm_match on n independent pairs in shared launches (pairs may have
 * different sizes; each has its own pyramids and workspace).  Arrays are
 * host arrays of length n: d_pyr1[i], d_pyr2[i], dims[4*i..4*i+3] = (w1, h1,
 * w2, h2), d_ws[i] (each >= pgm_match_workspace_bytes of that pair),
 * stream_ids[i].  The result of every pair equals pgm_match on that pair
 * alone.  Same errors as pgm_match, checked for every pair before any
 * launch. */
pgm_status pgm_match_batch(const pgm_params* p, int n, const void* const* d_pyr1,
                           const void* const* d_pyr2, const int32_t* dims,
                           const uint64_t* stream_ids, void* const* d_ws,
                           const size_t* ws_bytes, void* stream);

/* Where the state of one level and direction (0 forward, 1 backward) lives
 * in a match workspace: nx x ny seeds in raster order; u: int32 per seed,
 * low 16 bits ux, high 16 bits uy (two's complement); cost: uint64 per seed
 * (meaningful where valid); flags: uint8 per seed, bit 0 initialised, bit 1
 * outlier (O^l), bit 2 outlier record initialised. */
pgm_status pgm_field_layout(const pgm_params* p, int w1, int h1, int w2, int h2, int level,
                            int dir, int* nx, int* ny, size_t* off_u, size_t* off_cost,
                            size_t* off_flags);

/* ------------------------------------------------------------------ */
/* Final filter (Sec. III-E small-region removal, Sec. III-G export)    */
/* ------------------------------------------------------------------ */

/* On the level-0 forward field of a workspace filled by pgm_match: inlier
 * seeds (outlier record "no") that are lattice 4-neighbours join a region
 * iff |u_s - u_t|^2 < region_dmax2; regions with fewer than min_region seeds
 * are removed.  The survivors are written in lattice raster order as rows
 * (x1, y1, x2, y2) int32 of level-0 pixel coordinates to d_matches
 * [max_matches][4]; *d_count (device int32) receives the number of
 * survivors, which may exceed max_matches (then only max_matches rows are
 * written).  d_keep (optional, may be NULL): one uint8 per level-0 forward
 * seed, 1 = kept.
 * Errors: PGM_ERR_ARG, PGM_ERR_WORKSPACE, PGM_ERR_CUDA. */
pgm_status pgm_filter(const pgm_params* p, int w1, int h1, int w2, int h2, void* d_ws,
                      size_t ws_bytes, int32_t* d_matches, int64_t max_matches,
                      int32_t* d_count, uint8_t* d_keep, void* stream);

/* pgm_filter on n workspaces in shared launches (six in all).  Host arrays
 * of length n: dims[4*i..4*i+3] = (w1, h1, w2, h2); d_ws[i], ws_bytes[i];
 * d_matches[i] ([max_matches[i]][4] int32, 16-byte aligned); d_counts[i]
 * (device int32).  Each result equals pgm_filter on that workspace alone.
 * Every pair is checked before any launch; errors as pgm_filter. */
pgm_status pgm_filter_batch(const pgm_params* p, int n, const int32_t* dims, void* const* d_ws,
                            const size_t* ws_bytes, int32_t* const* d_matches,
                            const int64_t* max_matches, int32_t* const* d_counts, void* stream);

/* The same final filter for callers that cannot allocate device memory.
 * The paper has no counterpart; this is a deployment convenience.
 *
 * pgm_filter needs its scratch (region labels, region sizes, scan partial
 * sums) inside the caller's match workspace.  Some callers cannot provide
 * such a buffer: code that runs where allocation is forbidden or unsafe --
 * inside another framework's enqueue callback, in a real-time loop whose
 * memory budget is fixed up front, or next to an allocator that owns all of
 * the device's memory -- and that only holds the level-0 forward field.
 * This entry point takes that field and writes the matches, with its scratch
 * in a fixed array that the library itself places in device memory when it
 * is loaded (PGM_NOALLOC_MAX_SEEDS seeds, 8 MiB + 16 KiB per device, held
 * until the process exits).  It calls no cudaMalloc, cudaFree or other
 * allocating routine.
 *   d_u, d_flags: the nx x ny level-0 forward field, laid out as
 *                 pgm_field_layout describes (packed int32 displacement,
 *                 uint8 flags); read only.
 *   d_matches, max_matches, d_count: as for pgm_filter.
 * Result: identical to pgm_filter on the workspace holding that field.
 * A call made outside a stream capture looks up the array's device address
 * with the device current (so calls after a cudaDeviceReset find the
 * array's new place); a call inside a capture uses the address an earlier
 * call on that device found, so make one call before any stream capture.
 * All calls share the one array and it keeps the last call's contents
 * (every call re-initialises what it reads), so calls whose work overlaps
 * on the GPU -- e.g. on two streams at once -- race and must be serialised.
 * Errors: PGM_ERR_ARG (NULL pointer, nx or ny < 0, d_matches not 16-byte
 * aligned, d_u or d_count not 4-byte aligned; checked before anything is
 * launched), PGM_ERR_UNSUPPORTED (nx * ny > PGM_NOALLOC_MAX_SEEDS),
 * PGM_ERR_CUDA. */
#define PGM_NOALLOC_MAX_SEEDS (1 << 20)
pgm_status pgm_filter_noalloc(const pgm_params* p, int nx, int ny, const int32_t* d_u,
                              const uint8_t* d_flags, int32_t* d_matches, int64_t max_matches,
                              int32_t* d_count, void* stream);

/* Wait for `stream` and return the device-side status recorded in the
 * workspace (PGM_OK, PGM_ERR_TIMEOUT or PGM_ERR_DEVICE_BOUNDS), clearing
 * it.  Synchronising call. */
pgm_status pgm_sync_status(const pgm_params* p, int w1, int h1, int w2, int h2, void* d_ws,
                           size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------ */
/* Observability (no counterpart in the paper)                          */
/* ------------------------------------------------------------------ */

/* Workspace header: bytes [0, 4) hold the device status word; bytes
 * [8, 72) eight uint64 counters of patch distances (Eq. 3) actually
 * evaluated: propagation/search forward, backward; cost refresh forward,
 * backward; exhaustive initialisation forward, backward; and, of the
 * propagation/search and refresh ones, those scored outside the
 * shared-memory window (from global memory) forward, backward.  pgm_match
 * and pgm_match_batch zero them, and the status word, at their start. */
#define PGM_WS_EVALS_OFFSET 8
#define PGM_WS_EVALS_COUNT 8

/* Kernel classes for pgm_profile_read. */
enum { PGM_K_PYRAMID = 0, PGM_K_INIT = 1, PGM_K_COST = 2, PGM_K_PM = 3, PGM_K_CONSIST = 4,
       PGM_K_TRANSFER = 5, PGM_K_FILTER = 6, PGM_K_COUNT = 7 };

/* Number of kernels this library has launched in this process (all
 * threads, all devices).  Never fails. */
int64_t pgm_launch_count(void);

/* Start (on = 1) or stop (on = 0) per-kernel-class timing of the calling
 * host thread: while on, each kernel launch is bracketed by a CUDA event
 * pair recorded on its stream.  Starting clears the accumulated times.
 * Meant for profiling runs, not for timed runs (the events cost a little).
 * Errors: PGM_ERR_CUDA if an event cannot be created. */
pgm_status pgm_profile_enable(int on);

/* Wait for the recorded events and return, per kernel class, the summed
 * device milliseconds ms[PGM_K_COUNT] and launch counts
 * launches[PGM_K_COUNT] since the last pgm_profile_enable(1) (either
 * pointer may be NULL).  Errors: PGM_ERR_CUDA. */
pgm_status pgm_profile_read(double* ms, int64_t* launches);

/* Result-invariant tuning knobs (no counterpart in the paper): they change
 * only how work is laid out on the GPU, never a result.  Process-wide; set
 * them between calls, not while other threads launch.
 *   window_slack: margin (pixels, 0..32) of the shared-memory target window
 *                 around a tile's median match (default 2); candidates
 *                 outside it are scored from global memory.
 *   pairs_per_launch: pairs sharing one launch in pgm_match_batch (1..32,
 *                 default 32).
 *   tile_w:       seeds per row of a search tile: 4, 8 (default) or 16; a
 *                 tile holds 64 lattice seeds (tile_w x 64 / tile_w) and
 *                 stages one shared-memory window. */
typedef struct {
    int32_t window_slack;
    int32_t pairs_per_launch;
    int32_t tile_w;
} pgm_tuning;
/* NULL restores the defaults.  Errors: PGM_ERR_ARG (value out of range). */
pgm_status pgm_set_tuning(const pgm_tuning* t);
pgm_status pgm_get_tuning(pgm_tuning* t);

/* Limit, in SM clock cycles, of every bounded wait inside the search kernel
 * (a consumer waiting for a staged tile, the producer waiting for a free
 * buffer); 0 restores the default of 2^31 cycles (about a second).  A wait
 * that runs out sets PGM_ERR_TIMEOUT in the workspace status word
 * (pgm_sync_status) and ends the kernel's work early; the copies already in
 * flight are still waited for (with the default limit) before a block exits.
 * Process-wide; meant for failure-detection tests (a limit of a few cycles
 * makes the first wait run out).  Errors: PGM_ERR_ARG (cycles < 0). */
pgm_status pgm_set_wait_limit(int64_t cycles);

/* Host-side fault injection, for failure-handling tests (no counterpart in
 * the paper).  Counting from this call, over the following pgm_match and
 * pgm_match_batch calls of every thread, the `steps`-th launch step of the
 * matching schedule (the box sums of a level, the initialisation or a
 * transfer, a cost refresh, a colour phase, a consistency check) is not
 * enqueued: that call returns PGM_ERR_CUDA at once, pgm_error_detail names
 * the step, and the work the call had already enqueued -- including what it
 * forked onto its auxiliary streams -- is joined back to its stream, as on
 * any failure part-way through a call.  The failure fires once; 0 disarms.
 * Nothing reaches the GPU.  Errors: PGM_ERR_ARG (steps < 0). */
pgm_status pgm_inject_launch_failure(int steps);

/* 1 in the checked build (libpgm_checked.so, compiled with -DPGM_CHECKED):
 * the search, initialisation and consistency kernels check their shared-
 * and global-memory indices; a failed check sets PGM_ERR_DEVICE_BOUNDS in the
 * workspace status word (pgm_sync_status) and skips the access.  0 in the
 * regular build, where the checks compile away. */
int pgm_checked_build(void);

/* Nominal candidate evaluations of one pair under params (2 propagation + K
 * random-search candidates per seed and iteration, one cost per seed and
 * visit, both directions; the exhaustive init is not counted). */
int64_t pgm_nominal_evals(const pgm_params* p, int w1, int h1, int w2, int h2);

/* ---- sparse-to-dense interpolation (Sec. III-G) ---------------------------
 * The paper densifies its grid-3 matches with EpicFlow: an edge-aware
 * geodesic distance, then a Nadaraya-Watson (NW) average or a locally
 * weighted affine (LA) fit over a pixel's nearest matches, LA when the
 * matches exceed 2.2 % of the image size.  Here every pixel of image 1 takes
 * its k geodesically nearest matches, the geodesic step between 4-neighbours
 * p, q costing c(p) + c(q) with c = 1 + (sum of |g| over the level-0
 * descriptor channels of image 1) >> cost_shift, ties of distance going to
 * the smaller match index; weights exp(-(d - d_nearest) / lambda); LA falls
 * back to NW where its normal equations are degenerate.  The distances and
 * neighbour lists are exact integers; the interpolation runs in double
 * precision and is stored as float. */
enum { PGM_INTERP_AUTO = 0, PGM_INTERP_NW = 1, PGM_INTERP_LA = 2 };
typedef struct {
    int32_t k;             /* neighbours per pixel, 1..16 (default 16)      */
    int32_t mode;          /* PGM_INTERP_AUTO: LA iff n * 10^4 >
                              la_permyriad * w * h (n = matches), else NW;
                              PGM_INTERP_NW / PGM_INTERP_LA force one      */
    int32_t cost_shift;    /* 0..31 (default 10)                           */
    int32_t la_permyriad;  /* default 220 (2.2 %)                          */
    double lambda;         /* > 0, distance scale of the weights (32)      */
} pgm_interp_params;
void pgm_interp_default_params(pgm_interp_params* ip);
/* Workspace bytes for a w x h image (0: invalid size or k). */
size_t pgm_interp_workspace_bytes(int w, int h, const pgm_interp_params* ip);
/* Dense flow of image 1 (w x h, the size d_pyr1 was built for under p) from
 * the exported matches: d_matches [max_matches][4] int32 (x1, y1, x2, y2),
 * *d_count of them valid (the count pgm_filter wrote; at most max_matches
 * are read; match positions outside the image are ignored, two at one pixel
 * keep the first).  d_flow: [h][w][2] float (x, y displacement; 0 where no
 * match is reachable).  d_ws: pgm_interp_workspace_bytes, 256-byte aligned;
 * it holds, at offset 0, the k nearest matches of every pixel as
 * [h][w][k] uint64 keys d << 32 | index in ascending order (all ones where
 * fewer are reachable).  The call synchronises the stream (the relaxation
 * repeats until nothing changes), so it cannot be captured in a graph.
 * Errors: PGM_ERR_ARG, PGM_ERR_WORKSPACE, PGM_ERR_CUDA, PGM_ERR_UNSUPPORTED
 * (the relaxation did not settle within its launch bound). */
pgm_status pgm_interpolate(const pgm_params* p, const void* d_pyr1, int w, int h,
                           const int32_t* d_matches, const int32_t* d_count, int64_t max_matches,
                           const pgm_interp_params* ip, void* d_ws, size_t ws_bytes,
                           float* d_flow, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PGM_H */
