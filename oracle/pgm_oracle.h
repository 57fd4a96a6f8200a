/*
 * pgm_oracle.h -- plain, slow, single-threaded CPU oracle for Pyramidal
 * Gradient Matching (Li, arXiv 1704.03217).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA path; the two are compared
 * element by element on the same seeded inputs.
 *
 * Every function follows the paper's definitions directly (the equation or
 * section is cited at each function).  Where the paper is silent the
 * documented reading (R1..R20 in the design notes) is taken; each such place
 * says which reading it implements.
 */
#ifndef PGM_ORACLE_H
#define PGM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Parameter block.  Field order and meaning mirror the public library's
 * parameter struct, but this is an independent declaration. */
typedef struct {
    int32_t levels;        /* L, pyramid levels                           */
    int32_t seed_stride;   /* sigma, seed lattice stride in level pixels  */
    int32_t patch_fwd;     /* P for the forward field (2r+1, r=7 -> 15)   */
    int32_t patch_bwd;     /* P for the backward field (r=5 -> 11)        */
    int32_t sobel;         /* S: 3 or 5                                   */
    int32_t color;         /* 0 gray (PGM-G/GD), 1 colour (PGM-C/CD)      */
    int32_t descriptor;    /* 0 full gradient, 1 direction only,
                              2 uniform 8-sector angle                    */
    int32_t cs_sched;      /* 0 Table 2 colour-space schedule, 1 RGB only */
    int32_t norm;          /* 0 squared L2 (Eq. 3), 1 L1                  */
    int32_t iters_coarse;  /* propagation+search iterations at l > 0      */
    int32_t iters_fine;    /* ... at l = 0                                */
    int32_t refine_rounds; /* N                                           */
    int32_t rs_W;          /* W, random search radius                     */
    int32_t rs_mode;       /* 0 symmetric offsets, 1 literal floor        */
    int32_t tau2;          /* consistency threshold, squared level pixels */
    int32_t min_region;    /* regions smaller than this are removed       */
    int32_t region_dmax2;  /* neighbours join a region iff |du|^2 < this  */
    int32_t max_visits;    /* 0: whole schedule; k > 0: stop after k visits */
    int32_t ablation;      /* bit 0: no refinement, bit 1: propagate all,
                              bit 2: no outlier-record propagation        */
    int32_t rs_grid;       /* 0: search at every seed; g > 0: at level 0 only
                              where x and y are both == g/2 (mod g)        */
    uint64_t philox_key;
    int32_t iters_level[12]; /* entry l >= 0: iterations at level l in place
                                of iters_coarse / iters_fine; -1: unset    */
} orc_params;

enum { ORC_SCHED_CHECKERBOARD = 0, ORC_SCHED_SEQUENTIAL = 1 };
enum { ORC_SP_GRAY = 0, ORC_SP_RGB = 1, ORC_SP_LAB = 2, ORC_SP_YCRCB = 3 };

/* ---- single steps, exposed for the pins ---- */
void     orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
uint32_t orc_icbrt(uint64_t v);
/* rgb: interleaved n x 3; out: interleaved n x (space == GRAY ? 1 : 3) */
void     orc_convert(int space, const uint8_t* rgb, int64_t n, uint8_t* out);
void     orc_pyr_down(const uint8_t* in, int w, int h, uint8_t* out);
void     orc_sobel(const uint8_t* in, int w, int h, int S, int16_t* gx, int16_t* gy);
/* 8-sector angle code of a gradient as an integer unit vector (x64) */
void     orc_sector(int gx, int gy, int16_t out[2]);
uint64_t orc_patch_dist(const int16_t* A, int wa, int ha, const int16_t* B, int wb, int hb,
                        int nch, int ax, int ay, int bx, int by, int P, int norm);
int32_t  orc_rs_offset(uint32_t r, int k, int W, int mode);
/* one cell of the inter-level transfer, Eq. 7-8: out = (ux, uy, valid, outlier) */
void     orc_xfer_cell(int up, int n, const int32_t* ux, const int32_t* uy, const uint8_t* valid,
                       const uint8_t* outl, int prop_all, int32_t out[4]);

/* ---- gradient pyramid of one image (Sec. III-A, III-D, III-E) ---- */
typedef struct orc_pyr orc_pyr;
orc_pyr*       orc_pyr_build(const orc_params* p, const uint8_t* img, int w, int h, int c);
void           orc_pyr_free(orc_pyr* py);
int            orc_pyr_levels(const orc_pyr* py);
int            orc_pyr_schemes(const orc_pyr* py);
int            orc_pyr_channels(const orc_pyr* py);   /* C: 1 or 3 */
void           orc_pyr_dims(const orc_pyr* py, int level, int* w, int* h);
/* image pyramid before colour conversion, planar [C][h][w] */
const uint8_t* orc_pyr_image(const orc_pyr* py, int level);
/* colour-converted level image, planar [C][h][w] */
const uint8_t* orc_pyr_cimage(const orc_pyr* py, int scheme, int level);
/* descriptor, planar [2C][h][w]: planes 0..C-1 = Gx per channel, C..2C-1 = Gy */
const int16_t* orc_pyr_desc(const orc_pyr* py, int scheme, int level);

/* ---- pyramidal matching (Sec. III-B, III-D) ---- */
typedef struct orc_match orc_match;
orc_match* orc_match_run(const orc_params* p, const orc_pyr* p1, const orc_pyr* p2,
                         int schedule, uint64_t stream_id);
void       orc_match_free(orc_match* m);
int        orc_match_visits(const orc_match* m);        /* visits actually run */
int        orc_match_visit_level(const orc_match* m, int v);
int64_t    orc_match_evals(const orc_match* m);         /* patch distances evaluated */
void       orc_field_dims(const orc_match* m, int level, int dir, int* nx, int* ny);
/* Copy out one field: any pointer may be NULL. */
void       orc_field_get(const orc_match* m, int level, int dir, int32_t* ux, int32_t* uy,
                         uint8_t* valid, uint64_t* cost, uint8_t* outlier, uint8_t* oinit);

/* ---- final filter (Sec. III-E region removal, Sec. III-G grid export) ---- */
/* rows: [max_rows][4] (x1, y1, x2, y2); returns the number of matches (may
 * exceed max_rows, in which case only max_rows are written). keep: optional
 * per-seed 0/1 of the level-0 forward lattice. */
/* Region removal and export on a level-0 forward field given as arrays of
 * nx x ny seeds (raster order): ux, uy displacements, valid and outlier flags
 * (0/1).  Same rule and output as orc_filter. */
int64_t orc_filter_arrays(const orc_params* p, int nx, int ny, const int32_t* ux,
                          const int32_t* uy, const uint8_t* valid, const uint8_t* outl,
                          int32_t* rows, int64_t max_rows, uint8_t* keep_out);
int64_t orc_filter(const orc_params* p, const orc_match* m, int32_t* rows, int64_t max_rows,
                   uint8_t* keep);

/* ---- sparse-to-dense interpolation (Sec. III-G; readings R23-R25) -------- */
/* Per-pixel step cost of the geodesic distance (R23): 1 + (sum over the
 * descriptor channels of |g|) >> shift.  desc: nch planes of w x h int16. */
void orc_interp_cost(const int16_t* desc, int nch, int w, int h, int shift, uint32_t* cost);
/* The K geodesically nearest matches of every pixel (R24): 4-connected grid,
 * a step between neighbours p, q costs cost[p] + cost[q]; match i sits at
 * (sx[i], sy[i]) (a position given twice keeps the smaller index).  keys:
 * w x h x K, ascending, key = d << 32 | i, UINT64_MAX where fewer than K
 * matches are reachable.  Returns 0, or -1 when out of memory. */
int orc_interp_knn(int w, int h, const uint32_t* cost, const int32_t* sx, const int32_t* sy,
                   int64_t n, int K, uint64_t* keys);
/* Flow of every pixel from its K nearest matches (R25): weights
 * exp(-(d - d_nearest) / lambda); use_la = 0 Nadaraya-Watson average, 1
 * weighted affine fit evaluated at the pixel (Nadaraya-Watson where the fit
 * is degenerate).
 * fx, fy: the matches' displacements.  flow: w x h x 2 (0 where no match is
 * reachable). */
void orc_interp_flow(int w, int h, int K, const uint64_t* keys, const int32_t* sx,
                     const int32_t* sy, const int32_t* fx, const int32_t* fy, double lambda,
                     int use_la, double* flow);

#ifdef __cplusplus
}
#endif
#endif
