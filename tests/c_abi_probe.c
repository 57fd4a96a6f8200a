/* c_abi_probe.c -- a plain C99 user of include/pgm.h, built and run by
 * tests/test_c_header_cpu.py.  It makes only host-side calls (defaults,
 * status strings, size queries, argument checks), so it needs no GPU.  It
 * prints "key value" lines: the struct layouts a C compiler gives the
 * header's types, the header's constants, and what the library returns, for
 * the test to compare with the Python binding's declarations. */
#include <stddef.h>
#include <stdio.h>

#include "pgm.h"

#define FIELD(T, f) printf("off_" #T "_" #f " %zu\n", offsetof(T, f))

int main(void) {
    pgm_params p;
    pgm_interp_params ip;
    pgm_tuning t;
    int code;

    printf("sizeof_pgm_params %zu\n", sizeof(pgm_params));
    FIELD(pgm_params, levels); FIELD(pgm_params, seed_stride); FIELD(pgm_params, patch_fwd);
    FIELD(pgm_params, patch_bwd); FIELD(pgm_params, sobel); FIELD(pgm_params, color);
    FIELD(pgm_params, descriptor); FIELD(pgm_params, cs_sched); FIELD(pgm_params, norm);
    FIELD(pgm_params, iters_coarse); FIELD(pgm_params, iters_fine);
    FIELD(pgm_params, refine_rounds); FIELD(pgm_params, rs_W); FIELD(pgm_params, rs_mode);
    FIELD(pgm_params, tau2); FIELD(pgm_params, min_region); FIELD(pgm_params, region_dmax2);
    FIELD(pgm_params, max_visits); FIELD(pgm_params, ablation); FIELD(pgm_params, rs_grid);
    FIELD(pgm_params, philox_key); FIELD(pgm_params, iters_level);
    printf("sizeof_pgm_tuning %zu\n", sizeof(pgm_tuning));
    FIELD(pgm_tuning, window_slack); FIELD(pgm_tuning, pairs_per_launch); FIELD(pgm_tuning, tile_w);
    printf("sizeof_pgm_interp_params %zu\n", sizeof(pgm_interp_params));
    FIELD(pgm_interp_params, k); FIELD(pgm_interp_params, mode); FIELD(pgm_interp_params, cost_shift);
    FIELD(pgm_interp_params, la_permyriad); FIELD(pgm_interp_params, lambda);

    printf("const_PGM_NOALLOC_MAX_SEEDS %d\n", PGM_NOALLOC_MAX_SEEDS);
    printf("const_PGM_WS_EVALS_OFFSET %d\n", PGM_WS_EVALS_OFFSET);
    printf("const_PGM_WS_EVALS_COUNT %d\n", PGM_WS_EVALS_COUNT);
    printf("const_PGM_K_COUNT %d\n", PGM_K_COUNT);
    printf("const_PGM_ERR_UNSUPPORTED %d\n", (int)PGM_ERR_UNSUPPORTED);

    pgm_default_params(&p);
    printf("default_levels %d\n", p.levels);
    printf("default_patch_fwd %d\n", p.patch_fwd);
    printf("default_patch_bwd %d\n", p.patch_bwd);
    printf("default_rs_W %d\n", p.rs_W);
    printf("default_iters_level_11 %d\n", p.iters_level[11]);
    printf("default_philox_key %llu\n", (unsigned long long)p.philox_key);
    for (code = 0; code <= 7; ++code)
        printf("status_%d %s\n", code, pgm_status_string((pgm_status)code));

    p.levels = 5;
    printf("pyramid_bytes_1024x436 %zu\n", pgm_pyramid_bytes(&p, 1024, 436));
    printf("workspace_bytes_1024x436 %zu\n", pgm_match_workspace_bytes(&p, 1024, 436, 1024, 436));
    printf("nominal_evals_1024x436 %lld\n", (long long)pgm_nominal_evals(&p, 1024, 436, 1024, 436));
    /* argument checks return before any CUDA call */
    printf("match_null %d\n", (int)pgm_match(&p, NULL, NULL, 64, 64, 64, 64, 0, NULL, 0, NULL));
    p.patch_fwd = 17;
    printf("match_patch17 %d\n", (int)pgm_match(&p, (void*)256, (void*)512, 64, 64, 64, 64, 0,
                                                (void*)1024, (size_t)1 << 30, NULL));

    pgm_interp_default_params(&ip);
    printf("interp_k %d\n", ip.k);
    printf("interp_la_permyriad %d\n", ip.la_permyriad);
    printf("interp_lambda %.3f\n", ip.lambda);
    printf("interp_ws_bytes_64x48 %zu\n", pgm_interp_workspace_bytes(64, 48, &ip));

    printf("get_tuning %d\n", (int)pgm_get_tuning(&t));
    printf("tuning_tile_w %d\n", t.tile_w);
    t.tile_w = 5;
    printf("set_tuning_bad %d\n", (int)pgm_set_tuning(&t));
    printf("checked_build %d\n", pgm_checked_build());
    return 0;
}
