/* c_match_pair.c -- the whole hot path of include/pgm.h from plain C, with
 * no Python and no PyTorch: device memory from cudaMalloc, the legacy default
 * stream.  Built and run by tests/test_c_pipeline_gpu.py.
 *
 *   c_match_pair W H LEVELS COLOR DESCRIPTOR img1.rgb img2.rgb out.bin
 *
 * img*.rgb: W x H interleaved RGB bytes; COLOR and DESCRIPTOR set
 * pgm_params.color and .descriptor (the paper's defaults otherwise).  The
 * pyramid buffers and the match workspace are filled with 0xff before use
 * (their contents on entry must not matter).  out.bin:
 * int32 count, then count rows (x1, y1, x2, y2) int32.  Exit status 0 on
 * success; otherwise a message names the failing step. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include "pgm.h"

static int fail_pgm(const char* step, pgm_status s) {
    fprintf(stderr, "%s: %s [%s]\n", step, pgm_status_string(s), pgm_error_detail());
    return 1;
}

static int fail_cuda(const char* step, cudaError_t e) {
    fprintf(stderr, "%s: %s\n", step, cudaGetErrorString(e));
    return 1;
}

static unsigned char* read_file(const char* path, size_t n) {
    FILE* f = fopen(path, "rb");
    unsigned char* buf = malloc(n);
    if (!f || !buf || fread(buf, 1, n, f) != n) {
        if (f) fclose(f);
        free(buf);
        return NULL;
    }
    fclose(f);
    return buf;
}

int main(int argc, char** argv) {
    int w, h, levels, nx = 0, ny = 0, rc = 1;
    size_t img_bytes, pyr_bytes, ws_bytes, off_u, off_cost, off_flags;
    unsigned char *h1 = NULL, *h2 = NULL;
    int32_t count = 0, *rows = NULL;
    void *d_img1 = NULL, *d_img2 = NULL, *d_pyr1 = NULL, *d_pyr2 = NULL, *d_ws = NULL;
    void *d_rows = NULL, *d_count = NULL;
    pgm_params p;
    pgm_status s;
    cudaError_t e;
    FILE* out;

    if (argc != 9) {
        fprintf(stderr, "usage: %s W H LEVELS COLOR DESCRIPTOR img1.rgb img2.rgb out.bin\n",
                argv[0]);
        return 2;
    }
    w = atoi(argv[1]);
    h = atoi(argv[2]);
    levels = atoi(argv[3]);
    img_bytes = (size_t)w * h * 3;
    h1 = read_file(argv[6], img_bytes);
    h2 = read_file(argv[7], img_bytes);
    if (!h1 || !h2) {
        fprintf(stderr, "cannot read the images\n");
        goto done;
    }

    pgm_default_params(&p);            /* the paper's settings */
    p.levels = levels;
    p.color = atoi(argv[4]);
    p.descriptor = atoi(argv[5]);
    pyr_bytes = pgm_pyramid_bytes(&p, w, h);
    ws_bytes = pgm_match_workspace_bytes(&p, w, h, w, h);
    if (!pyr_bytes || !ws_bytes) {
        fprintf(stderr, "invalid size or parameters\n");
        goto done;
    }
    s = pgm_field_layout(&p, w, h, w, h, 0, 0, &nx, &ny, &off_u, &off_cost, &off_flags);
    if (s != PGM_OK) { rc = fail_pgm("pgm_field_layout", s); goto done; }

    if ((e = cudaMalloc(&d_img1, img_bytes)) != cudaSuccess ||
        (e = cudaMalloc(&d_img2, img_bytes)) != cudaSuccess ||
        (e = cudaMalloc(&d_pyr1, pyr_bytes)) != cudaSuccess ||
        (e = cudaMalloc(&d_pyr2, pyr_bytes)) != cudaSuccess ||
        (e = cudaMalloc(&d_ws, ws_bytes)) != cudaSuccess ||
        (e = cudaMalloc(&d_rows, (size_t)nx * ny * 16)) != cudaSuccess ||
        (e = cudaMalloc(&d_count, 4)) != cudaSuccess) {
        rc = fail_cuda("cudaMalloc", e);
        goto done;
    }
    if ((e = cudaMemcpy(d_img1, h1, img_bytes, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(d_img2, h2, img_bytes, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(d_pyr1, 0xff, pyr_bytes)) != cudaSuccess ||
        (e = cudaMemset(d_pyr2, 0xff, pyr_bytes)) != cudaSuccess ||
        (e = cudaMemset(d_ws, 0xff, ws_bytes)) != cudaSuccess) {
        rc = fail_cuda("copy in", e);
        goto done;
    }

    s = pgm_build_pyramid(&p, d_img1, w, h, 3, (size_t)w * 3, d_pyr1, pyr_bytes, NULL);
    if (s != PGM_OK) { rc = fail_pgm("pgm_build_pyramid 1", s); goto done; }
    s = pgm_build_pyramid(&p, d_img2, w, h, 3, (size_t)w * 3, d_pyr2, pyr_bytes, NULL);
    if (s != PGM_OK) { rc = fail_pgm("pgm_build_pyramid 2", s); goto done; }
    s = pgm_match(&p, d_pyr1, d_pyr2, w, h, w, h, 7, d_ws, ws_bytes, NULL);
    if (s != PGM_OK) { rc = fail_pgm("pgm_match", s); goto done; }
    s = pgm_filter(&p, w, h, w, h, d_ws, ws_bytes, d_rows, (int64_t)nx * ny, d_count, NULL, NULL);
    if (s != PGM_OK) { rc = fail_pgm("pgm_filter", s); goto done; }
    s = pgm_sync_status(&p, w, h, w, h, d_ws, ws_bytes, NULL);
    if (s != PGM_OK) { rc = fail_pgm("pgm_sync_status", s); goto done; }

    if ((e = cudaMemcpy(&count, d_count, 4, cudaMemcpyDeviceToHost)) != cudaSuccess) {
        rc = fail_cuda("copy the count out", e);
        goto done;
    }
    if (count < 0 || count > nx * ny) {
        fprintf(stderr, "bad match count %d\n", (int)count);
        goto done;
    }
    rows = malloc((size_t)(count > 0 ? count : 1) * 16);
    if (!rows) goto done;
    if ((e = cudaMemcpy(rows, d_rows, (size_t)count * 16, cudaMemcpyDeviceToHost)) != cudaSuccess) {
        rc = fail_cuda("copy the rows out", e);
        goto done;
    }
    out = fopen(argv[8], "wb");
    if (!out) goto done;
    if (fwrite(&count, 4, 1, out) != 1 || fwrite(rows, 16, (size_t)count, out) != (size_t)count) {
        fclose(out);
        goto done;
    }
    fclose(out);
    rc = 0;

done:
    cudaFree(d_img1); cudaFree(d_img2); cudaFree(d_pyr1); cudaFree(d_pyr2);
    cudaFree(d_ws); cudaFree(d_rows); cudaFree(d_count);
    free(h1); free(h2); free(rows);
    return rc;
}
