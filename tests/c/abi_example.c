/*
 * A plain C user of libsepconv5: only <sepconv5.h> and the CUDA runtime.
 *   abi_example host   -- host-only calls (no GPU needed): the compiled
 *                         shapes, a refused descriptor, the error message.
 *   abi_example gpu    -- convolve a 3 x 67 x 133 image with k = e_2 (the
 *                         identity tap) and check the result equals the
 *                         interior of the input exactly: through a plan,
 *                         one pyramid REDUCE step, and the serving calls
 *                         (the output buffer is named at submission and
 *                         holds the result once serve_poll returns OK).
 * Prints "OK" and exits 0 on success.
 */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime.h>

#include "sepconv5.h"

static int host_checks(void)
{
    int32_t cfg[3 * 32], n = 0;
    if (sepconv5_fused_configs(SC5_F32, SC5_F32, cfg, 32, &n) != SC5_OK || n < 1) {
        fprintf(stderr, "fused_configs failed: %s\n", sepconv5_last_error());
        return 1;
    }
    if (cfg[1] != 128) return 1;
    sc5_plan_desc d;
    memset(&d, 0, sizeof d);
    d.planes = 3;
    d.H = 4; /* too small */
    d.W = 64;
    d.in_pitch = 64;
    d.out_pitch = 60;
    sc5_plan p = NULL;
    if (sepconv5_plan(&d, &p) != SC5_EINVAL || p != NULL) return 1;
    if (strlen(sepconv5_last_error()) == 0) return 1;
    return 0;
}

static int gpu_checks(void)
{
    const int P = 3, H = 67, W = 133, pitch = 136, Hv = H - 4, Wv = W - 4;
    const size_t n_in = (size_t)P * H * pitch, n_out = (size_t)P * Hv * Wv;
    float *a = (float *)malloc(n_in * sizeof(float)), *b = (float *)malloc(n_out * sizeof(float));
    for (size_t i = 0; i < n_in; ++i) a[i] = (float)((i * 2654435761u) % 256u);
    float *da = NULL, *db = NULL;
    if (cudaMalloc((void **)&da, n_in * sizeof(float)) != cudaSuccess) return 1;
    if (cudaMalloc((void **)&db, n_out * sizeof(float)) != cudaSuccess) return 1;
    cudaMemcpy(da, a, n_in * sizeof(float), cudaMemcpyHostToDevice);
    sc5_plan_desc d;
    memset(&d, 0, sizeof d);
    d.planes = P;
    d.H = H;
    d.W = W;
    d.in_pitch = pitch;
    d.out_pitch = Wv;
    d.in_dtype = d.out_dtype = SC5_F32;
    d.border = SC5_BORDER_VALID;
    d.algo = SC5_ALGO_FUSED;
    sc5_plan p = NULL;
    if (sepconv5_plan(&d, &p) != SC5_OK) {
        fprintf(stderr, "plan: %s\n", sepconv5_last_error());
        return 1;
    }
    const float k[5] = {0.f, 0.f, 1.f, 0.f, 0.f};
    if (sepconv5_run(p, da, db, k, 1.f, 1.f, NULL) != SC5_OK) {
        fprintf(stderr, "run: %s\n", sepconv5_last_error());
        return 1;
    }
    int32_t code = 0;
    if (sepconv5_device_status(NULL, &code) != SC5_OK) return 1;
    cudaMemcpy(b, db, n_out * sizeof(float), cudaMemcpyDeviceToHost);
    for (int pl = 0; pl < P; ++pl)
        for (int y = 0; y < Hv; ++y)
            for (int x = 0; x < Wv; ++x)
                if (b[((size_t)pl * Hv + y) * Wv + x] != a[((size_t)pl * H + y + 2) * pitch + x + 2]) {
                    fprintf(stderr, "mismatch at %d %d %d\n", pl, y, x);
                    return 1;
                }
    int32_t th = 0, tw = 0, st = 0, ctas = 0;
    if (sepconv5_plan_info(p, &th, &tw, &st, &ctas) != SC5_OK || th < 1 || tw < 1 || st < 1 || ctas < 1) return 1;
    sepconv5_plan_destroy(p);

    /* one REDUCE step through the pyramid calls: with the centre tap alone the
       level is the input at every second row and column from (2, 2) */
    sc5_pyramid_desc pd;
    memset(&pd, 0, sizeof pd);
    pd.planes = P;
    pd.H = H;
    pd.W = W;
    pd.in_pitch = pitch;
    pd.in_dtype = pd.out_dtype = SC5_F32;
    pd.levels = 1;
    sc5_pyramid pyr = NULL;
    if (sepconv5_pyramid_create(&pd, &pyr) != SC5_OK) {
        fprintf(stderr, "pyramid: %s\n", sepconv5_last_error());
        return 1;
    }
    int32_t h1 = 0, w1 = 0;
    int64_t p1 = 0;
    if (sepconv5_pyramid_level(pyr, 1, &h1, &w1, &p1) != SC5_OK) return 1;
    if (h1 != (H - 3) / 2 || w1 != (W - 3) / 2 || p1 < w1 || (p1 * 4) % 16) return 1;
    float *dl = NULL;
    if (cudaMalloc((void **)&dl, (size_t)P * h1 * p1 * sizeof(float)) != cudaSuccess) return 1;
    void *levels[1] = {dl};
    if (sepconv5_pyramid_run(pyr, da, levels, k, 1.f, 1.f, NULL) != SC5_OK) {
        fprintf(stderr, "pyramid run: %s\n", sepconv5_last_error());
        return 1;
    }
    if (sepconv5_device_status(NULL, &code) != SC5_OK) return 1;
    float *l = (float *)malloc((size_t)P * h1 * p1 * sizeof(float));
    cudaMemcpy(l, dl, (size_t)P * h1 * p1 * sizeof(float), cudaMemcpyDeviceToHost);
    for (int pl = 0; pl < P; ++pl)
        for (int y = 0; y < h1; ++y)
            for (int x = 0; x < w1; ++x)
                if (l[((size_t)pl * h1 + y) * p1 + x] != a[((size_t)pl * H + 2 * y + 2) * pitch + 2 * x + 2]) {
                    fprintf(stderr, "pyramid mismatch at %d %d %d\n", pl, y, x);
                    return 1;
                }
    sepconv5_pyramid_destroy(pyr);
    free(l);

    /* serving: two requests of the same image in page-locked host memory */
    float *hin = NULL, *hout[2] = {NULL, NULL};
    if (cudaMallocHost((void **)&hin, n_in * sizeof(float)) != cudaSuccess) return 1;
    for (int r = 0; r < 2; ++r)
        if (cudaMallocHost((void **)&hout[r], n_out * sizeof(float)) != cudaSuccess) return 1;
    memcpy(hin, a, n_in * sizeof(float));
    sc5_serve_cfg sc;
    memset(&sc, 0, sizeof sc);
    sc.hbm_budget_bytes = (size_t)64 << 20;
    sc.max_inflight = 4;
    sc.dtype = SC5_F32;
    sc.planes = P;
    sc.n_streams = 1;
    sc.max_merge = 8;
    sc.merge = 1;
    sc5_server srv = NULL;
    if (serve_create(&sc, &srv) != SC5_OK) {
        fprintf(stderr, "serve_create: %s\n", sepconv5_last_error());
        return 1;
    }
    uint64_t tickets[2];
    for (int r = 0; r < 2; ++r) {
        sc5_image im;
        memset(&im, 0, sizeof im);
        im.in = hin;
        im.out = hout[r];
        im.H = H;
        im.W = W;
        im.in_pitch = pitch;
        im.out_pitch = Wv;
        memcpy(im.k, k, sizeof k);
        im.in_scale = im.out_scale = 1.f;
        if (serve_submit(srv, &im, &tickets[r]) != SC5_OK) {
            fprintf(stderr, "serve_submit: %s\n", sepconv5_last_error());
            return 1;
        }
    }
    for (int r = 0; r < 2; ++r) {
        double lat = 0.0;
        if (serve_poll(srv, tickets[r], -1, &lat) != SC5_OK || !(lat > 0.0)) {
            fprintf(stderr, "serve_poll: %s\n", sepconv5_last_error());
            return 1;
        }
        for (int pl = 0; pl < P; ++pl)
            for (int y = 0; y < Hv; ++y)
                for (int x = 0; x < Wv; ++x)
                    if (hout[r][((size_t)pl * Hv + y) * Wv + x] != a[((size_t)pl * H + y + 2) * pitch + x + 2]) {
                        fprintf(stderr, "served mismatch at %d %d %d\n", pl, y, x);
                        return 1;
                    }
    }
    double lat = 0.0;
    if (serve_poll(srv, tickets[0], 0, &lat) != SC5_ENOTFOUND) return 1; /* retired */
    if (serve_destroy(srv) != SC5_OK) return 1;
    cudaFreeHost(hin);
    cudaFreeHost(hout[0]);
    cudaFreeHost(hout[1]);
    cudaFree(dl);
    cudaFree(da);
    cudaFree(db);
    free(a);
    free(b);
    return 0;
}

int main(int argc, char **argv)
{
    const int gpu = argc > 1 && strcmp(argv[1], "gpu") == 0;
    if (host_checks()) {
        fprintf(stderr, "host checks failed\n");
        return 1;
    }
    if (gpu && gpu_checks()) {
        fprintf(stderr, "gpu checks failed\n");
        return 1;
    }
    printf("OK\n");
    return 0;
}
