/*
 * sc5_cpu_twopass.c -- the timed CPU baseline of the benchmark: the two-pass
 * form of the separable width-5 convolution in FP32 on every host core.
 *
 * It follows the loop structure of the paper's OpenMP two-pass code
 * (Sec. 5.1 and Listing 1): planes one after another; for each plane a
 * parallel loop over rows runs the horizontal 1-D pass into an FP32
 * intermediate, then a second parallel loop over rows runs the vertical 1-D
 * pass; the inner loops over columns are plain unit-stride loops the
 * compiler vectorises.  Two departures, both stated in the benchmark's
 * documentation: the horizontal pass covers every row (the listing leaves
 * the first and last two rows of the intermediate unwritten while the
 * vertical pass reads them), and the result goes to a separate VALID image
 * ((H-4) x (W-4) per plane) instead of back into the input.
 *
 * This file is benchmark infrastructure: it shares no code with the CUDA
 * library or with the FP64 oracle.  Build: gcc -O3 -fopenmp -fPIC -shared.
 */
#include <stddef.h>
#include <stdint.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads an OpenMP parallel region gets (1 without OpenMP). */
int sc5cpu_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * A: [P][H][W] FP32 input, T: [H][W-4] FP32 scratch (one plane), B: [P][H-4][W-4]
 * FP32 output; k: the 5 taps, tap t on offset t-2.  Returns 0, or -1 for a
 * shape below 5 x 5.
 */
int sc5cpu_two_pass(const float *A, int64_t P, int64_t H, int64_t W, const float *k, float *T, float *B)
{
    if (P < 1 || H < 5 || W < 5) return -1;
    const int64_t Wv = W - 4, Hv = H - 4;
    const float k0 = k[0], k1 = k[1], k2 = k[2], k3 = k[3], k4 = k[4];
    for (int64_t p = 0; p < P; ++p) {
        const float *a = A + p * H * W;
        float *b = B + p * Hv * Wv;
#pragma omp parallel for schedule(static)
        for (int64_t y = 0; y < H; ++y) {
            const float *r = a + y * W;
            float *t = T + y * Wv;
            for (int64_t x = 0; x < Wv; ++x)
                t[x] = r[x] * k0 + r[x + 1] * k1 + r[x + 2] * k2 + r[x + 3] * k3 + r[x + 4] * k4;
        }
#pragma omp parallel for schedule(static)
        for (int64_t y = 0; y < Hv; ++y) {
            const float *t0 = T + y * Wv;
            float *o = b + y * Wv;
            for (int64_t x = 0; x < Wv; ++x)
                o[x] = t0[x] * k0 + t0[x + Wv] * k1 + t0[x + 2 * Wv] * k2 + t0[x + 3 * Wv] * k3 +
                       t0[x + 4 * Wv] * k4;
        }
    }
    return 0;
}
