/*
 * sepconv5_oracle.c -- plain, slow FP64 CPU oracle for the separable width-5
 * convolution of planar images (arXiv 1711.09791, "2D Image Convolution using
 * Three Parallel Programming Models on the Xeon Phi").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this code;
 * only the test suite, the smoke check and the timed CPU baseline of the
 * benchmark use it.  It shares no header, helper, table or constant with the
 * CUDA library.
 *
 * Every routine here is the plain definition, written for checking by eye:
 *
 *   Eq. 1 (Sec. 1):       B[y][x] = sum_i sum_j A[y+i][x+j] * K[i][j]
 *   separable kernel:     K[i][j] = k[i] * k[j]           (Sec. 1, below Eq. 1)
 *   width 5 kernel:       taps t = 0..4 act at offset t-2 (Eq. 2, Sec. 5.2;
 *                         Listing 1 puts k[0] on column j-2 and k[4] on j+2)
 *   interior only:        output starts at input pixel (2,2); edges are
 *                         ignored (Sec. 5, first paragraph)
 *   two-pass form:        a horizontal 1D pass into an intermediate, then a
 *                         vertical 1D pass (Sec. 5.1; Listing 1)
 *
 * Readings of the paper taken here:
 *   - The operation is a correlation: tap t weights offset t-2 on both axes;
 *     the first index of K runs along rows (Eq. 2: A[i+kx-2][j+ky-2]*K[kx][ky]).
 *   - The result is the VALID region: plane p of the output is (H-4) x (W-4)
 *     and output (y, x) is centred on input (y+2, x+2).
 *   - The horizontal pass covers all H rows (Listing 2 has no row guard in
 *     that pass), so the two-pass form equals Eq. 1 on the whole VALID region.
 *
 * Precision: all arithmetic in IEEE double.  Reduced-precision inputs are
 * decoded exactly to double first (the decoders below follow the published
 * bit layouts of bfloat16, IEEE binary16 and OCP FP8 E4M3).
 *
 * Layout: every image is planar and dense, [P][H][W] row-major doubles; the
 * VALID output is dense [P][H-4][W-4]; the horizontal-pass intermediate is
 * dense [P][H][W-4].  Return 0 on success, -1 on bad sizes.
 */
#include <stdint.h>
#include <string.h>
#include <math.h>

#define SC5O_TAPS 5

/* K[i][j] = k[i] * k[j]  (Sec. 1: the matrix of a separable convolution vector). */
void sc5o_outer(const double k[SC5O_TAPS], double K[SC5O_TAPS * SC5O_TAPS])
{
    for (int i = 0; i < SC5O_TAPS; ++i)
        for (int j = 0; j < SC5O_TAPS; ++j)
            K[i * SC5O_TAPS + j] = k[i] * k[j];
}

/*
 * Single-pass (direct) form, Eq. 1 with a general 5x5 matrix K, four nested
 * loops as in Sec. 5.1 ("single-pass algorithm"): for every VALID output
 * pixel, sum over the kernel rows i and columns j of A[y+i][x+j] * K[i][j],
 * where (y, x) indexes the VALID output and so A[y+i][x+j] is the input at
 * offset (i-2, j-2) from the centre (y+2, x+2).
 */
int sc5o_direct_K(const double *A, int64_t P, int64_t H, int64_t W,
                  const double K[SC5O_TAPS * SC5O_TAPS], double *B)
{
    if (P < 1 || H < SC5O_TAPS || W < SC5O_TAPS) return -1;
    const int64_t Hv = H - 4, Wv = W - 4;
    for (int64_t p = 0; p < P; ++p) {
        const double *Ap = A + p * H * W;
        double *Bp = B + p * Hv * Wv;
        for (int64_t y = 0; y < Hv; ++y) {
            for (int64_t x = 0; x < Wv; ++x) {
                double s = 0.0;
                for (int i = 0; i < SC5O_TAPS; ++i)
                    for (int j = 0; j < SC5O_TAPS; ++j)
                        s += Ap[(y + i) * W + (x + j)] * K[i * SC5O_TAPS + j];
                Bp[y * Wv + x] = s;
            }
        }
    }
    return 0;
}

/* Eq. 1 with K = k k^T: the single-pass form for a separable kernel. */
int sc5o_direct(const double *A, int64_t P, int64_t H, int64_t W,
                const double k[SC5O_TAPS], double *B)
{
    double K[SC5O_TAPS * SC5O_TAPS];
    sc5o_outer(k, K);
    return sc5o_direct_K(A, P, H, W, K, B);
}

/*
 * Horizontal 1D pass of the two-pass form (Sec. 5.1; Listing 1, first loop
 * nest): T[p][y][x] = sum_t A[p][y][x+t] * k[t] for every row y in [0, H) and
 * every column x in [0, W-4) (input column x+2 is the centre).
 */
int sc5o_hpass(const double *A, int64_t P, int64_t H, int64_t W,
               const double k[SC5O_TAPS], double *T)
{
    if (P < 1 || H < 1 || W < SC5O_TAPS) return -1;
    const int64_t Wt = W - 4;
    for (int64_t p = 0; p < P; ++p)
        for (int64_t y = 0; y < H; ++y)
            for (int64_t x = 0; x < Wt; ++x) {
                double s = 0.0;
                for (int t = 0; t < SC5O_TAPS; ++t)
                    s += A[(p * H + y) * W + x + t] * k[t];
                T[(p * H + y) * Wt + x] = s;
            }
    return 0;
}

/*
 * Vertical 1D pass of the two-pass form (Sec. 5.1; Listing 1, second loop
 * nest): B[p][y][x] = sum_t T[p][y+t][x] * k[t] for y in [0, H-4) and x in
 * [0, Wt), where T is [P][H][Wt] (row y+2 of T is the centre).
 */
int sc5o_vpass(const double *T, int64_t P, int64_t H, int64_t Wt,
               const double k[SC5O_TAPS], double *B)
{
    if (P < 1 || H < SC5O_TAPS || Wt < 1) return -1;
    const int64_t Hv = H - 4;
    for (int64_t p = 0; p < P; ++p)
        for (int64_t y = 0; y < Hv; ++y)
            for (int64_t x = 0; x < Wt; ++x) {
                double s = 0.0;
                for (int t = 0; t < SC5O_TAPS; ++t)
                    s += T[(p * H + y + t) * Wt + x] * k[t];
                B[(p * Hv + y) * Wt + x] = s;
            }
    return 0;
}

/*
 * Eq. 1 with K = k k^T at chosen output pixels only, reading a strided
 * single-precision planar image [P][H][pitch] (each value widened exactly to
 * double).  pts holds n triples (p, y, x) of VALID output coordinates.  For
 * spot checks of images too large to convolve whole on the host.
 */
int sc5o_points_f32(const float *A, int64_t P, int64_t H, int64_t W, int64_t pitch,
                    const double k[SC5O_TAPS], const int64_t *pts, int64_t n,
                    double *out)
{
    if (P < 1 || H < SC5O_TAPS || W < SC5O_TAPS || pitch < W) return -1;
    double K[SC5O_TAPS * SC5O_TAPS];
    sc5o_outer(k, K);
    for (int64_t q = 0; q < n; ++q) {
        const int64_t p = pts[3 * q], y = pts[3 * q + 1], x = pts[3 * q + 2];
        if (p < 0 || p >= P || y < 0 || y >= H - 4 || x < 0 || x >= W - 4) return -1;
        double s = 0.0;
        for (int i = 0; i < SC5O_TAPS; ++i)
            for (int j = 0; j < SC5O_TAPS; ++j)
                s += (double)A[(p * H + y + i) * pitch + x + j] * K[i * SC5O_TAPS + j];
        out[q] = s;
    }
    return 0;
}

/*
 * Eq. 1 for a kernel of any odd width n (the width-5 routines above are the
 * n = 5 case): B[p][y][x] = sum_{i<n} sum_{j<n} A[p][y+i][x+j] * K[i*n+j] on
 * the VALID region, plane p of B being (H-n+1) x (W-n+1); output (y, x) is
 * centred on input (y+r, x+r) with r = (n-1)/2, so K[i][j] sits at offset
 * (i-r, j-r).  A separable kernel passes K[i][j] = k[i] * k[j].
 */
int sc5o_direct_Kn(const double *A, int64_t P, int64_t H, int64_t W, int64_t n,
                   const double *K, double *B)
{
    if (n < 1 || n % 2 == 0 || P < 1 || H < n || W < n) return -1;
    const int64_t Hv = H - n + 1, Wv = W - n + 1;
    for (int64_t p = 0; p < P; ++p) {
        const double *Ap = A + p * H * W;
        double *Bp = B + p * Hv * Wv;
        for (int64_t y = 0; y < Hv; ++y)
            for (int64_t x = 0; x < Wv; ++x) {
                double s = 0.0;
                for (int64_t i = 0; i < n; ++i)
                    for (int64_t j = 0; j < n; ++j)
                        s += Ap[(y + i) * W + (x + j)] * K[i * n + j];
                Bp[y * Wv + x] = s;
            }
    }
    return 0;
}

/*
 * One REDUCE step of an image pyramid: Eq. 1 with K = k k^T kept at every
 * second output row and column.  The paper names "convolution and scaling"
 * as the two steps that take most of its stereo pipeline's time (Sec. 1) but
 * does not define the scaling; the reading taken here is the blur-then-
 * subsample step of a Gaussian pyramid on the VALID region:
 *
 *   B[p][y][x] = sum_i sum_j A[p][2y+i][2x+j] * k[i] * k[j]
 *
 * for y < Ho = ceil((H-4)/2), x < Wo = ceil((W-4)/2): output (y, x) is the
 * VALID output (2y, 2x), centred on input (2y+2, 2x+2).  A is dense
 * [P][H][W], B dense [P][Ho][Wo].
 */
int sc5o_reduce(const double *A, int64_t P, int64_t H, int64_t W,
                const double k[SC5O_TAPS], double *B)
{
    if (P < 1 || H < SC5O_TAPS || W < SC5O_TAPS) return -1;
    const int64_t Ho = (H - 4 + 1) / 2, Wo = (W - 4 + 1) / 2;
    double K[SC5O_TAPS * SC5O_TAPS];
    sc5o_outer(k, K);
    for (int64_t p = 0; p < P; ++p) {
        const double *Ap = A + p * H * W;
        double *Bp = B + p * Ho * Wo;
        for (int64_t y = 0; y < Ho; ++y)
            for (int64_t x = 0; x < Wo; ++x) {
                double s = 0.0;
                for (int i = 0; i < SC5O_TAPS; ++i)
                    for (int j = 0; j < SC5O_TAPS; ++j)
                        s += Ap[(2 * y + i) * W + (2 * x + j)] * K[i * SC5O_TAPS + j];
                Bp[y * Wo + x] = s;
            }
    }
    return 0;
}

/* ---- storage-format decoders (exact, from the published bit layouts) ---- */

/* bfloat16: the upper 16 bits of an IEEE binary32 (1 sign, 8 exponent, 7 fraction). */
static double bf16_value(uint16_t c)
{
    uint32_t u = (uint32_t)c << 16;
    float f;
    memcpy(&f, &u, sizeof f);
    return (double)f;
}

/* IEEE 754 binary16: 1 sign, 5 exponent (bias 15), 10 fraction; subnormals,
 * infinities and NaNs as in the standard. */
static double f16_value(uint16_t c)
{
    const int s = (c >> 15) & 1, e = (c >> 10) & 0x1f, m = c & 0x3ff;
    double v;
    if (e == 0)
        v = ldexp((double)m, -24);                      /* m * 2^-10 * 2^-14 */
    else if (e == 31)
        v = (m == 0) ? INFINITY : NAN;
    else
        v = ldexp(1.0 + (double)m / 1024.0, e - 15);
    return s ? -v : v;
}

/* OCP 8-bit floating point E4M3 (the "fn" variant): 1 sign, 4 exponent
 * (bias 7), 3 fraction; no infinities; S.1111.111 is NaN; largest finite
 * magnitude 448; subnormals m * 2^-9. */
static double e4m3_value(uint8_t c)
{
    const int s = (c >> 7) & 1, e = (c >> 3) & 0xf, m = c & 0x7;
    double v;
    if (e == 15 && m == 7)
        v = NAN;
    else if (e == 0)
        v = ldexp((double)m, -9);                       /* m * 2^-3 * 2^-6 */
    else
        v = ldexp(1.0 + (double)m / 8.0, e - 7);
    return s ? -v : v;
}

/*
 * Decode n stored values into doubles.  dtype: 0 = binary32, 1 = bfloat16,
 * 2 = binary16, 3 = FP8 E4M3.  A stored code c represents the real value
 * value(c) / scale (scale > 0; 1 for the 16- and 32-bit formats in practice).
 */
int sc5o_decode(int dtype, const void *codes, int64_t n, double scale, double *out)
{
    if (!(scale > 0.0)) return -1;
    for (int64_t i = 0; i < n; ++i) {
        double v;
        switch (dtype) {
        case 0: v = (double)((const float *)codes)[i]; break;
        case 1: v = bf16_value(((const uint16_t *)codes)[i]); break;
        case 2: v = f16_value(((const uint16_t *)codes)[i]); break;
        case 3: v = e4m3_value(((const uint8_t *)codes)[i]); break;
        default: return -1;
        }
        out[i] = v / scale;
    }
    return 0;
}
