// sc5_fused_direct_strip.cuh -- one consumer lane's strip of the fused
// kernel in the direct form.  Included by sc5_fused_impl.cuh inside
// namespace sc5, after the helpers it uses (row_pairs, store_row); not a
// standalone header.
#pragma once

// One lane's strip, direct form (the single-pass algorithm of Sec. 5.1 with
// a general 5x5 matrix): every output is one FP32 chain of 25 products in the
// row-major order of Eq. 3, K[0][0]*A[y][x] first, then fused multiply-adds
// through K[4][4]*A[y+4][x+4].  KK holds the 25 entries as pairs (K, K).
template <class TIn, class TOut, int R, int BW, bool FULL = false>
__device__ __forceinline__ void conv_strip_direct(const TIn *__restrict__ s, const uint64_t (&KK)[kTaps * kTaps],
                                                  uint64_t os2, bool scaled, TOut *__restrict__ out,
                                                  int64_t out_pitch, int rows_valid, int cols_valid, bool vec)
{
    // FULL: an interior strip (all R rows and 4 columns inside the image, vector
    // stores aligned); the guards are then compile-time true.
    if constexpr (FULL) {
        rows_valid = R;
        cols_valid = kColsPerThread;
        vec = true;
    }
    uint64_t accL[R], accR[R];
#pragma unroll
    for (int r = 0; r < R + kHalo; ++r) {
        uint64_t PL[kTaps], PR[kTaps];
        row_pairs<TIn>(s + r * BW, PL, PR);
        // input row r is kernel row i = r - o of output row o
#pragma unroll
        for (int i = 0; i < kTaps; ++i) {
            const int o = r - i;
            if (o >= 0 && o < R) {
#pragma unroll
                for (int j = 0; j < kTaps; ++j) {
                    const uint64_t Kij = KK[i * kTaps + j];
                    if (i == 0 && j == 0) {
                        accL[o] = mul2(Kij, PL[0]);
                        accR[o] = mul2(Kij, PR[0]);
                    } else {
                        accL[o] = fma2(Kij, PL[j], accL[o]);
                        accR[o] = fma2(Kij, PR[j], accR[o]);
                    }
                }
            }
        }
        const int o = r - kHalo;
        if (o >= 0 && o < rows_valid)
            store_row<TIn, TOut>(accL[o], accR[o], os2, scaled, out + static_cast<int64_t>(o) * out_pitch,
                                 cols_valid, vec);
    }
}
