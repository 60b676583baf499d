// sc5_fused_direct.cu -- instantiations of the direct single-pass kernels
// (general 5x5 matrix, 25 products per output) for every storage format.
#include "sc5_fused_entry.cuh"

namespace sc5 {

// Shapes, the first being the default: 128x128 tiles with 8 rows per lane and
// 3 stages measured fastest for every pair on 3x8192x8192 (FP32 0.248 ms
// against 0.267 ms for 64x128/4/3; BF16 0.211 against 0.252 ms; FP8 0.220
// against 0.262 ms).
int fused_direct_entries_f32(int out_dtype, const FusedEntry **out)
{
    static const FusedEntry f32_f32[] = {
        make_entry<float, float, 128, 128, 8, 3, true>(),
        make_entry<float, float, 64, 128, 4, 3, true>(),
        make_entry<float, float, 32, 128, 2, 4, true>(),
    };
    if (out_dtype == SC5_F32) { *out = f32_f32; return static_cast<int>(sizeof f32_f32 / sizeof f32_f32[0]); }
    return 0;
}

#define SC5_DIRECT_16(TI, TO)                                   \
    {                                                           \
        make_entry<TI, TO, 128, 128, 8, 3, true>(),             \
        make_entry<TI, TO, 64, 128, 4, 4, true>(),              \
    }

int fused_direct_entries_16(int in_dtype, int out_dtype, const FusedEntry **out)
{
    static const FusedEntry bf_bf[] = SC5_DIRECT_16(bf16_t, bf16_t);
    static const FusedEntry bf_f32[] = SC5_DIRECT_16(bf16_t, float);
    static const FusedEntry h_h[] = SC5_DIRECT_16(f16_t, f16_t);
    static const FusedEntry h_f32[] = SC5_DIRECT_16(f16_t, float);
    constexpr int n = static_cast<int>(sizeof bf_bf / sizeof bf_bf[0]);
    if (in_dtype == SC5_BF16 && out_dtype == SC5_BF16) { *out = bf_bf; return n; }
    if (in_dtype == SC5_BF16 && out_dtype == SC5_F32) { *out = bf_f32; return n; }
    if (in_dtype == SC5_F16 && out_dtype == SC5_F16) { *out = h_h; return n; }
    if (in_dtype == SC5_F16 && out_dtype == SC5_F32) { *out = h_f32; return n; }
    return 0;
}

int fused_direct_entries_fp8(int out_dtype, const FusedEntry **out)
{
    static const FusedEntry e_e[] = {
        make_entry<fp8e4m3_t, fp8e4m3_t, 128, 128, 8, 3, true>(),
        make_entry<fp8e4m3_t, fp8e4m3_t, 64, 128, 4, 4, true>(),
    };
    static const FusedEntry e_f32[] = {
        make_entry<fp8e4m3_t, float, 128, 128, 8, 3, true>(),
        make_entry<fp8e4m3_t, float, 64, 128, 4, 4, true>(),
    };
    if (out_dtype == SC5_FP8E4M3) { *out = e_e; return 2; }
    if (out_dtype == SC5_F32) { *out = e_f32; return 2; }
    return 0;
}

}  // namespace sc5
