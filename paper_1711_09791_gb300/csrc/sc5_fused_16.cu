// sc5_fused_16.cu -- fused-kernel instantiations for bfloat16 and binary16
// storage (output in the same format or in FP32).
#include "sc5_fused_impl.cuh"

namespace sc5 {

#define SC5_SHAPES_16(TI, TO)                                   \
    {                                                           \
        make_entry<TI, TO, 64, 128, 4, 6>(),                    \
        make_entry<TI, TO, 128, 128, 8, 4>(),                   \
        make_entry<TI, TO, 64, 128, 4, 4>(),                    \
        make_entry<TI, TO, 32, 128, 2, 8>(),                    \
        make_entry<TI, TO, 120, 128, 4, 4>(),                   \
        make_entry<TI, TO, 240, 128, 8, 3>(),                   \
        make_entry<TI, TO, 128, 128, 16, 3>(),                  \
        make_entry<TI, TO, 128, 128, 16, 2>(),                  \
    }

int fused_entries_16(int in_dtype, int out_dtype, const FusedEntry **out)
{
    static const FusedEntry bf_bf[] = SC5_SHAPES_16(bf16_t, bf16_t);
    static const FusedEntry bf_f32[] = SC5_SHAPES_16(bf16_t, float);
    static const FusedEntry h_h[] = SC5_SHAPES_16(f16_t, f16_t);
    static const FusedEntry h_f32[] = SC5_SHAPES_16(f16_t, float);
    if (in_dtype == SC5_BF16 && out_dtype == SC5_BF16) { *out = bf_bf; return static_cast<int>(sizeof bf_bf / sizeof bf_bf[0]); }
    if (in_dtype == SC5_BF16 && out_dtype == SC5_F32) { *out = bf_f32; return static_cast<int>(sizeof bf_f32 / sizeof bf_f32[0]); }
    if (in_dtype == SC5_F16 && out_dtype == SC5_F16) { *out = h_h; return static_cast<int>(sizeof h_h / sizeof h_h[0]); }
    if (in_dtype == SC5_F16 && out_dtype == SC5_F32) { *out = h_f32; return static_cast<int>(sizeof h_f32 / sizeof h_f32[0]); }
    return 0;
}

#define SC5_DIRECT_16(TI, TO)                                   \
    {                                                           \
        make_entry<TI, TO, 64, 128, 4, 4, true>(),              \
        make_entry<TI, TO, 128, 128, 8, 3, true>(),             \
    }

int fused_direct_entries_16(int in_dtype, int out_dtype, const FusedEntry **out)
{
    static const FusedEntry bf_bf[] = SC5_DIRECT_16(bf16_t, bf16_t);
    static const FusedEntry bf_f32[] = SC5_DIRECT_16(bf16_t, float);
    static const FusedEntry h_h[] = SC5_DIRECT_16(f16_t, f16_t);
    static const FusedEntry h_f32[] = SC5_DIRECT_16(f16_t, float);
    if (in_dtype == SC5_BF16 && out_dtype == SC5_BF16) { *out = bf_bf; return 2; }
    if (in_dtype == SC5_BF16 && out_dtype == SC5_F32) { *out = bf_f32; return 2; }
    if (in_dtype == SC5_F16 && out_dtype == SC5_F16) { *out = h_h; return 2; }
    if (in_dtype == SC5_F16 && out_dtype == SC5_F32) { *out = h_f32; return 2; }
    return 0;
}

// Other odd widths (3, 7, 9) of the separable kernel: one shape each.
#define SC5_WIDTHS_16(TI, TO, N) {make_entry<TI, TO, 128, 128, 16, 2, false, N>()}

int fused_width_entries_16(int in_dtype, int out_dtype, int taps, const FusedEntry **out)
{
    static const FusedEntry bb3[] = SC5_WIDTHS_16(bf16_t, bf16_t, 3), bb7[] = SC5_WIDTHS_16(bf16_t, bf16_t, 7),
                            bb9[] = SC5_WIDTHS_16(bf16_t, bf16_t, 9);
    static const FusedEntry bf3[] = SC5_WIDTHS_16(bf16_t, float, 3), bf7[] = SC5_WIDTHS_16(bf16_t, float, 7),
                            bf9[] = SC5_WIDTHS_16(bf16_t, float, 9);
    static const FusedEntry hh3[] = SC5_WIDTHS_16(f16_t, f16_t, 3), hh7[] = SC5_WIDTHS_16(f16_t, f16_t, 7),
                            hh9[] = SC5_WIDTHS_16(f16_t, f16_t, 9);
    static const FusedEntry hf3[] = SC5_WIDTHS_16(f16_t, float, 3), hf7[] = SC5_WIDTHS_16(f16_t, float, 7),
                            hf9[] = SC5_WIDTHS_16(f16_t, float, 9);
    const FusedEntry *t3 = nullptr, *t7 = nullptr, *t9 = nullptr;
    if (in_dtype == SC5_BF16 && out_dtype == SC5_BF16) { t3 = bb3; t7 = bb7; t9 = bb9; }
    if (in_dtype == SC5_BF16 && out_dtype == SC5_F32) { t3 = bf3; t7 = bf7; t9 = bf9; }
    if (in_dtype == SC5_F16 && out_dtype == SC5_F16) { t3 = hh3; t7 = hh7; t9 = hh9; }
    if (in_dtype == SC5_F16 && out_dtype == SC5_F32) { t3 = hf3; t7 = hf7; t9 = hf9; }
    if (!t3) return 0;
    switch (taps) {
    case 3: *out = t3; return 1;
    case 7: *out = t7; return 1;
    case 9: *out = t9; return 1;
    default: return 0;
    }
}

}  // namespace sc5
