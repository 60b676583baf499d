// sc5_fused_fp8.cu -- fused-kernel instantiations for FP8 E4M3 storage
// (output in E4M3 or in FP32).
#include "sc5_fused_impl.cuh"

namespace sc5 {

#define SC5_SHAPES_8(TI, TO)                                    \
    {                                                           \
        make_entry<TI, TO, 128, 128, 8, 6>(),                   \
        make_entry<TI, TO, 64, 128, 4, 8>(),                    \
        make_entry<TI, TO, 128, 128, 8, 4>(),                   \
        make_entry<TI, TO, 64, 128, 4, 12>(),                   \
        make_entry<TI, TO, 32, 128, 2, 12>(),                   \
        make_entry<TI, TO, 240, 128, 8, 4>(),                   \
        make_entry<TI, TO, 120, 128, 4, 6>(),                   \
        make_entry<TI, TO, 128, 128, 16, 5>(),                  \
        make_entry<TI, TO, 128, 128, 16, 3>(),                  \
    }

int fused_entries_fp8(int out_dtype, const FusedEntry **out)
{
    static const FusedEntry e_e[] = SC5_SHAPES_8(fp8e4m3_t, fp8e4m3_t);
    static const FusedEntry e_f32[] = SC5_SHAPES_8(fp8e4m3_t, float);
    if (out_dtype == SC5_FP8E4M3) { *out = e_e; return static_cast<int>(sizeof e_e / sizeof e_e[0]); }
    if (out_dtype == SC5_F32) { *out = e_f32; return static_cast<int>(sizeof e_f32 / sizeof e_f32[0]); }
    return 0;
}

int fused_direct_entries_fp8(int out_dtype, const FusedEntry **out)
{
    static const FusedEntry e_e[] = {
        make_entry<fp8e4m3_t, fp8e4m3_t, 64, 128, 4, 4, true>(),
        make_entry<fp8e4m3_t, fp8e4m3_t, 128, 128, 8, 3, true>(),
    };
    static const FusedEntry e_f32[] = {
        make_entry<fp8e4m3_t, float, 64, 128, 4, 4, true>(),
        make_entry<fp8e4m3_t, float, 128, 128, 8, 3, true>(),
    };
    if (out_dtype == SC5_FP8E4M3) { *out = e_e; return 2; }
    if (out_dtype == SC5_F32) { *out = e_f32; return 2; }
    return 0;
}

// Other odd widths (3, 7, 9) of the separable kernel: one shape each.
int fused_width_entries_fp8(int out_dtype, int taps, const FusedEntry **out)
{
    static const FusedEntry ee3[] = {make_entry<fp8e4m3_t, fp8e4m3_t, 128, 128, 16, 3, false, 3>()};
    static const FusedEntry ee7[] = {make_entry<fp8e4m3_t, fp8e4m3_t, 128, 128, 16, 3, false, 7>()};
    static const FusedEntry ee9[] = {make_entry<fp8e4m3_t, fp8e4m3_t, 128, 128, 16, 3, false, 9>()};
    static const FusedEntry ef3[] = {make_entry<fp8e4m3_t, float, 128, 128, 16, 3, false, 3>()};
    static const FusedEntry ef7[] = {make_entry<fp8e4m3_t, float, 128, 128, 16, 3, false, 7>()};
    static const FusedEntry ef9[] = {make_entry<fp8e4m3_t, float, 128, 128, 16, 3, false, 9>()};
    const bool e = out_dtype == SC5_FP8E4M3;
    if (!e && out_dtype != SC5_F32) return 0;
    switch (taps) {
    case 3: *out = e ? ee3 : ef3; return 1;
    case 7: *out = e ? ee7 : ef7; return 1;
    case 9: *out = e ? ee9 : ef9; return 1;
    default: return 0;
    }
}

}  // namespace sc5
