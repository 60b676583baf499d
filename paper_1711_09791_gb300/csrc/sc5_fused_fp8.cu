// sc5_fused_fp8.cu -- fused-kernel instantiations for FP8 E4M3 storage
// (output in E4M3 or in FP32).
#include "sc5_fused_entry.cuh"

namespace sc5 {

#define SC5_SHAPES_8(TI, TO)                                    \
    {                                                           \
        make_entry<TI, TO, 128, 128, 16, 3>(), /* default */    \
        make_entry<TI, TO, 128, 128, 16, 5>(),                  \
        make_entry<TI, TO, 128, 128, 8, 6>(),                   \
        make_entry<TI, TO, 64, 128, 4, 8>(),                    \
        make_entry<TI, TO, 128, 128, 8, 4>(),                   \
        make_entry<TI, TO, 64, 128, 4, 12>(),                   \
        make_entry<TI, TO, 32, 128, 2, 12>(),                   \
        make_entry<TI, TO, 240, 128, 8, 4>(),                   \
        make_entry<TI, TO, 120, 128, 4, 6>(),                   \
        /* 256-wide tiles: 8 output columns per lane */         \
        make_entry<TI, TO, 128, 256, 16, 2>(),                  \
        make_entry<TI, TO, 64, 256, 16, 3>(),                   \
        make_entry<TI, TO, 64, 256, 8, 4>(),                    \
        make_entry<TI, TO, 96, 256, 16, 3>(),                   \
        make_entry<TI, TO, 32, 256, 8, 6>(),                    \
        make_entry<TI, TO, 48, 256, 16, 4>(),                   \
    }

int fused_entries_fp8(int out_dtype, const FusedEntry **out)
{
    static const FusedEntry e_e[] = SC5_SHAPES_8(fp8e4m3_t, fp8e4m3_t);
    static const FusedEntry e_f32[] = SC5_SHAPES_8(fp8e4m3_t, float);
    if (out_dtype == SC5_FP8E4M3) { *out = e_e; return static_cast<int>(sizeof e_e / sizeof e_e[0]); }
    if (out_dtype == SC5_F32) { *out = e_f32; return static_cast<int>(sizeof e_f32 / sizeof e_f32[0]); }
    return 0;
}

}  // namespace sc5
