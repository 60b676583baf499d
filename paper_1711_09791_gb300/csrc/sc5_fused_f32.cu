// sc5_fused_f32.cu -- fused-kernel instantiations for FP32 storage.
#include "sc5_fused_entry.cuh"

namespace sc5 {

int fused_entries_f32(int out_dtype, const FusedEntry **out)
{
    // (tile_h, tile_w, rows per thread, stages)
    static const FusedEntry f32_f32[] = {
        make_entry<float, float, 64, 128, 4, 3>(),   // default: 16 consumer warps, 108 KB
        make_entry<float, float, 64, 128, 4, 4>(),
        make_entry<float, float, 64, 128, 4, 2>(),
        make_entry<float, float, 128, 128, 8, 3>(),
        make_entry<float, float, 32, 128, 4, 2>(),
        make_entry<float, float, 32, 128, 2, 4>(),
        make_entry<float, float, 32, 128, 4, 5>(),
        make_entry<float, float, 120, 128, 4, 3>(),  // 30 consumer warps
    };
    if (out_dtype == SC5_F32) { *out = f32_f32; return static_cast<int>(sizeof f32_f32 / sizeof f32_f32[0]); }
    return 0;
}

}  // namespace sc5
