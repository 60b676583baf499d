// sc5_fused_f16.cu -- fused-kernel instantiations for binary16 storage (output
// in binary16 or FP32).
#include "sc5_fused_16_shapes.cuh"

namespace sc5 {

int fused_entries_f16(int out_dtype, const FusedEntry **out)
{
    static const FusedEntry h_h[] = SC5_SHAPES_16(f16_t, f16_t);
    static const FusedEntry h_f32[] = SC5_SHAPES_16_F32(f16_t);
    if (out_dtype == SC5_F16) { *out = h_h; return static_cast<int>(sizeof h_h / sizeof h_h[0]); }
    if (out_dtype == SC5_F32) { *out = h_f32; return static_cast<int>(sizeof h_f32 / sizeof h_f32[0]); }
    return 0;
}

}  // namespace sc5
