// sc5_fused_16.cu -- fused-kernel instantiations for bfloat16 storage (output
// in bfloat16 or FP32); binary16 is in sc5_fused_f16.cu, so that the two
// compile in parallel.
#include "sc5_fused_16_shapes.cuh"

namespace sc5 {

int fused_entries_f16(int out_dtype, const FusedEntry **out);

int fused_entries_16(int in_dtype, int out_dtype, const FusedEntry **out)
{
    if (in_dtype == SC5_F16) return fused_entries_f16(out_dtype, out);
    static const FusedEntry bf_bf[] = SC5_SHAPES_16(bf16_t, bf16_t);
    static const FusedEntry bf_f32[] = SC5_SHAPES_16_F32(bf16_t);
    if (in_dtype == SC5_BF16 && out_dtype == SC5_BF16) { *out = bf_bf; return static_cast<int>(sizeof bf_bf / sizeof bf_bf[0]); }
    if (in_dtype == SC5_BF16 && out_dtype == SC5_F32) { *out = bf_f32; return static_cast<int>(sizeof bf_f32 / sizeof bf_f32[0]); }
    return 0;
}

}  // namespace sc5
