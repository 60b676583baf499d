// sc5_fused_widths.cu -- instantiations of the fused separable kernel for
// the odd widths other than 5 (3, 7, 9), FP32 storage.
#include "sc5_fused_entry.cuh"

namespace sc5 {

// Other odd widths (3, 7, 9) of the separable kernel, the first shape of each
// list being the default.
int fused_width_entries_f32(int out_dtype, int taps, const FusedEntry **out)
{
    // width 3 runs one CTA per SM when untuned (3x8192x8192: 0.254 ms against
    // 0.276 ms at 2 or more)
    static const FusedEntry w3[] = {make_entry<float, float, 64, 128, 4, 3, false, 3>(1)};
    static const FusedEntry w7[] = {make_entry<float, float, 128, 128, 8, 2, false, 7>()};
    // width 9: 3 stages (3x8192x8192: 0.257 ms against 0.262 ms with 2); for
    // widths 3 and 7 a stage more measured slower (0.271 / 0.291 ms)
    static const FusedEntry w9[] = {make_entry<float, float, 128, 128, 8, 3, false, 9>(),
                                    make_entry<float, float, 128, 128, 8, 2, false, 9>()};
    if (out_dtype != SC5_F32) return 0;
    switch (taps) {
    case 3: *out = w3; return 1;
    case 7: *out = w7; return 1;
    case 9: *out = w9; return 2;
    default: return 0;
    }
}

}  // namespace sc5
