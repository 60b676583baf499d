// sc5_fused_widths_narrow.cu -- instantiations of the fused separable kernel
// for the odd widths other than 5 (3, 7, 9), bfloat16 / binary16 / FP8 storage.
#include "sc5_fused_entry.cuh"

namespace sc5 {

// Other odd widths (3, 7, 9) of the separable kernel: one shape each.  Width 3
// runs one CTA per SM when untuned (3x8192x8192 BF16: 0.142 ms against 0.154 ms
// at 2 or more).
#define SC5_WIDTHS_16(TI, TO, N) {make_entry<TI, TO, 128, 128, 16, 2, false, N>((N) == 3 ? 1 : 0)}

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
