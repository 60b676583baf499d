// sc5_fused_16_shapes.cuh -- the compiled fused-kernel shapes of the 16-bit
// storage formats (bfloat16 and binary16, output in the same format or in
// FP32), shared by the two translation units that instantiate them.
#pragma once

#include "sc5_fused_entry.cuh"

namespace sc5 {

// 256-wide tiles: 8 output columns per lane, two TMA boxes per tile.
#define SC5_SHAPES_16_WIDE(TI, TO)                              \
        make_entry<TI, TO, 128, 256, 16, 2>(),                  \
        make_entry<TI, TO, 64, 256, 16, 2>(),                   \
        make_entry<TI, TO, 64, 256, 8, 3>(),                    \
        make_entry<TI, TO, 96, 256, 16, 2>(),                   \
        make_entry<TI, TO, 32, 256, 8, 4>(),                    \
        make_entry<TI, TO, 48, 256, 16, 3>(),

// The default shape runs 2 CTAs per SM when untuned: on 3x8192x8192 BF16 it
// measured 0.131 ms there against 0.149-0.150 ms at 1 or 3.
#define SC5_SHAPES_16(TI, TO)                                   \
    {                                                           \
        make_entry<TI, TO, 128, 128, 16, 2>(2), /* default */   \
        make_entry<TI, TO, 128, 128, 16, 3>(),                  \
        make_entry<TI, TO, 128, 128, 8, 4>(),                   \
        make_entry<TI, TO, 64, 128, 4, 6>(),                    \
        make_entry<TI, TO, 64, 128, 4, 4>(),                    \
        make_entry<TI, TO, 32, 128, 2, 8>(),                    \
        make_entry<TI, TO, 120, 128, 4, 4>(),                   \
        make_entry<TI, TO, 240, 128, 8, 3>(),                   \
        SC5_SHAPES_16_WIDE(TI, TO)                              \
    }

// The same shapes with FP32 output, default first: 64x128 tiles, 4 rows per
// lane, 6 stages (3x8192x8192 BF16 -> FP32: 0.190 ms against 0.209 ms for
// the 128x128/16 shape, at any CTA count).
#define SC5_SHAPES_16_F32(TI)                                   \
    {                                                           \
        make_entry<TI, float, 64, 128, 4, 6>(), /* default */   \
        make_entry<TI, float, 128, 128, 16, 2>(),               \
        make_entry<TI, float, 128, 128, 16, 3>(),               \
        make_entry<TI, float, 128, 128, 8, 4>(),                \
        make_entry<TI, float, 64, 128, 4, 4>(),                 \
        make_entry<TI, float, 32, 128, 2, 8>(),                 \
        make_entry<TI, float, 120, 128, 4, 4>(),                \
        make_entry<TI, float, 240, 128, 8, 3>(),                \
        SC5_SHAPES_16_WIDE(TI, float)                           \
    }

}  // namespace sc5
