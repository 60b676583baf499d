// sc5_tune.h -- autotuner table lookups used by the planner.
#pragma once

#include <stdint.h>

namespace sc5 {

constexpr int kNumClasses = 7;

// Size class of a plane of `px` pixels: 0 for < 2^14, then one class per
// factor of 4 up to class 6 for >= 2^24.
int size_class(double px);

// Tuned choice for a dtype pair and plane size; false if the table has none.
bool tune_lookup_internal(int in_dtype, int out_dtype, int H, int W, int *tile_h, int *tile_w,
                          int *stages, int *ctas_per_sm);

}  // namespace sc5
