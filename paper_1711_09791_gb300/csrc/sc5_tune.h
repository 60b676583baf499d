// sc5_tune.h -- autotuner table lookups used by the planner.
#pragma once

#include <stdint.h>

namespace sc5 {

constexpr int kNumClasses = 7;

// Size class of a plane of `px` pixels: 0 for < 2^14, then one class per
// factor of 4 up to class 6 for >= 2^24.
int size_class(double px);

// Kernel kinds tuned separately: the single-image kernel of a plan and the
// work-list kernel of batches and merged serving launches.  The same shape can
// rank differently in the two (3x8192x8192 FP32, 64x128 tiles with 4 stages:
// 0.287 ms single-image, 0.241 ms as a batch; with 3 stages 0.238 / 0.250 ms).
constexpr int kKindSingle = 0, kKindBatch = 1;

// Tuned choice for a dtype pair, plane size and kernel kind; false if the
// table has none.
bool tune_lookup_internal(int in_dtype, int out_dtype, int H, int W, int kind, int *tile_h, int *tile_w,
                          int *stages, int *ctas_per_sm);

// The environment override, applied once per dtype pair on the pair's first
// plan, batch or merged serving launch in the process:
//   SEPCONV5_TUNE_FILE=path   load a saved table (entries for other GPUs are
//                             ignored) and write the table back there after
//                             tuning;
//   SEPCONV5_TUNE=off         the built-in defaults unless a table is loaded;
//   SEPCONV5_TUNE=quick|full  tune the pair (3 or 10 repetitions per
//                             configuration, a few seconds of GPU time) unless
//                             the table already holds all of its entries.
// Failures leave the defaults in place (and a message in sepconv5_last_error).
void tune_from_environment(int in_dtype, int out_dtype);

}  // namespace sc5
