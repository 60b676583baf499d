// sc5_fused_entry.cuh -- the host-side record of one compiled fused-kernel
// shape (tile, rows per thread, stages, its single-image and batch kernels,
// shared memory, threads, default CTAs per SM).  Kept apart from the kernel
// header so that registry changes leave the kernel source untouched.
#pragma once

#include "sc5_fused_impl.cuh"

namespace sc5 {

struct FusedEntry {
    FusedShape shape;
    const void *single_fn;
    const void *batch_fn;
    int smem;
    int threads;
    int ctas_default;  // CTAs per SM for untuned plans; 0: as many as fit
};

template <class TIn, class TOut, int TH, int TW, int R, int S, bool DIRECT = false, int TAPS = kTaps>
FusedEntry make_entry(int ctas_default = 0)
{
    FusedEntry e;
    e.shape = FusedShape{TH, TW, R, S};
    e.single_fn = reinterpret_cast<const void *>(&fused_kernel<TIn, TOut, TH, TW, R, S, false, DIRECT, TAPS>);
    e.batch_fn = reinterpret_cast<const void *>(&fused_kernel<TIn, TOut, TH, TW, R, S, true, DIRECT, TAPS>);
    e.smem = S * fused_stage_bytes<TIn, TH, TW, TAPS>();
    e.threads = 32 * (TH / R + 1);
    e.ctas_default = ctas_default;
    return e;
}

}  // namespace sc5
