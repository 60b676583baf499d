// sc5_fused_impl.cuh -- the fused single-pass kernel (template), included by
// the per-format translation units.
//
// What it computes: the single-pass result of Sec. 5.1 / Sec. 7 ("single-pass
// without copy-back"): B[p][y][x] = sum_a sum_b A[p][y+a][x+b] k[a] k[b] on the
// VALID region, evaluated as the separable 5+5 form (Sec. 5.1) with the
// horizontal-pass values kept in registers, so every input pixel crosses HBM
// once in and every output pixel once out.
//
// Structure of one CTA (persistent; tiles t = blockIdx.x + i * gridDim.x):
//   * warp NC (the producer) -- one lane issues a TMA 3-D box load of the
//     (TH+4) x BW input window of each tile into stage i % S of a ring of S
//     shared-memory buffers, signalling `full[s]` with transaction bytes; it
//     refills a stage only after every consumer warp has released it on
//     `empty[s]`.
//   * warps 0..NC-1 (consumers) -- warp w owns output rows [w*R, w*R+R) of the
//     tile, lane l owns output columns [4l, 4l+4).  For each of its R+4 input
//     rows a lane reads 8 stored values from shared memory, widens them to
//     FP32, forms the 4 horizontal-pass values, and adds each into the (at
//     most 5) pending output rows it contributes to; an output row is stored
//     as soon as its fifth tap has arrived.  Stores are 4-wide and streaming.
// All waits are bounded by global time; on time-out the kernel records an
// error in the status word and returns (no trap).
#pragma once

#include "sc5_device.cuh"

namespace sc5 {

constexpr uint64_t kWaitLimitNs = 1000ull * 1000ull * 1000ull;  // 1 s per wait
constexpr uint64_t kDrainLimitNs = 100ull * 1000ull * 1000ull;  // 0.1 s after an error

template <class TIn>
__host__ __device__ constexpr int fused_box_w(int tw)
{
    // TW + 4 columns rounded up so that a box row is a multiple of 16 bytes
    return ((tw + kHalo) * Fmt<TIn>::bytes + 15) / 16 * 16 / Fmt<TIn>::bytes;
}

template <class TIn, int TH, int TW>
__host__ __device__ constexpr int fused_stage_bytes()
{
    return (fused_box_w<TIn>(TW) * (TH + kHalo) * Fmt<TIn>::bytes + 127) / 128 * 128;
}

// One lane's strip: R output rows x 4 output columns.
//   s:   shared memory at (first input row of the strip, first input column)
//   out: global memory at (first output row, first output column)
template <class TIn, class TOut, int R, int BW>
__device__ __forceinline__ void conv_strip(const TIn *__restrict__ s, const float (&k)[kTaps],
                                           float oscale, TOut *__restrict__ out, int64_t out_pitch,
                                           int rows_valid, int cols_valid, bool vec)
{
    float acc[R][kColsPerThread];
#pragma unroll
    for (int r = 0; r < R + kHalo; ++r) {
        float a[8];
        Fmt<TIn>::load8(s + r * BW, a);
        float h[kColsPerThread];
#pragma unroll
        for (int c = 0; c < kColsPerThread; ++c) h[c] = hdot(k, a + c);
        // input row r carries tap t = r - o of output row o
#pragma unroll
        for (int t = 0; t < kTaps; ++t) {
            const int o = r - t;
            if (o >= 0 && o < R) {
#pragma unroll
                for (int c = 0; c < kColsPerThread; ++c)
                    acc[o][c] = (t == 0) ? __fmul_rn(k[0], h[c]) : __fmaf_rn(k[t], h[c], acc[o][c]);
            }
        }
        const int o = r - kHalo;  // output row o has all five taps now
        if (o >= 0 && o < rows_valid) {
            float v[kColsPerThread];
#pragma unroll
            for (int c = 0; c < kColsPerThread; ++c) v[c] = __fmul_rn(acc[o][c], oscale);
            TOut *dst = out + static_cast<int64_t>(o) * out_pitch;
            if (vec && cols_valid == kColsPerThread) {
                Fmt<TOut>::store4(dst, v);
            } else {
#pragma unroll
                for (int c = 0; c < kColsPerThread; ++c)
                    if (c < cols_valid) Fmt<TOut>::store1(dst + c, v[c]);
            }
        }
    }
}

__device__ __forceinline__ void record_error(int *status, int code)
{
    atomicCAS(status, 0, code);
}

template <class TIn, class TOut, int TH, int TW, int R, int S, bool BATCH>
__global__ void __launch_bounds__(32 * (TH / R + 1), 1)
fused_kernel(const __grid_constant__ ImgDesc single, const ImgDesc *__restrict__ descs,
             const TileRec *__restrict__ tiles, int64_t ntiles, int *status)
{
    static_assert(TW == 32 * kColsPerThread, "one warp spans the tile width");
    static_assert(TH % R == 0, "rows per thread must divide the tile height");
    constexpr int NC = TH / R;                       // consumer warps
    constexpr int BW = fused_box_w<TIn>(TW);
    constexpr int STAGE = fused_stage_bytes<TIn, TH, TW>();
    constexpr uint32_t TX = BW * (TH + kHalo) * Fmt<TIn>::bytes;

    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[S];
    __shared__ __align__(8) uint64_t empty[S];
    __shared__ TileRec info[S];

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NC);
        }
        fence_barrier_init();
        if (!BATCH) prefetch_tmap(&single.tmap);
    }
    __syncthreads();

    if (warp == NC) {
        // ------------------------------------------------------------ producer
        if (lane != 0) return;
        int64_t issued = 0;
        for (int64_t i = 0;; ++i) {
            const int64_t t = blockIdx.x + i * static_cast<int64_t>(gridDim.x);
            if (t >= ntiles) break;
            const int s = static_cast<int>(i % S);
            const uint32_t use = static_cast<uint32_t>(i / S);
            if (use > 0 && !mbar_wait_bounded(&empty[s], (use - 1) & 1, kWaitLimitNs)) {
                record_error(status, kDevErrTmaTimeout);
                break;
            }
            TileRec rec;
            const CUtensorMap *m;
            if (BATCH) {
                rec = tiles[t];
                m = &descs[rec.img].tmap;
            } else {
                const int64_t per_plane = static_cast<int64_t>(single.tiles_x) * single.tiles_y;
                rec.img = 0;
                rec.plane = static_cast<int32_t>(t / per_plane);
                const int64_t r = t - rec.plane * per_plane;
                rec.ty = static_cast<int32_t>(r / single.tiles_x);
                rec.tx = static_cast<int32_t>(r - static_cast<int64_t>(rec.ty) * single.tiles_x);
                m = &single.tmap;
            }
            info[s] = rec;
            mbar_arrive_expect_tx(&full[s], TX);
            tma_load_3d(smem + s * STAGE, m, &full[s], rec.tx * TW, rec.ty * TH, rec.plane);
            ++issued;
        }
        // Leave only once the loads this lane issued have landed (bounded).
        for (int64_t j = (issued > S ? issued - S : 0); j < issued; ++j)
            mbar_wait_bounded(&full[j % S], static_cast<uint32_t>(j / S) & 1, kDrainLimitNs);
        return;
    }

    // ---------------------------------------------------------------- consumers
    float k[kTaps];
    float oscale = 1.f;
    if (!BATCH) {
#pragma unroll
        for (int t = 0; t < kTaps; ++t) k[t] = single.k[t];
        oscale = single.oscale;
    }
    for (int64_t i = 0;; ++i) {
        const int64_t t = blockIdx.x + i * static_cast<int64_t>(gridDim.x);
        if (t >= ntiles) break;
        const int s = static_cast<int>(i % S);
        const uint32_t use = static_cast<uint32_t>(i / S);
        if (!mbar_wait_bounded(&full[s], use & 1, kWaitLimitNs)) {
            if (lane == 0) record_error(status, kDevErrTmaTimeout);
            mbar_wait_bounded(&full[s], use & 1, kDrainLimitNs);
            return;
        }
        const TileRec rec = info[s];
        const ImgDesc *d = BATCH ? &descs[rec.img] : &single;
        if (BATCH) {
#pragma unroll
            for (int q = 0; q < kTaps; ++q) k[q] = d->k[q];
            oscale = d->oscale;
        }
        const int ry0 = rec.ty * TH + warp * R;
        const int cx = rec.tx * TW + lane * kColsPerThread;
        const int rows_valid = min(R, d->Hv - ry0);
        const int cols_valid = min(kColsPerThread, d->Wv - cx);
        if (rows_valid > 0 && cols_valid > 0) {
            const TIn *src = reinterpret_cast<const TIn *>(smem + s * STAGE) +
                             (warp * R) * BW + lane * kColsPerThread;
            TOut *dst = reinterpret_cast<TOut *>(d->out) + rec.plane * d->out_plane +
                        static_cast<int64_t>(ry0) * d->out_pitch + cx;
            conv_strip<TIn, TOut, R, BW>(src, k, oscale, dst, d->out_pitch, rows_valid,
                                         cols_valid, d->vec != 0);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
    }
}

// ------------------------------------------------------------------ registry

struct FusedEntry {
    FusedShape shape;
    const void *single_fn;
    const void *batch_fn;
    int smem;
    int threads;
};

template <class TIn, class TOut, int TH, int TW, int R, int S>
FusedEntry make_entry()
{
    FusedEntry e;
    e.shape = FusedShape{TH, TW, R, S};
    e.single_fn = reinterpret_cast<const void *>(&fused_kernel<TIn, TOut, TH, TW, R, S, false>);
    e.batch_fn = reinterpret_cast<const void *>(&fused_kernel<TIn, TOut, TH, TW, R, S, true>);
    e.smem = S * fused_stage_bytes<TIn, TH, TW>();
    e.threads = 32 * (TH / R + 1);
    return e;
}

}  // namespace sc5
