// sc5_reduce.cu -- one REDUCE step of an image pyramid: the separable width-5
// convolution (Eq. 1 with K = k k^T) on the VALID region, kept at every
// second row and column.  The paper names "convolution and scaling" as the
// steps that take most of its stereo pipeline's time (Sec. 1) and leaves the
// scaling undefined; this is the blur-then-subsample reading:
//
//   B[p][y][x] = sum_i sum_j A[p][2y+i][2x+j] k[i] k[j],
//   y < ceil((H-4)/2), x < ceil((W-4)/2)   (centred on input (2y+2, 2x+2)).
//
// The kernel is the fused kernel's pipeline with a decimating consumer.  A
// tile covers TH input rows x 128 input columns (TH/2 x 64 outputs), so its
// TMA box is exactly the fused kernel's box for a TH x 128 tile.  Warp w owns
// input rows [w*R, w*R+R) of the tile (R/2 output rows), lane l input columns
// [4l, 4l+4) (outputs 2l and 2l+1).  For each of the R+3 input rows it needs,
// a lane forms the row-pass values at input columns 4l and 4l+2 as one packed
// pair, (k0*a0, k0*a2) then fused multiply-adds of (a[t], a[t+2]); the column
// pass adds each into the output rows it belongs to.  Every output is the
// same FP32 sequence as the fused kernel's output at that position (row pass
// t = 0..4, column pass t = 0..4, then the output scale), so the result is
// the fused result at even rows and columns, bit for bit.
// All waits are bounded by global time; on time-out the kernel records an
// error in the status word and returns (no trap).
#include <mutex>
#include <set>
#include <utility>

#include "sc5_fused_impl.cuh"

namespace sc5 {

namespace {

constexpr int kReduceTW = 128;  // input columns per tile (64 outputs)
constexpr int kReduceTaps = kTaps;

// One lane's strip: R input rows (R/2 output rows) x 2 output columns.
//   s:   shared memory at (first input row of the strip, input column 4l)
//   out: global memory at (first output row, output column 2l)
template <class TIn, class TOut, int R, int BW>
__device__ __forceinline__ void reduce_strip(const TIn *__restrict__ s, const uint64_t (&kk)[kReduceTaps],
                                             uint64_t os2, bool scaled, TOut *__restrict__ out, int64_t out_pitch,
                                             int rows_valid, int cols_valid)
{
    constexpr int RO = R / 2;  // output rows of the strip
    uint64_t acc[RO];
#pragma unroll
    for (int r = 0; r < R + kReduceTaps - 2; ++r) {
        float a[8];
        Fmt<TIn>::load4(s + r * BW, a);
        Fmt<TIn>::load4(s + r * BW + 4, a + 4);
        // row pass at input columns 4l and 4l+2: pairs (a[t], a[t+2])
        uint64_t h = mul2(kk[0], pack2(a[0], a[2]));
#pragma unroll
        for (int t = 1; t < kReduceTaps; ++t) h = fma2(kk[t], pack2(a[t], a[t + 2]), h);
        // input row r carries tap t = r - 2o of output row o
#pragma unroll
        for (int o = 0; o < RO; ++o) {
            const int t = r - 2 * o;
            if (t >= 0 && t < kReduceTaps) acc[o] = (t == 0) ? mul2(kk[0], h) : fma2(kk[t], h, acc[o]);
        }
        if (r >= kReduceTaps - 1 && (r - (kReduceTaps - 1)) % 2 == 0) {
            const int o = (r - (kReduceTaps - 1)) / 2;  // output row o has all its taps now
            if (o < RO && o < rows_valid) {
                uint64_t v = acc[o];
                if (scaled) v = mul2(v, os2);
                float v0, v1;
                unpack2(v, v0, v1);
                TOut *dst = out + static_cast<int64_t>(o) * out_pitch;
                if (cols_valid > 0) Fmt<TOut>::store1(dst, v0);
                if (cols_valid > 1) Fmt<TOut>::store1(dst + 1, v1);
            }
        }
    }
}

// TH: input rows per tile (even), R: input rows per consumer warp (even), S: stages.
// d.Hv / d.Wv hold the output extents (Ho, Wo); d.tiles_x / d.tiles_y the tile grid.
template <class TIn, class TOut, int TH, int R, int S>
__global__ void __launch_bounds__(32 * (TH / R + 1), 1)
reduce_kernel(const __grid_constant__ ImgDesc d, int64_t ntiles, int *status)
{
    static_assert(TH % R == 0 && R % 2 == 0, "even rows per warp dividing the tile height");
    constexpr int NC = TH / R;
    constexpr int BW = fused_box_w<TIn, kReduceTaps>(kReduceTW);
    constexpr int STAGE = fused_stage_bytes<TIn, TH, kReduceTW, kReduceTaps>();
    constexpr uint32_t TX = BW * (TH + kReduceTaps - 1) * Fmt<TIn>::bytes;

    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[S];
    __shared__ __align__(8) uint64_t empty[S];

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NC);
        }
        fence_barrier_init();
        prefetch_tmap(&d.tmap);
    }
    __syncthreads();

    const int64_t per_plane = static_cast<int64_t>(d.tiles_x) * d.tiles_y;
    if (warp == NC) {
        // ------------------------------------------------------------ producer
        if (lane != 0) return;
        int64_t issued = 0;
        int s = 0;
        uint32_t phase = 0;
        bool wrapped = false;
        for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
            if (wrapped && !mbar_wait_bounded(&empty[s], phase ^ 1u, kWaitLimitNs)) {
                record_error(status, kDevErrTmaTimeout);
                break;
            }
            const int plane = static_cast<int>(t / per_plane);
            const int64_t r = t - plane * per_plane;
            const int ty = static_cast<int>(r / d.tiles_x);
            const int tx = static_cast<int>(r - static_cast<int64_t>(ty) * d.tiles_x);
            mbar_arrive_expect_tx(&full[s], TX);
            tma_load_3d(smem + s * STAGE, &d.tmap, &full[s], tx * kReduceTW, ty * TH, plane);
            ++issued;
            if (++s == S) {
                s = 0;
                phase ^= 1u;
                wrapped = true;
            }
        }
        for (int64_t j = (issued > S ? issued - S : 0); j < issued; ++j)
            mbar_wait_bounded(&full[j % S], static_cast<uint32_t>(j / S) & 1, kDrainLimitNs);
        return;
    }

    // ---------------------------------------------------------------- consumers
    uint64_t kk[kReduceTaps];
#pragma unroll
    for (int q = 0; q < kReduceTaps; ++q) kk[q] = pack2(d.k[q], d.k[q]);
    const uint64_t os2 = pack2(d.oscale, d.oscale);
    const bool scaled = d.oscale != 1.f;
    int s = 0;
    uint32_t phase = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        if (!mbar_wait_bounded(&full[s], phase, kWaitLimitNs)) {
            if (lane == 0) record_error(status, kDevErrTmaTimeout);
            mbar_wait_bounded(&full[s], phase, kDrainLimitNs);
            return;
        }
        const int plane = static_cast<int>(t / per_plane);
        const int64_t rr = t - plane * per_plane;
        const int ty = static_cast<int>(rr / d.tiles_x);
        const int tx = static_cast<int>(rr - static_cast<int64_t>(ty) * d.tiles_x);
        const int yo0 = ty * (TH / 2) + warp * (R / 2);
        const int xo0 = tx * (kReduceTW / 2) + 2 * lane;
        const int rows_valid = min(R / 2, d.Hv - yo0);
        const int cols_valid = min(2, d.Wv - xo0);
        if (rows_valid > 0 && cols_valid > 0) {
            const TIn *src = reinterpret_cast<const TIn *>(smem + s * STAGE) + (warp * R) * BW + 4 * lane;
            TOut *dst = reinterpret_cast<TOut *>(d.out) + plane * d.out_plane +
                        static_cast<int64_t>(yo0) * d.out_pitch + xo0;
            reduce_strip<TIn, TOut, R, BW>(src, kk, os2, scaled, dst, d.out_pitch, rows_valid, cols_valid);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        if (++s == S) {
            s = 0;
            phase ^= 1u;
        }
    }
}

struct ReduceEntry {
    int tile_h, rows, stages;
    const void *fn;
    int smem, threads;
};

template <class TIn, class TOut, int TH, int R, int S>
ReduceEntry reduce_entry()
{
    return ReduceEntry{TH, R, S, reinterpret_cast<const void *>(&reduce_kernel<TIn, TOut, TH, R, S>),
                       S * fused_stage_bytes<TIn, TH, kReduceTW, kReduceTaps>(), 32 * (TH / R + 1)};
}

// Compiled shapes per storage pair, (input rows per tile, input rows per warp,
// stages), unique per (input rows per tile, stages).  A warp re-forms the row
// pass of the R+3 input rows its R/2 output rows need, so taller strips repeat
// less of it ((R+3)/R: 1.75 at R = 4, 1.19 at R = 16).  The first entry is the
// default, chosen by measurement on 3x8192x8192: FP32 128/8/3 (0.156 ms
// against 0.160 ms for 64/4/3); 16-bit to 16-bit 128/16/3 (BF16 0.086 ms
// against 0.126 ms); 16-bit to FP32 128/8/4 (BF16 0.099 ms); FP8 to FP8 and
// to FP32 128/16/5 (0.095 / 0.096 ms against 0.142 / 0.107 ms).
#define SC5_RED(TI, TO, TH, R, S) reduce_entry<TI, TO, TH, R, S>()
constexpr int kReduceShapes = 4;

const ReduceEntry *reduce_entries(int in_dtype, int out_dtype)
{
    static const ReduceEntry f32_f32[] = {SC5_RED(float, float, 128, 8, 3), SC5_RED(float, float, 64, 4, 3),
                                          SC5_RED(float, float, 64, 8, 2), SC5_RED(float, float, 128, 16, 2)};
#define SC5_RED_16(TI)                                                                               \
    {SC5_RED(TI, TI, 128, 16, 3), SC5_RED(TI, TI, 64, 4, 4), SC5_RED(TI, TI, 64, 8, 3),             \
     SC5_RED(TI, TI, 128, 8, 4)}
#define SC5_RED_16_F32(TI)                                                                           \
    {SC5_RED(TI, float, 128, 8, 4), SC5_RED(TI, float, 64, 4, 4), SC5_RED(TI, float, 64, 8, 3),     \
     SC5_RED(TI, float, 128, 16, 3)}
    static const ReduceEntry bf_bf[] = SC5_RED_16(bf16_t);
    static const ReduceEntry bf_f32[] = SC5_RED_16_F32(bf16_t);
    static const ReduceEntry h_h[] = SC5_RED_16(f16_t);
    static const ReduceEntry h_f32[] = SC5_RED_16_F32(f16_t);
    static const ReduceEntry e_e[] = {SC5_RED(fp8e4m3_t, fp8e4m3_t, 128, 16, 5),
                                      SC5_RED(fp8e4m3_t, fp8e4m3_t, 64, 4, 6),
                                      SC5_RED(fp8e4m3_t, fp8e4m3_t, 64, 8, 5),
                                      SC5_RED(fp8e4m3_t, fp8e4m3_t, 128, 8, 6)};
    static const ReduceEntry e_f32[] = {SC5_RED(fp8e4m3_t, float, 128, 16, 5), SC5_RED(fp8e4m3_t, float, 64, 4, 6),
                                        SC5_RED(fp8e4m3_t, float, 64, 8, 5), SC5_RED(fp8e4m3_t, float, 128, 8, 6)};
#undef SC5_RED_16
#undef SC5_RED_16_F32
    if (in_dtype == SC5_F32 && out_dtype == SC5_F32) return f32_f32;
    if (in_dtype == SC5_BF16 && out_dtype == SC5_BF16) return bf_bf;
    if (in_dtype == SC5_BF16 && out_dtype == SC5_F32) return bf_f32;
    if (in_dtype == SC5_F16 && out_dtype == SC5_F16) return h_h;
    if (in_dtype == SC5_F16 && out_dtype == SC5_F32) return h_f32;
    if (in_dtype == SC5_FP8E4M3 && out_dtype == SC5_FP8E4M3) return e_e;
    if (in_dtype == SC5_FP8E4M3 && out_dtype == SC5_F32) return e_f32;
    return nullptr;
}

// The entry with these input rows per tile and stages (0 = any stages), or
// the default when tile_h is 0; false if none is compiled.
bool reduce_lookup(int in_dtype, int out_dtype, int tile_h, int stages, ReduceEntry *e)
{
    const ReduceEntry *list = reduce_entries(in_dtype, out_dtype);
    if (!list) return false;
    for (int i = 0; i < kReduceShapes; ++i)
        if (tile_h == 0 || (list[i].tile_h == tile_h && (stages == 0 || list[i].stages == stages))) {
            *e = list[i];
            return true;
        }
    return false;
}

}  // namespace

int *status_word();  // sc5_fused.cu

bool reduce_shape(int in_dtype, int out_dtype, int tile_h, int stages, FusedShape *sh)
{
    ReduceEntry e;
    if (!reduce_lookup(in_dtype, out_dtype, tile_h, stages, &e)) return false;
    *sh = FusedShape{e.tile_h, kReduceTW, e.rows, e.stages};
    return true;
}

cudaError_t launch_reduce(int in_dtype, int out_dtype, const FusedShape &sh, const ImgDesc &desc, int64_t ntiles,
                          int ctas_per_sm, cudaStream_t st)
{
    ReduceEntry e;
    if (!reduce_lookup(in_dtype, out_dtype, sh.tile_h, sh.stages, &e) || e.rows != sh.rows_per_thread)
        return cudaErrorInvalidValue;
    if (ntiles <= 0) return cudaSuccess;
    static std::mutex mu;
    static std::set<std::pair<const void *, int>> done;
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!done.count({e.fn, dev})) {
            err = cudaFuncSetAttribute(e.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, e.smem);
            if (err != cudaSuccess) return err;
            done.insert({e.fn, dev});
        }
    }
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, e.fn, e.threads, e.smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
    const int64_t cap = static_cast<int64_t>(num_sms()) * per_sm;
    const int grid = static_cast<int>(ntiles < cap ? ntiles : cap);
    int *status = status_word();
    if (!status) return cudaErrorInvalidDevicePointer;
    void *args[] = {const_cast<ImgDesc *>(&desc), &ntiles, &status};
    err = cudaLaunchKernel(e.fn, dim3(grid), dim3(e.threads), args, e.smem, st);
    if (err == cudaSuccess) note_launches(1);
    return err;
}

}  // namespace sc5
