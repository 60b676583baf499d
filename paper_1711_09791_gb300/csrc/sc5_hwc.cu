// sc5_hwc.cu -- the fused single-pass kernel for pixel-interleaved (HWC)
// images: value (p, y, x) of a 3-plane image at y*pitch + 3*x + p.
//
// TMA boxes must start on a 16-byte boundary in their innermost dimension,
// so one plane of an interleaved row cannot be fetched on its own.  Whole
// RGB runs can: a tile of 128 output pixels needs input pixels
// [x0, x0+132), loaded as two boxes of 68 pixels x 3 values, A = [x0, x0+68)
// and B = [x0+64, x0+132); both start at 3*x0 (+192) elements, 16-byte
// aligned.  Lane l of a consumer warp owns output pixels [4l, 4l+4) of the
// tile for all three planes: it reads its 8 input pixels x 3 values
// contiguously from box A (l < 16) or B, splits them into three planes in
// registers, and runs the separable arithmetic of the planar kernel on each
// plane (same FP32 operations in the same order, so results are bitwise
// those of the planar fused kernel).  Outputs are written interleaved, 12
// contiguous values per lane and row.
#include <cstring>
#include <mutex>
#include <set>
#include <utility>

#include "sc5_fused_impl.cuh"

namespace sc5 {

constexpr int kHwcPlanes = 3;
constexpr int kHwcTW = 128;        // output pixels per tile
constexpr int kHwcBoxPx = 68;      // input pixels per box
constexpr int kHwcBoxBOffset = 64; // first pixel of box B

template <class TIn>
__host__ __device__ constexpr int hwc_box_w()
{
    // 68 pixels x 3 values, rounded up to 16 bytes
    return (kHwcBoxPx * kHwcPlanes * Fmt<TIn>::bytes + 15) / 16 * 16 / Fmt<TIn>::bytes;
}

template <class TIn, int TH>
__host__ __device__ constexpr int hwc_box_bytes()
{
    return hwc_box_w<TIn>() * (TH + kHalo) * Fmt<TIn>::bytes;
}

// box B starts on a 128-byte boundary after box A
template <class TIn, int TH>
__host__ __device__ constexpr int hwc_boxb_offset()
{
    return (hwc_box_bytes<TIn, TH>() + 127) / 128 * 128;
}

template <class TIn, int TH>
__host__ __device__ constexpr int hwc_stage_bytes()
{
    return (hwc_boxb_offset<TIn, TH>() + hwc_box_bytes<TIn, TH>() + 127) / 128 * 128;
}

// Pairs of plane c of one input row (8 pixels x 3 values in v) for the
// packed row pass, in the pairing of the planar kernel.
template <class TIn>
__device__ __forceinline__ void hwc_plane_pairs(const float (&v)[24], int c, uint64_t (&PL)[kTaps],
                                                uint64_t (&PR)[kTaps])
{
    float a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = v[3 * j + c];
    if constexpr (Fmt<TIn>::kStride2) {
#pragma unroll
        for (int j = 0; j < kTaps; ++j) {
            PL[j] = pack2(a[j], a[j + 2]);
            PR[j] = pack2(a[j + 1], a[j + 3]);
        }
    } else {
#pragma unroll
        for (int j = 0; j < kTaps; ++j) {
            PL[j] = pack2(a[j], a[j + 1]);
            PR[j] = pack2(a[j + 2], a[j + 3]);
        }
    }
}

// Store 4 pixels x 3 planes of one output row, interleaved.
template <class TIn, class TOut>
__device__ __forceinline__ void hwc_store_row(const uint64_t (&vL)[kHwcPlanes], const uint64_t (&vR)[kHwcPlanes],
                                              uint64_t os2, bool scaled, TOut *dst, int px_valid, bool vec)
{
    float w[12];
#pragma unroll
    for (int c = 0; c < kHwcPlanes; ++c) {
        uint64_t l = vL[c], r = vR[c];
        if (scaled) {
            l = mul2(l, os2);
            r = mul2(r, os2);
        }
        float v[4];
        if constexpr (Fmt<TIn>::kStride2) {
            unpack2(l, v[0], v[2]);
            unpack2(r, v[1], v[3]);
        } else {
            unpack2(l, v[0], v[1]);
            unpack2(r, v[2], v[3]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) w[3 * j + c] = v[j];
    }
    if (vec && px_valid == 4) {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const float u[4] = {w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]};
            Fmt<TOut>::store4(dst + 4 * q, u);
        }
    } else {
#pragma unroll
        for (int q = 0; q < 12; ++q)
            if (q < 3 * px_valid) Fmt<TOut>::store1(dst + q, w[q]);
    }
}

template <class TIn, class TOut, int R, int BW, bool FULL = false>
__device__ __forceinline__ void hwc_strip(const TIn *__restrict__ s, const uint64_t (&kk)[kTaps], uint64_t os2,
                                          bool scaled, TOut *__restrict__ out, int64_t out_pitch, int rows_valid,
                                          int px_valid, bool vec)
{
    // FULL: all R rows and 4 pixels inside the image, vector stores aligned.
    if constexpr (FULL) {
        rows_valid = R;
        px_valid = 4;
        vec = true;
    }
    uint64_t accL[R][kHwcPlanes], accR[R][kHwcPlanes];
#pragma unroll
    for (int r = 0; r < R + kHalo; ++r) {
        float v[24];
#pragma unroll
        for (int q = 0; q < 24; q += 4) Fmt<TIn>::load4(s + r * BW + q, v + q);
#pragma unroll
        for (int c = 0; c < kHwcPlanes; ++c) {
            uint64_t PL[kTaps], PR[kTaps];
            hwc_plane_pairs<TIn>(v, c, PL, PR);
            uint64_t hL = mul2(kk[0], PL[0]);
            uint64_t hR = mul2(kk[0], PR[0]);
#pragma unroll
            for (int t = 1; t < kTaps; ++t) {
                hL = fma2(kk[t], PL[t], hL);
                hR = fma2(kk[t], PR[t], hR);
            }
#pragma unroll
            for (int t = 0; t < kTaps; ++t) {
                const int o = r - t;
                if (o >= 0 && o < R) {
                    accL[o][c] = (t == 0) ? mul2(kk[0], hL) : fma2(kk[t], hL, accL[o][c]);
                    accR[o][c] = (t == 0) ? mul2(kk[0], hR) : fma2(kk[t], hR, accR[o][c]);
                }
            }
        }
        const int o = r - kHalo;
        if (o >= 0 && o < rows_valid)
            hwc_store_row<TIn, TOut>(accL[o], accR[o], os2, scaled, out + static_cast<int64_t>(o) * out_pitch,
                                     px_valid, vec);
    }
}

// Per-image parameters of the HWC kernel.
struct alignas(128) HwcDesc {  // CUtensorMap's own alignment
    CUtensorMap tmap;   // 2-D: (3*W values, H rows)
    void *out;          // first VALID output value
    int64_t out_pitch;  // elements
    int32_t Hv, Wv, tiles_x, tiles_y;
    float k[kTaps];
    float oscale;
    int32_t vec;
};

template <class TIn, class TOut, int TH, int R, int S>
__global__ void __launch_bounds__(32 * (TH / R + 1), 1)
hwc_kernel(const __grid_constant__ HwcDesc d, int64_t ntiles, int *status)
{
    constexpr int NC = TH / R;
    constexpr int BW = hwc_box_w<TIn>();
    constexpr int BOX_BYTES = hwc_box_bytes<TIn, TH>();
    constexpr int BOXB = hwc_boxb_offset<TIn, TH>();
    constexpr int STAGE = hwc_stage_bytes<TIn, TH>();
    constexpr uint32_t TX = 2 * BOX_BYTES;

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

    if (warp == NC) {
        if (lane != 0) return;
        int64_t issued = 0;
        int s = 0;             // stage of this tile
        uint32_t phase = 0;    // parity of the stage's current use
        bool wrapped = false;  // every stage has been used once
        for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
            if (wrapped && !mbar_wait_bounded(&empty[s], phase ^ 1u, kWaitLimitNs)) {
                record_error(status, kDevErrTmaTimeout);
                break;
            }
            const int ty = static_cast<int>(t / d.tiles_x);
            const int tx = static_cast<int>(t - static_cast<int64_t>(ty) * d.tiles_x);
            mbar_arrive_expect_tx(&full[s], TX);
            unsigned char *dst = smem + s * STAGE;
            const int x0 = tx * kHwcTW * kHwcPlanes;
            tma_load_3d(dst, &d.tmap, &full[s], x0, ty * TH, 0);
            tma_load_3d(dst + BOXB, &d.tmap, &full[s], x0 + kHwcBoxBOffset * kHwcPlanes, ty * TH, 0);
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

    uint64_t kk[kTaps];
#pragma unroll
    for (int q = 0; q < kTaps; ++q) kk[q] = pack2(d.k[q], d.k[q]);
    const uint64_t os2 = pack2(d.oscale, d.oscale);
    const bool scaled = d.oscale != 1.f;
    const int half = lane >> 4;              // 0: box A, 1: box B
    const int lpx = 4 * (lane & 15);         // first pixel of the lane inside its box
    int s = 0;
    uint32_t phase = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        if (!mbar_wait_bounded(&full[s], phase, kWaitLimitNs)) {
            if (lane == 0) record_error(status, kDevErrTmaTimeout);
            mbar_wait_bounded(&full[s], phase, kDrainLimitNs);
            return;
        }
        const int ty = static_cast<int>(t / d.tiles_x);
        const int tx = static_cast<int>(t - static_cast<int64_t>(ty) * d.tiles_x);
        const int ry0 = ty * TH + warp * R;
        const int px = tx * kHwcTW + 4 * lane;   // first output pixel of the lane
        const int rows_valid = min(R, d.Hv - ry0);
        const int px_valid = min(4, d.Wv - px);
        if (rows_valid > 0 && px_valid > 0) {
            const TIn *src = reinterpret_cast<const TIn *>(smem + s * STAGE + half * BOXB) +
                             (warp * R) * BW + lpx * kHwcPlanes;
            TOut *dst = reinterpret_cast<TOut *>(d.out) + static_cast<int64_t>(ry0) * d.out_pitch +
                        static_cast<int64_t>(px) * kHwcPlanes;
            // guard-free interior strips for 8/16-bit in and out (3x8192^2: BF16
            // 0.156 -> 0.152 ms, FP8 0.175 -> 0.163 ms); with FP32 output they
            // measured 21% slower here, so those keep the guarded strips
            if (sizeof(TIn) < 4 && sizeof(TOut) < 4 && rows_valid == R && px_valid == 4 && d.vec != 0)
                hwc_strip<TIn, TOut, R, BW, true>(src, kk, os2, scaled, dst, d.out_pitch, R, 4, true);
            else
                hwc_strip<TIn, TOut, R, BW, false>(src, kk, os2, scaled, dst, d.out_pitch, rows_valid, px_valid,
                                                   d.vec != 0);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        if (++s == S) {
            s = 0;
            phase ^= 1u;
        }
    }
}

// ------------------------------------------------------------------ host side

struct HwcEntry {
    int tile_h;
    const void *fn;
    int smem, threads;
};

template <class TIn, class TOut, int TH, int R, int S>
static HwcEntry hwc_entry()
{
    return HwcEntry{TH, reinterpret_cast<const void *>(&hwc_kernel<TIn, TOut, TH, R, S>),
                    S * hwc_stage_bytes<TIn, TH>(), 32 * (TH / R + 1)};
}

static bool hwc_lookup(int in_dtype, int out_dtype, HwcEntry *e)
{
    // (tile rows, rows per lane, stages): 16 consumer warps, 3 planes per lane.
    // FP32: 32-row tiles with 2 rows per lane and 3 stages (3x8192x8192: 0.253 ms
    // against 0.276 ms for 64/4/2); the 8/16-bit formats lose with 2-row strips
    // (BF16 0.19 against 0.15 ms) and keep 4 rows.
    static const HwcEntry f32_f32 = hwc_entry<float, float, 32, 2, 3>();
    static const HwcEntry bf_bf = hwc_entry<bf16_t, bf16_t, 64, 4, 3>();
    // BF16 -> FP32 is closer to HBM-bound and takes FP32's 2-row strips (0.208
    // ms against 0.231 ms for 64/4/3); FP16 -> FP32 (its widening costs more)
    // gains nothing there (0.228 against 0.226 ms) and FP8 -> FP32 loses (0.240
    // against 0.187 ms): both keep 4-row strips
    static const HwcEntry bf_f32 = hwc_entry<bf16_t, float, 32, 2, 6>();
    static const HwcEntry h_h = hwc_entry<f16_t, f16_t, 64, 4, 3>();
    static const HwcEntry h_f32 = hwc_entry<f16_t, float, 64, 4, 3>();
    static const HwcEntry e_e = hwc_entry<fp8e4m3_t, fp8e4m3_t, 64, 4, 5>();
    static const HwcEntry e_f32 = hwc_entry<fp8e4m3_t, float, 64, 4, 5>();
    const HwcEntry *r = nullptr;
    if (in_dtype == SC5_F32 && out_dtype == SC5_F32) r = &f32_f32;
    if (in_dtype == SC5_BF16 && out_dtype == SC5_BF16) r = &bf_bf;
    if (in_dtype == SC5_BF16 && out_dtype == SC5_F32) r = &bf_f32;
    if (in_dtype == SC5_F16 && out_dtype == SC5_F16) r = &h_h;
    if (in_dtype == SC5_F16 && out_dtype == SC5_F32) r = &h_f32;
    if (in_dtype == SC5_FP8E4M3 && out_dtype == SC5_FP8E4M3) r = &e_e;
    if (in_dtype == SC5_FP8E4M3 && out_dtype == SC5_F32) r = &e_f32;
    if (!r) return false;
    *e = *r;
    return true;
}

int hwc_box_cols(int in_dtype)
{
    switch (in_dtype) {
    case SC5_F32: return hwc_box_w<float>();
    case SC5_BF16: return hwc_box_w<bf16_t>();
    case SC5_F16: return hwc_box_w<f16_t>();
    case SC5_FP8E4M3: return hwc_box_w<fp8e4m3_t>();
    default: return 0;
    }
}

int hwc_tile_h(int in_dtype, int out_dtype)
{
    HwcEntry e;
    return hwc_lookup(in_dtype, out_dtype, &e) ? e.tile_h : 0;
}

int *status_word();  // sc5_fused.cu

cudaError_t launch_hwc(int in_dtype, int out_dtype, const void *desc_ptr, int64_t ntiles, int ctas_per_sm,
                       cudaStream_t st)
{
    HwcEntry e;
    if (!hwc_lookup(in_dtype, out_dtype, &e)) return cudaErrorInvalidValue;
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
    void *args[] = {const_cast<void *>(desc_ptr), &ntiles, &status};
    err = cudaLaunchKernel(e.fn, dim3(grid), dim3(e.threads), args, e.smem, st);
    if (err == cudaSuccess) note_launches(1);
    return err;
}

// Fill the HWC descriptor: the caller passes the encoded tensor map.
size_t hwc_desc_size() { return sizeof(HwcDesc); }

void hwc_fill(void *desc_ptr, const CUtensorMap &m, void *out, int64_t out_pitch, int Hv, int Wv, int tile_h,
              const float *k, float oscale, bool vec)
{
    HwcDesc *d = static_cast<HwcDesc *>(desc_ptr);
    std::memset(d, 0, sizeof *d);
    d->tmap = m;
    d->out = out;
    d->out_pitch = out_pitch;
    d->Hv = Hv;
    d->Wv = Wv;
    d->tiles_x = (Wv + kHwcTW - 1) / kHwcTW;
    d->tiles_y = (Hv + tile_h - 1) / tile_h;
    for (int i = 0; i < kTaps; ++i) d->k[i] = k[i];
    d->oscale = oscale;
    d->vec = vec ? 1 : 0;
}

}  // namespace sc5
