// sc5_api.cu -- the C ABI of libsepconv5: plans (validation, TMA tensor
// maps, tile grid, launch configuration), single-image runs of every form
// (fused, two-pass, direct, HWC, pyramid REDUCE step), the in-place and
// offload calls, pyramids (chained REDUCE plans, optionally a CUDA graph),
// batches with a tile work-list (one-shot or captured in a CUDA graph), the
// device status word, the empty-launch probe and the launch counter.
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "sc5_internal.h"
#include "sc5_tune.h"

namespace sc5 {

static thread_local std::string t_err;
static std::atomic<int64_t> g_launches{0};

void note_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

sc5_status fail(sc5_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_err = buf;
    return st;
}

sc5_status fail_cuda(cudaError_t e, const char *what)
{
    return fail(e == cudaErrorMemoryAllocation ? SC5_ENOMEM : SC5_ECUDA, "%s: %s (%s)", what,
                cudaGetErrorString(e), cudaGetErrorName(e));
}

void clear_error() { t_err.clear(); }

int dtype_bytes(int dtype)
{
    switch (dtype) {
    case SC5_F32: return 4;
    case SC5_BF16:
    case SC5_F16: return 2;
    case SC5_FP8E4M3: return 1;
    default: return 0;
    }
}

int num_sms()
{
    static std::mutex mu;
    static int cache[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    std::lock_guard<std::mutex> lk(mu);
    if (!cache[dev]) cudaDeviceGetAttribute(&cache[dev], cudaDevAttrMultiProcessorCount, dev);
    return cache[dev];
}

static bool pair_supported(int in_dtype, int out_dtype)
{
    return fused_num_shapes(in_dtype, out_dtype) > 0;
}

// ------------------------------------------------------------------ tensor maps

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// 3-D map of a planar image (x = column, y = row, z = plane), box of
// box_w x box_h x 1 elements, zero fill outside the image.
static sc5_status encode_image_map(CUtensorMap *m, int dtype, const void *base, int P, int H, int W,
                                   int64_t pitch, int box_w, int box_h, int64_t plane_stride = 0)
{
    if (plane_stride <= 0) plane_stride = pitch * H;
    auto fn = encode_fn();
    if (!fn) return fail(SC5_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const int es = dtype_bytes(dtype);
    CUtensorMapDataType t = es == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                            : es == 2 ? CU_TENSOR_MAP_DATA_TYPE_UINT16
                                      : CU_TENSOR_MAP_DATA_TYPE_UINT8;
    const cuuint64_t dims[3] = {static_cast<cuuint64_t>(W), static_cast<cuuint64_t>(H),
                                static_cast<cuuint64_t>(P)};
    const cuuint64_t strides[2] = {static_cast<cuuint64_t>(pitch) * es,
                                   static_cast<cuuint64_t>(plane_stride) * es};
    const cuuint32_t box[3] = {static_cast<cuuint32_t>(box_w), static_cast<cuuint32_t>(box_h), 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(m, t, 3, const_cast<void *>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(SC5_EINVAL, "cuTensorMapEncodeTiled failed (CUresult %d)", (int)r);
    return SC5_OK;
}

// Columns of one TMA box (as fused_box_w in the kernel): the 128 columns a
// box covers (a 256-wide tile is two boxes) plus the taps-1 halo, rounded up
// to 16 bytes and to the last lane's whole 4-element loads (4 output columns
// per lane in 128-wide tiles, 8 in 256-wide ones).
static int box_w_for(int dtype, int tile_w, int taps = kTaps)
{
    const int es = dtype_bytes(dtype);
    const int cols = tile_w / 32;
    const int cover = std::min(tile_w, 128);
    const int row_elems = (cols + taps - 1 + 3) / 4 * 4;
    const int need = std::max(cover + taps - 1, cover - cols + row_elems);
    return (need * es + 15) / 16 * 16 / es;
}

// ------------------------------------------------------------------ validation

// Planes of an image do not overlap: stacked (stride >= rows * pitch) or
// row-interleaved (stride >= width and pitch >= planes * stride).
static bool planes_disjoint(int P, int64_t rows, int64_t width, int64_t pitch, int64_t stride)
{
    return P == 1 || stride >= rows * pitch || (stride >= width && pitch >= P * stride);
}

static sc5_status check_image(int in_dtype, int out_dtype, int border, const void *in, const void *out,
                              int P, int H, int W, int64_t in_pitch, int64_t out_pitch, float in_scale,
                              float out_scale, bool need_ptrs, int64_t in_ps = 0, int64_t out_ps = 0,
                              int taps = kTaps)
{
    if (P < 1 || H < taps || W < taps)
        return fail(SC5_EINVAL, "need planes >= 1, H >= %d, W >= %d (got %d, %d, %d)", taps, taps, P, H, W);
    const int halo = taps - 1;
    if (H > 65535 * 8 || W > (1 << 30)) return fail(SC5_EINVAL, "image too large (H <= 524280, W < 2^30)");
    const int ei = dtype_bytes(in_dtype), eo = dtype_bytes(out_dtype);
    if (!ei || !eo) return fail(SC5_EINVAL, "unknown dtype (%d, %d)", in_dtype, out_dtype);
    if (border != SC5_BORDER_VALID && border != SC5_BORDER_KEEP) return fail(SC5_EINVAL, "unknown border %d", border);
    const int64_t wout = border == SC5_BORDER_KEEP ? W : W - halo;
    if (in_pitch < W) return fail(SC5_EINVAL, "in_pitch %lld < W %d", (long long)in_pitch, W);
    if (out_pitch < wout) return fail(SC5_EINVAL, "out_pitch %lld < output width %lld", (long long)out_pitch, (long long)wout);
    if ((in_pitch * ei) % 16) return fail(SC5_EINVAL, "in_pitch * element size must be a multiple of 16 bytes");
    const int64_t hout = border == SC5_BORDER_KEEP ? H : H - halo;
    if (in_ps < 0 || out_ps < 0) return fail(SC5_EINVAL, "negative plane stride");
    if (in_ps == 0) in_ps = static_cast<int64_t>(H) * in_pitch;
    if (out_ps == 0) out_ps = hout * out_pitch;
    if ((in_ps * ei) % 16) return fail(SC5_EINVAL, "in_plane_stride * element size must be a multiple of 16 bytes");
    if (!planes_disjoint(P, H, W, in_pitch, in_ps) || !planes_disjoint(P, hout, wout, out_pitch, out_ps))
        return fail(SC5_EINVAL, "plane stride makes planes overlap (need stacked or row-interleaved planes)");
    if ((static_cast<double>(in_pitch) * ei * H * P) >= 1099511627776.0) return fail(SC5_EINVAL, "image larger than 2^40 bytes");
    if (!(in_scale > 0.f) || !std::isfinite(in_scale) || !(out_scale > 0.f) || !std::isfinite(out_scale))
        return fail(SC5_EINVAL, "scales must be finite and > 0");
    if (need_ptrs) {
        if (!in || !out) return fail(SC5_EINVAL, "null image pointer");
        if (reinterpret_cast<uintptr_t>(in) % 16) return fail(SC5_EINVAL, "input must be 16-byte aligned");
        if (reinterpret_cast<uintptr_t>(out) % eo) return fail(SC5_EINVAL, "output not aligned to its element size");
        const char *a = static_cast<const char *>(in), *b = static_cast<const char *>(out);
        // one past the last element of the last row of the last plane
        const char *a_end = a + (static_cast<size_t>(P - 1) * in_ps + static_cast<size_t>(H - 1) * in_pitch + W) * ei;
        const char *b_end = b + (static_cast<size_t>(P - 1) * out_ps + static_cast<size_t>(hout - 1) * out_pitch + wout) * eo;
        if (a < b_end && b < a_end) return fail(SC5_EINVAL, "input and output overlap");
    }
    return SC5_OK;
}

static bool taps_finite(const float *k)
{
    for (int i = 0; i < kTaps; ++i)
        if (!std::isfinite(k[i])) return false;
    return true;
}

// Effective plane strides of a plan (elements).
static int64_t in_plane_of(const sc5_plan_desc &d)
{
    return d.in_plane_stride > 0 ? d.in_plane_stride : static_cast<int64_t>(d.H) * d.in_pitch;
}

static int taps_of(const sc5_plan_desc &d) { return d.taps > 0 ? d.taps : kTaps; }

static int64_t out_plane_of(const sc5_plan_desc &d)
{
    const int64_t hout = d.border == SC5_BORDER_KEEP ? d.H : d.H - (taps_of(d) - 1);
    return d.out_plane_stride > 0 ? d.out_plane_stride : hout * d.out_pitch;
}

static bool default_strides(const sc5_plan_desc &d)
{
    return d.in_plane_stride == 0 && d.out_plane_stride == 0;
}

// Fill an ImgDesc for one image (tensor map included).
static sc5_status fill_desc(ImgDesc *d, int in_dtype, int out_dtype, int border, const FusedShape &sh,
                            const void *in, void *out, int P, int H, int W, int64_t in_pitch,
                            int64_t out_pitch, const float *k, float in_scale, float out_scale,
                            const float *K = nullptr, int64_t in_ps = 0, int64_t out_ps = 0, int taps = kTaps)
{
    std::memset(d, 0, sizeof *d);
    const int halo = taps - 1, radius = halo / 2;
    sc5_status st = encode_image_map(&d->tmap, in_dtype, in, P, H, W, in_pitch,
                                     box_w_for(in_dtype, sh.tile_w, taps), sh.tile_h + halo, in_ps);
    if (st != SC5_OK) return st;
    const int eo = dtype_bytes(out_dtype);
    char *ob = static_cast<char *>(out);
    int64_t plane_rows = H - halo;
    if (border == SC5_BORDER_KEEP) {
        ob += (radius * out_pitch + radius) * eo;
        plane_rows = H;
    }
    d->out = ob;
    d->out_pitch = out_pitch;
    d->out_plane = out_ps > 0 ? out_ps : plane_rows * out_pitch;
    d->Hv = H - halo;
    d->Wv = W - halo;
    d->tiles_x = (d->Wv + sh.tile_w - 1) / sh.tile_w;
    d->tiles_y = (d->Hv + sh.tile_h - 1) / sh.tile_h;
    for (int i = 0; i < taps; ++i) d->k[i] = k[i];
    if (taps == kTaps)
        for (int i = 0; i < kTaps * kTaps; ++i)
            d->K[i] = K ? K[i] : static_cast<float>(static_cast<double>(k[i / kTaps]) * k[i % kTaps]);
    d->oscale = static_cast<float>(static_cast<double>(out_scale) / static_cast<double>(in_scale));
    d->vec = (reinterpret_cast<uintptr_t>(ob) % (4 * eo) == 0 && out_pitch % 4 == 0) ? 1 : 0;
    return SC5_OK;
}

}  // namespace sc5

using namespace sc5;

// ------------------------------------------------------------------ plans

struct sc5_plan_s {
    sc5_plan_desc d;
    int device = 0;
    int shape_idx = 0;
    FusedShape shape{};
    int ctas_per_sm = 0;
    float *T = nullptr;
    int64_t t_pitch = 0;
    // batch workspace (device + pinned staging), grown on demand
    unsigned char *ws_dev = nullptr;
    size_t ws_cap = 0;
    unsigned char *ws_host = nullptr;
    size_t ws_host_cap = 0;
    cudaEvent_t ws_done = nullptr;
    bool ws_pending = false;
    // copy-back scratch (sepconv5_run_inplace with a single-pass algo)
    void *scratch = nullptr;
    // offload staging (sepconv5_run_host)
    void *stage_in = nullptr;
    void *stage_out = nullptr;
    cudaStream_t s_in = nullptr, s_out = nullptr;
    std::vector<cudaEvent_t> ev;
};

namespace sc5 {
sc5_status choose_shape(int in_dtype, int out_dtype, int H, int W, const sc5_plan_desc *ov, int *idx, int *ctas,
                        bool direct, int taps, bool batch)
{
    if (ov && (ov->tile_h || ov->tile_w || ov->stages)) {
        const int i = fused_find_shape(in_dtype, out_dtype, ov->tile_h ? ov->tile_h : 64,
                                       ov->tile_w ? ov->tile_w : 128, ov->stages, direct, taps);
        if (i < 0) return fail(SC5_EINVAL, "no compiled fused shape %dx%d with %d stages for this dtype pair",
                               ov->tile_h, ov->tile_w, ov->stages);
        *idx = i;
        *ctas = ov->ctas_per_sm > 0 ? ov->ctas_per_sm : 0;
    } else if (direct || taps != kTaps) {
        *idx = 0;
        *ctas = (ov && ov->ctas_per_sm > 0) ? ov->ctas_per_sm : fused_default_ctas(in_dtype, out_dtype, 0, direct, taps);
    } else {
        int th, tw, stg, c;
        tune_from_environment(in_dtype, out_dtype);
        // the table's entry, else the shape's own default (0: as many as fit);
        // the descriptor overrides either
        *ctas = 0;
        bool tuned = false;
        if (tune_lookup_internal(in_dtype, out_dtype, H, W, batch ? kKindBatch : kKindSingle, &th, &tw, &stg, &c)) {
            *idx = fused_find_shape(in_dtype, out_dtype, th, tw, stg);
            *ctas = c;
            tuned = *idx >= 0;
        }
        if (*idx < 0) *idx = 0;
        if (!tuned) *ctas = fused_default_ctas(in_dtype, out_dtype, *idx);
        if (ov && ov->ctas_per_sm > 0) *ctas = ov->ctas_per_sm;
    }
    const int maxc = fused_max_ctas_per_sm(in_dtype, out_dtype, *idx, direct, taps);
    if (maxc <= 0) return fail(SC5_ECUDA, "occupancy query failed for fused shape %d", *idx);
    if (*ctas <= 0 || *ctas > maxc) *ctas = maxc;
    return SC5_OK;
}
}  // namespace sc5

// Pixel-interleaved 3-plane images: validation and plan.
static sc5_status plan_hwc(const sc5_plan_desc &d, sc5_plan *out)
{
    if (d.planes != 3) return fail(SC5_EINVAL, "the HWC layout is built for 3 planes");
    if (d.algo != SC5_ALGO_FUSED || d.taps != kTaps || d.border != SC5_BORDER_VALID)
        return fail(SC5_EINVAL, "the HWC layout is built for the fused form, width 5, VALID border");
    if (d.in_plane_stride || d.out_plane_stride) return fail(SC5_EINVAL, "plane strides do not apply to HWC");
    if (d.H < 5 || d.W < 5 || d.H > 65535 * 8 || d.W > (1 << 28)) return fail(SC5_EINVAL, "bad image size");
    const int ei = dtype_bytes(d.in_dtype), th = hwc_tile_h(d.in_dtype, d.out_dtype);
    if (!ei || !th) return fail(SC5_EINVAL, "dtype pair (%d -> %d) not built", d.in_dtype, d.out_dtype);
    if (d.in_pitch < 3ll * d.W || (d.in_pitch * ei) % 16)
        return fail(SC5_EINVAL, "HWC in_pitch must be >= 3*W values with in_pitch * element size a multiple of 16");
    if (d.out_pitch < 3ll * (d.W - kHalo)) return fail(SC5_EINVAL, "HWC out_pitch must be >= 3*(W-4) values");
    sc5_plan p = new (std::nothrow) sc5_plan_s;
    if (!p) return fail(SC5_ENOMEM, "host allocation failed");
    p->d = d;
    cudaGetDevice(&p->device);
    p->shape = FusedShape{th, 128, 4, 0};
    if (cudaEventCreateWithFlags(&p->ws_done, cudaEventDisableTiming) != cudaSuccess) {
        delete p;
        return fail(SC5_ECUDA, "cudaEventCreate failed");
    }
    *out = p;
    return SC5_OK;
}

static sc5_status run_hwc(sc5_plan p, const void *in, void *out, const float *k, float in_scale, float out_scale,
                          cudaStream_t s)
{
    const sc5_plan_desc &d = p->d;
    const int ei = dtype_bytes(d.in_dtype), eo = dtype_bytes(d.out_dtype);
    if (!in || !out) return fail(SC5_EINVAL, "null image pointer");
    if (reinterpret_cast<uintptr_t>(in) % 16) return fail(SC5_EINVAL, "input must be 16-byte aligned");
    if (reinterpret_cast<uintptr_t>(out) % eo) return fail(SC5_EINVAL, "output not aligned to its element size");
    if (!(in_scale > 0.f) || !std::isfinite(in_scale) || !(out_scale > 0.f) || !std::isfinite(out_scale))
        return fail(SC5_EINVAL, "scales must be finite and > 0");
    if (!taps_finite(k)) return fail(SC5_EINVAL, "taps must be finite");
    const int Hv = d.H - kHalo, Wv = d.W - kHalo;
    const char *a = static_cast<const char *>(in), *b = static_cast<const char *>(out);
    const char *a_end = a + (static_cast<size_t>(d.H - 1) * d.in_pitch + 3ull * d.W) * ei;
    const char *b_end = b + (static_cast<size_t>(Hv - 1) * d.out_pitch + 3ull * Wv) * eo;
    if (a < b_end && b < a_end) return fail(SC5_EINVAL, "input and output overlap");
    CUtensorMap m;
    sc5_status st = encode_image_map(&m, d.in_dtype, in, 1, d.H, 3 * d.W, d.in_pitch, hwc_box_cols(d.in_dtype),
                                     p->shape.tile_h + kHalo);
    if (st != SC5_OK) return st;
    alignas(64) unsigned char desc[512];
    if (hwc_desc_size() > sizeof desc) return fail(SC5_ECUDA, "descriptor too large");
    const bool vec = reinterpret_cast<uintptr_t>(out) % (4 * eo) == 0 && d.out_pitch % 4 == 0;
    const float oscale = static_cast<float>(static_cast<double>(out_scale) / in_scale);
    hwc_fill(desc, m, out, d.out_pitch, Hv, Wv, p->shape.tile_h, k, oscale, vec);
    const int64_t ntiles = static_cast<int64_t>((Wv + 127) / 128) * ((Hv + p->shape.tile_h - 1) / p->shape.tile_h);
    cudaError_t e = launch_hwc(d.in_dtype, d.out_dtype, desc, ntiles, d.ctas_per_sm, s);
    return e == cudaSuccess ? SC5_OK : fail_cuda(e, "HWC launch");
}

// One pyramid REDUCE step: validation and plan.
static sc5_status plan_reduce(const sc5_plan_desc &d, sc5_plan *out)
{
    if (d.taps != kTaps || d.border != SC5_BORDER_VALID)
        return fail(SC5_EINVAL, "the REDUCE step is built for width 5 and SC5_BORDER_VALID");
    if (!default_strides(d)) return fail(SC5_EINVAL, "the REDUCE step takes stacked planes (plane strides 0)");
    FusedShape sh;
    if (!reduce_shape(d.in_dtype, d.out_dtype, 0, 0, &sh))
        return fail(SC5_EINVAL, "dtype pair (%d -> %d) not built for the REDUCE step", d.in_dtype, d.out_dtype);
    if ((d.tile_h || d.stages) && !reduce_shape(d.in_dtype, d.out_dtype, d.tile_h ? d.tile_h : sh.tile_h, d.stages, &sh))
        return fail(SC5_EINVAL, "no compiled REDUCE shape with %d input rows per tile and %d stages", d.tile_h,
                    d.stages);
    if (d.tile_w && d.tile_w != sh.tile_w) return fail(SC5_EINVAL, "REDUCE tiles are %d input columns wide", sh.tile_w);
    // the full-resolution VALID output is never stored; check the input side only
    sc5_status st = check_image(d.in_dtype, d.out_dtype, d.border, nullptr, nullptr, d.planes, d.H, d.W,
                                d.in_pitch, d.W - kHalo, 1.f, 1.f, false);
    if (st != SC5_OK) return st;
    const int64_t Wo = (d.W - kHalo + 1) / 2;
    if (d.out_pitch < Wo) return fail(SC5_EINVAL, "REDUCE out_pitch %lld < Wo %lld", (long long)d.out_pitch,
                                      (long long)Wo);
    sc5_plan p = new (std::nothrow) sc5_plan_s;
    if (!p) return fail(SC5_ENOMEM, "host allocation failed");
    p->d = d;
    cudaGetDevice(&p->device);
    p->shape = sh;
    p->ctas_per_sm = d.ctas_per_sm > 0 ? d.ctas_per_sm : 0;
    if (cudaEventCreateWithFlags(&p->ws_done, cudaEventDisableTiming) != cudaSuccess) {
        delete p;
        return fail(SC5_ECUDA, "cudaEventCreate failed");
    }
    *out = p;
    return SC5_OK;
}

static bool is_reduce(const sc5_plan_desc &d) { return d.layout == SC5_LAYOUT_PLANAR && d.algo == SC5_ALGO_REDUCE; }

static sc5_status run_reduce(sc5_plan p, const void *in, void *out, const float *k, float in_scale,
                             float out_scale, cudaStream_t s)
{
    const sc5_plan_desc &d = p->d;
    const int eo = dtype_bytes(d.out_dtype);
    if (!in || !out) return fail(SC5_EINVAL, "null image pointer");
    if (reinterpret_cast<uintptr_t>(in) % 16) return fail(SC5_EINVAL, "input must be 16-byte aligned");
    if (reinterpret_cast<uintptr_t>(out) % eo) return fail(SC5_EINVAL, "output not aligned to its element size");
    if (!(in_scale > 0.f) || !std::isfinite(in_scale) || !(out_scale > 0.f) || !std::isfinite(out_scale))
        return fail(SC5_EINVAL, "scales must be finite and > 0");
    if (!taps_finite(k)) return fail(SC5_EINVAL, "taps must be finite");
    const int Ho = (d.H - kHalo + 1) / 2, Wo = (d.W - kHalo + 1) / 2;
    const int ei = dtype_bytes(d.in_dtype);
    const char *a = static_cast<const char *>(in), *b = static_cast<const char *>(out);
    const char *a_end = a + (static_cast<size_t>(d.planes) * d.H * d.in_pitch) * ei;
    const char *b_end = b + (static_cast<size_t>(d.planes - 1) * Ho * d.out_pitch +
                             static_cast<size_t>(Ho - 1) * d.out_pitch + Wo) * eo;
    if (a < b_end && b < a_end) return fail(SC5_EINVAL, "input and output overlap");
    ImgDesc desc;
    std::memset(&desc, 0, sizeof desc);
    sc5_status st = encode_image_map(&desc.tmap, d.in_dtype, in, d.planes, d.H, d.W, d.in_pitch,
                                     box_w_for(d.in_dtype, p->shape.tile_w, kTaps), p->shape.tile_h + kHalo);
    if (st != SC5_OK) return st;
    desc.out = out;
    desc.out_pitch = d.out_pitch;
    desc.out_plane = static_cast<int64_t>(Ho) * d.out_pitch;
    desc.Hv = Ho;
    desc.Wv = Wo;
    desc.tiles_x = (Wo + p->shape.tile_w / 2 - 1) / (p->shape.tile_w / 2);
    desc.tiles_y = (Ho + p->shape.tile_h / 2 - 1) / (p->shape.tile_h / 2);
    for (int i = 0; i < kTaps; ++i) desc.k[i] = k[i];
    desc.oscale = static_cast<float>(static_cast<double>(out_scale) / static_cast<double>(in_scale));
    const int64_t ntiles = static_cast<int64_t>(d.planes) * desc.tiles_x * desc.tiles_y;
    cudaError_t e = launch_reduce(d.in_dtype, d.out_dtype, p->shape, desc, ntiles, p->ctas_per_sm, s);
    return e == cudaSuccess ? SC5_OK : fail_cuda(e, "REDUCE launch");
}

extern "C" sc5_status sepconv5_plan(const sc5_plan_desc *desc, sc5_plan *out)
{
    clear_error();
    if (!desc || !out) return fail(SC5_EINVAL, "null argument");
    *out = nullptr;
    sc5_plan_desc d = *desc;
    if (d.taps == 0) d.taps = kTaps;
    if (d.layout == SC5_LAYOUT_HWC) return plan_hwc(d, out);
    if (d.layout != SC5_LAYOUT_PLANAR) return fail(SC5_EINVAL, "unknown layout %d", d.layout);
    if (d.algo == SC5_ALGO_REDUCE) return plan_reduce(d, out);
    if (d.algo != SC5_ALGO_FUSED && d.algo != SC5_ALGO_TWO_PASS && d.algo != SC5_ALGO_DIRECT)
        return fail(SC5_EINVAL, "unknown algo %d", d.algo);
    if (d.taps != 3 && d.taps != 5 && d.taps != 7 && d.taps != 9)
        return fail(SC5_EINVAL, "taps must be 3, 5, 7 or 9 (got %d)", d.taps);
    if (d.taps != kTaps && d.algo != SC5_ALGO_FUSED)
        return fail(SC5_EINVAL, "widths other than 5 are built for the fused form only");
    sc5_status st = check_image(d.in_dtype, d.out_dtype, d.border, nullptr, nullptr, d.planes, d.H, d.W,
                                d.in_pitch, d.out_pitch, 1.f, 1.f, false, d.in_plane_stride, d.out_plane_stride,
                                d.taps);
    if (st != SC5_OK) return st;
    if (!pair_supported(d.in_dtype, d.out_dtype))
        return fail(SC5_EINVAL, "dtype pair (%d -> %d) not built: the output must be the input format or FP32",
                    d.in_dtype, d.out_dtype);
    sc5_plan p = new (std::nothrow) sc5_plan_s;
    if (!p) return fail(SC5_ENOMEM, "host allocation failed");
    p->d = d;
    cudaGetDevice(&p->device);
    const bool direct = d.algo == SC5_ALGO_DIRECT;
    st = choose_shape(d.in_dtype, d.out_dtype, d.H, d.W, &d, &p->shape_idx, &p->ctas_per_sm, direct, d.taps);
    if (st != SC5_OK) {
        delete p;
        return st;
    }
    fused_shape(d.in_dtype, d.out_dtype, p->shape_idx, &p->shape, direct, d.taps);
    if (d.algo == SC5_ALGO_TWO_PASS) {
        p->t_pitch = (static_cast<int64_t>(d.W - kHalo) + 3) / 4 * 4;
        const size_t bytes = static_cast<size_t>(d.planes) * d.H * p->t_pitch * sizeof(float);
        cudaError_t e = cudaMalloc(&p->T, bytes);
        if (e != cudaSuccess) {
            delete p;
            return fail_cuda(e, "cudaMalloc of the two-pass intermediate");
        }
    }
    if (cudaEventCreateWithFlags(&p->ws_done, cudaEventDisableTiming) != cudaSuccess) {
        cudaFree(p->T);
        delete p;
        return fail(SC5_ECUDA, "cudaEventCreate failed");
    }
    *out = p;
    return SC5_OK;
}

extern "C" sc5_status sepconv5_plan_info(sc5_plan p, int32_t *tile_h, int32_t *tile_w, int32_t *stages,
                                         int32_t *ctas_per_sm)
{
    clear_error();
    if (!p) return fail(SC5_EINVAL, "null plan");
    if (tile_h) *tile_h = p->shape.tile_h;
    if (tile_w) *tile_w = p->shape.tile_w;
    if (stages) *stages = p->shape.stages;
    if (ctas_per_sm) *ctas_per_sm = p->ctas_per_sm;
    return SC5_OK;
}

// ------------------------------------------------------------------ pyramids

struct sc5_pyramid_s {
    sc5_pyramid_desc d{};
    std::vector<sc5_plan> plans;       // step l reduces level l to level l+1
    std::vector<int32_t> h, w;         // level sizes, 0..levels
    std::vector<int64_t> pitch;        // level pitches (elements of their format)
    cudaGraph_t graph = nullptr;       // sepconv5_pyramid_capture
    cudaGraphExec_t exec = nullptr;
};

extern "C" sc5_status sepconv5_pyramid_destroy(sc5_pyramid pyr);

extern "C" sc5_status sepconv5_pyramid_create(const sc5_pyramid_desc *desc, sc5_pyramid *out)
{
    clear_error();
    if (!desc || !out) return fail(SC5_EINVAL, "null argument");
    *out = nullptr;
    const sc5_pyramid_desc &d = *desc;
    if (d.levels < 1 || d.levels > 30) return fail(SC5_EINVAL, "levels must be 1..30 (got %d)", d.levels);
    if (d.out_dtype != d.in_dtype && d.out_dtype != SC5_F32)
        return fail(SC5_EINVAL, "pyramid levels are stored in the input's format or FP32");
    std::unique_ptr<sc5_pyramid_s> p(new (std::nothrow) sc5_pyramid_s);
    if (!p) return fail(SC5_ENOMEM, "host allocation failed");
    p->d = d;
    p->h.push_back(d.H);
    p->w.push_back(d.W);
    p->pitch.push_back(d.in_pitch);
    const int eo = dtype_bytes(d.out_dtype);
    if (!eo) return fail(SC5_EINVAL, "unknown dtype %d", d.out_dtype);
    for (int l = 0; l < d.levels; ++l) {
        const int H = p->h.back(), W = p->w.back();
        if (H < 5 || W < 5) {
            sepconv5_pyramid_destroy(p.release());
            return fail(SC5_EINVAL, "level %d is %d x %d: too small for another step", l, H, W);
        }
        const int Ho = (H - kHalo + 1) / 2, Wo = (W - kHalo + 1) / 2;
        const int64_t op = (static_cast<int64_t>(Wo) * eo + 15) / 16 * 16 / eo;
        sc5_plan_desc pd{};
        pd.planes = d.planes;
        pd.H = H;
        pd.W = W;
        pd.in_pitch = p->pitch.back();
        pd.out_pitch = op;
        pd.in_dtype = l == 0 ? d.in_dtype : d.out_dtype;
        pd.out_dtype = d.out_dtype;
        pd.border = SC5_BORDER_VALID;
        pd.algo = SC5_ALGO_REDUCE;
        pd.taps = kTaps;
        sc5_plan plan = nullptr;
        const sc5_status st = sepconv5_plan(&pd, &plan);
        if (st != SC5_OK) {
            const std::string msg = sepconv5_last_error();  // cleanup clears it
            sepconv5_pyramid_destroy(p.release());
            return fail(st, "level %d: %s", l, msg.c_str());
        }
        p->plans.push_back(plan);
        p->h.push_back(Ho);
        p->w.push_back(Wo);
        p->pitch.push_back(op);
    }
    *out = p.release();
    return SC5_OK;
}

extern "C" sc5_status sepconv5_pyramid_level(sc5_pyramid pyr, int32_t level, int32_t *H, int32_t *W,
                                             int64_t *pitch)
{
    clear_error();
    if (!pyr) return fail(SC5_EINVAL, "null pyramid");
    if (level < 0 || level > pyr->d.levels) return fail(SC5_EINVAL, "level %d outside 0..%d", level, pyr->d.levels);
    if (H) *H = pyr->h[level];
    if (W) *W = pyr->w[level];
    if (pitch) *pitch = pyr->pitch[level];
    return SC5_OK;
}

extern "C" sc5_status sepconv5_pyramid_run(sc5_pyramid pyr, const void *in, void *const *levels, const float k[5],
                                           float in_scale, float out_scale, void *stream)
{
    clear_error();
    if (!pyr || !in || !levels || !k) return fail(SC5_EINVAL, "null argument");
    const void *src = in;
    for (int l = 0; l < pyr->d.levels; ++l) {
        if (!levels[l]) return fail(SC5_EINVAL, "levels[%d] is null", l);
        const float is = l == 0 ? in_scale : out_scale;
        const sc5_status st = sepconv5_run(pyr->plans[l], src, levels[l], k, is, out_scale, stream);
        if (st != SC5_OK) return st;
        src = levels[l];
    }
    return SC5_OK;
}

extern "C" sc5_status sepconv5_pyramid_capture(sc5_pyramid pyr, const void *in, void *const *levels,
                                               const float k[5], float in_scale, float out_scale)
{
    clear_error();
    if (!pyr || !in || !levels || !k) return fail(SC5_EINVAL, "null argument");
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return fail_cuda(e, "capture stream");
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    sc5_status st = SC5_OK;
    cudaGraph_t g = nullptr;
    if (e == cudaSuccess) {
        st = sepconv5_pyramid_run(pyr, in, levels, k, in_scale, out_scale, cs);
        const cudaError_t ee = cudaStreamEndCapture(cs, &g);
        if (st == SC5_OK && ee != cudaSuccess) e = ee;
    }
    cudaGraphExec_t x = nullptr;
    if (e == cudaSuccess && st == SC5_OK) e = cudaGraphInstantiate(&x, g, 0);
    cudaStreamDestroy(cs);
    if (st != SC5_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return st != SC5_OK ? st : fail_cuda(e, "pyramid graph capture");
    }
    if (pyr->exec) cudaGraphExecDestroy(pyr->exec);
    if (pyr->graph) cudaGraphDestroy(pyr->graph);
    pyr->graph = g;
    pyr->exec = x;
    return SC5_OK;
}

extern "C" sc5_status sepconv5_pyramid_replay(sc5_pyramid pyr, void *stream)
{
    clear_error();
    if (!pyr) return fail(SC5_EINVAL, "null pyramid");
    if (!pyr->exec) return fail(SC5_EINVAL, "nothing captured: call sepconv5_pyramid_capture first");
    const cudaError_t e = cudaGraphLaunch(pyr->exec, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail_cuda(e, "pyramid graph launch");
    note_launches(pyr->d.levels);
    return SC5_OK;
}

extern "C" sc5_status sepconv5_pyramid_destroy(sc5_pyramid pyr)
{
    clear_error();
    if (!pyr) return SC5_OK;
    if (pyr->exec) cudaGraphExecDestroy(pyr->exec);
    if (pyr->graph) cudaGraphDestroy(pyr->graph);
    for (sc5_plan p : pyr->plans) sepconv5_plan_destroy(p);
    delete pyr;
    return SC5_OK;
}

extern "C" sc5_status sepconv5_plan_destroy(sc5_plan p)
{
    clear_error();
    if (!p) return SC5_OK;
    if (p->ws_pending) cudaEventSynchronize(p->ws_done);
    if (p->s_in) cudaStreamSynchronize(p->s_in);
    if (p->s_out) cudaStreamSynchronize(p->s_out);
    cudaFree(p->T);
    cudaFree(p->ws_dev);
    cudaFreeHost(p->ws_host);
    cudaEventDestroy(p->ws_done);
    cudaFree(p->stage_in);
    cudaFree(p->stage_out);
    cudaFree(p->scratch);
    if (p->s_in) cudaStreamDestroy(p->s_in);
    if (p->s_out) cudaStreamDestroy(p->s_out);
    for (cudaEvent_t e : p->ev) cudaEventDestroy(e);
    delete p;
    return SC5_OK;
}

static sc5_status run_two_pass(sc5_plan p, const void *in, void *out, const float *k, float in_scale,
                               float out_scale, cudaStream_t st)
{
    const sc5_plan_desc &d = p->d;
    cudaError_t e = launch_hpass(d.in_dtype, in, d.planes, d.H, d.W, d.in_pitch, p->T, p->t_pitch, k, st,
                                 in_plane_of(d));
    if (e != cudaSuccess) return fail_cuda(e, "hpass launch");
    const int eo = dtype_bytes(d.out_dtype);
    char *ob = static_cast<char *>(out);
    if (d.border == SC5_BORDER_KEEP) ob += (2 * d.out_pitch + 2) * eo;
    const int64_t op = out_plane_of(d);
    const bool vec = reinterpret_cast<uintptr_t>(ob) % (4 * eo) == 0 && d.out_pitch % 4 == 0 && op % 4 == 0;
    const float oscale = static_cast<float>(static_cast<double>(out_scale) / in_scale);
    e = launch_vpass(d.out_dtype, p->T, d.planes, d.H, d.W - kHalo, p->t_pitch, ob, d.out_pitch, op, k, oscale,
                     vec, st);
    if (e != cudaSuccess) return fail_cuda(e, "vpass launch");
    return SC5_OK;
}

static sc5_status run_frame(const sc5_plan_desc &d, const void *in, void *out, float in_scale,
                            float out_scale, cudaStream_t st)
{
    if (d.border != SC5_BORDER_KEEP) return SC5_OK;
    const float ratio = static_cast<float>(static_cast<double>(out_scale) / in_scale);
    cudaError_t e = launch_keep_frame(d.in_dtype, d.out_dtype, in, d.planes, d.H, d.W, d.in_pitch, out,
                                      d.out_pitch, ratio, st, in_plane_of(d), out_plane_of(d), (taps_of(d) - 1) / 2);
    return e == cudaSuccess ? SC5_OK : fail_cuda(e, "frame launch");
}

// One launch of the fused (separable) or direct single-pass kernel over the image.
static sc5_status run_single_pass(sc5_plan p, const void *in, void *out, const float *k, const float *K,
                                  float in_scale, float out_scale, cudaStream_t s)
{
    const sc5_plan_desc &d = p->d;
    ImgDesc desc;
    sc5_status st = fill_desc(&desc, d.in_dtype, d.out_dtype, d.border, p->shape, in, out, d.planes, d.H, d.W,
                              d.in_pitch, d.out_pitch, k, in_scale, out_scale, K, d.in_plane_stride,
                              d.out_plane_stride, taps_of(d));
    if (desc.out_plane % 4) desc.vec = 0;
    if (st != SC5_OK) return st;
    const int64_t ntiles = static_cast<int64_t>(d.planes) * desc.tiles_x * desc.tiles_y;
    const int64_t cap = static_cast<int64_t>(num_sms()) * p->ctas_per_sm;
    const int grid = static_cast<int>(std::max<int64_t>(1, std::min(ntiles, cap)));
    cudaError_t e = launch_fused_single(d.in_dtype, d.out_dtype, p->shape_idx, desc, ntiles, grid, s,
                                        d.algo == SC5_ALGO_DIRECT, taps_of(d));
    return e == cudaSuccess ? SC5_OK : fail_cuda(e, "single-pass launch");
}

extern "C" sc5_status sepconv5_run(sc5_plan p, const void *in, void *out, const float k[5],
                                   float in_scale, float out_scale, void *stream)
{
    clear_error();
    if (!p || !k) return fail(SC5_EINVAL, "null argument");
    const sc5_plan_desc &d = p->d;
    if (d.layout == SC5_LAYOUT_HWC) return run_hwc(p, in, out, k, in_scale, out_scale, static_cast<cudaStream_t>(stream));
    if (is_reduce(d)) return run_reduce(p, in, out, k, in_scale, out_scale, static_cast<cudaStream_t>(stream));
    sc5_status st = check_image(d.in_dtype, d.out_dtype, d.border, in, out, d.planes, d.H, d.W, d.in_pitch,
                                d.out_pitch, in_scale, out_scale, true, d.in_plane_stride, d.out_plane_stride,
                                taps_of(d));
    if (st != SC5_OK) return st;
    for (int t = 0; t < taps_of(d); ++t)
        if (!std::isfinite(k[t])) return fail(SC5_EINVAL, "taps must be finite");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (d.algo == SC5_ALGO_TWO_PASS) {
        st = run_two_pass(p, in, out, k, in_scale, out_scale, s);
    } else {
        st = run_single_pass(p, in, out, k, nullptr, in_scale, out_scale, s);
    }
    if (st != SC5_OK) return st;
    return run_frame(d, in, out, in_scale, out_scale, s);
}

extern "C" sc5_status sepconv5_run_K(sc5_plan p, const void *in, void *out, const float K[25], float in_scale,
                                     float out_scale, void *stream)
{
    clear_error();
    if (!p || !K) return fail(SC5_EINVAL, "null argument");
    const sc5_plan_desc &d = p->d;
    if (d.algo != SC5_ALGO_DIRECT || d.layout != SC5_LAYOUT_PLANAR)
        return fail(SC5_EINVAL, "sepconv5_run_K needs a planar plan with algo SC5_ALGO_DIRECT");
    sc5_status st = check_image(d.in_dtype, d.out_dtype, d.border, in, out, d.planes, d.H, d.W, d.in_pitch,
                                d.out_pitch, in_scale, out_scale, true, d.in_plane_stride, d.out_plane_stride);
    if (st != SC5_OK) return st;
    for (int i = 0; i < kTaps * kTaps; ++i)
        if (!std::isfinite(K[i])) return fail(SC5_EINVAL, "K must be finite");
    const float zero_k[kTaps] = {0.f, 0.f, 0.f, 0.f, 0.f};
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    st = run_single_pass(p, in, out, zero_k, K, in_scale, out_scale, s);
    if (st != SC5_OK) return st;
    return run_frame(d, in, out, in_scale, out_scale, s);
}

extern "C" sc5_status sepconv5_run_inplace(sc5_plan p, void *img, const float k[5], float scale, void *stream)
{
    clear_error();
    if (!p || !img || !k) return fail(SC5_EINVAL, "null argument");
    const sc5_plan_desc &d = p->d;
    if (is_reduce(d)) return fail(SC5_EINVAL, "a REDUCE plan runs through sepconv5_run only");
    if (d.in_dtype != d.out_dtype || d.border != SC5_BORDER_KEEP || d.out_pitch != d.in_pitch)
        return fail(SC5_EINVAL, "in-place needs in_dtype == out_dtype, border KEEP and out_pitch == in_pitch");
    if (!default_strides(d)) return fail(SC5_EINVAL, "in-place takes stacked planes (plane strides 0)");
    if (taps_of(d) != kTaps || d.layout != SC5_LAYOUT_PLANAR)
        return fail(SC5_EINVAL, "in-place is built for planar images of width 5");
    if (reinterpret_cast<uintptr_t>(img) % 16) return fail(SC5_EINVAL, "image must be 16-byte aligned");
    if (!(scale > 0.f) || !std::isfinite(scale)) return fail(SC5_EINVAL, "scale must be finite and > 0");
    if (!taps_finite(k)) return fail(SC5_EINVAL, "taps must be finite");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int es = dtype_bytes(d.in_dtype);
    const int Hv = d.H - kHalo, Wv = d.W - kHalo;
    char *base = static_cast<char *>(img);
    char *interior = base + (2 * d.in_pitch + 2) * es;
    const int64_t plane = static_cast<int64_t>(d.H) * d.in_pitch;
    if (d.algo == SC5_ALGO_TWO_PASS) {
        cudaError_t e = launch_hpass(d.in_dtype, img, d.planes, d.H, d.W, d.in_pitch, p->T, p->t_pitch, k, s);
        if (e != cudaSuccess) return fail_cuda(e, "hpass launch");
        e = launch_vpass(d.out_dtype, p->T, d.planes, d.H, Wv, p->t_pitch, interior, d.in_pitch, plane, k, 1.f,
                         false, s);
        return e == cudaSuccess ? SC5_OK : fail_cuda(e, "vpass launch");
    }
    // single pass into the scratch (VALID layout, pitch rounded to 16 bytes), then copy back
    const int64_t sp = (static_cast<int64_t>(Wv) * es + 15) / 16 * 16 / es;
    if (!p->scratch) {
        cudaError_t e = cudaMalloc(&p->scratch, static_cast<size_t>(d.planes) * Hv * sp * es);
        if (e != cudaSuccess) return fail_cuda(e, "cudaMalloc of the copy-back scratch");
    }
    sc5_plan_desc vd = d;
    vd.border = SC5_BORDER_VALID;
    vd.out_pitch = sp;
    sc5_plan_s tmp = *p;
    tmp.d = vd;
    sc5_status st = run_single_pass(&tmp, img, p->scratch, k, nullptr, scale, scale, s);
    if (st != SC5_OK) return st;
    cudaError_t e = launch_copy_interior(d.in_dtype, p->scratch, sp, static_cast<int64_t>(Hv) * sp, interior,
                                         d.in_pitch, plane, d.planes, Hv, Wv, s);
    return e == cudaSuccess ? SC5_OK : fail_cuda(e, "copy-back");
}

extern "C" sc5_status sepconv5_run_host(sc5_plan p, const void *host_in, void *host_out, const float k[5],
                                        float in_scale, float out_scale, void *stream)
{
    clear_error();
    if (!p || !host_in || !host_out || !k) return fail(SC5_EINVAL, "null argument");
    const sc5_plan_desc &d = p->d;
    if (is_reduce(d)) return fail(SC5_EINVAL, "a REDUCE plan runs through sepconv5_run only");
    if (!default_strides(d)) return fail(SC5_EINVAL, "the offload call takes stacked planes (plane strides 0)");
    if (taps_of(d) != kTaps || d.layout != SC5_LAYOUT_PLANAR)
        return fail(SC5_EINVAL, "the offload call is built for planar images of width 5");
    sc5_status st = check_image(d.in_dtype, d.out_dtype, d.border, nullptr, nullptr, d.planes, d.H, d.W, d.in_pitch,
                                d.out_pitch, in_scale, out_scale, false);
    if (st != SC5_OK) return st;
    if (!taps_finite(k)) return fail(SC5_EINVAL, "taps must be finite");
    const int ei = dtype_bytes(d.in_dtype), eo = dtype_bytes(d.out_dtype);
    const int Hv = d.H - kHalo;
    const int64_t hout = d.border == SC5_BORDER_KEEP ? d.H : Hv;
    const size_t in_row = static_cast<size_t>(d.in_pitch) * ei, out_row = static_cast<size_t>(d.out_pitch) * eo;
    const size_t in_bytes = in_row * d.H * d.planes, out_bytes = out_row * hout * d.planes;
    cudaError_t e = cudaSuccess;
    if (!p->stage_in) e = cudaMalloc(&p->stage_in, in_bytes);
    if (e == cudaSuccess && !p->stage_out) e = cudaMalloc(&p->stage_out, out_bytes);
    if (e == cudaSuccess && !p->s_in) e = cudaStreamCreateWithFlags(&p->s_in, cudaStreamNonBlocking);
    if (e == cudaSuccess && !p->s_out) e = cudaStreamCreateWithFlags(&p->s_out, cudaStreamNonBlocking);
    if (e != cudaSuccess) return fail_cuda(e, "offload staging");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char *din = static_cast<char *>(p->stage_in), *dout = static_cast<char *>(p->stage_out);
    const char *hin = static_cast<const char *>(host_in);
    char *hout_c = static_cast<char *>(host_out);

    if (d.algo != SC5_ALGO_FUSED || d.border != SC5_BORDER_VALID) {
        // whole image: copy in, run, copy out
        e = cudaMemcpyAsync(din, hin, in_bytes, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return fail_cuda(e, "copy to device");
        st = sepconv5_run(p, din, dout, k, in_scale, out_scale, stream);
        if (st != SC5_OK) return st;
        // the output rows' valid values only: the caller's row padding stays as it was
        e = cudaMemcpy2DAsync(hout_c, out_row, dout, out_row, static_cast<size_t>(d.border == SC5_BORDER_KEEP ? d.W : d.W - kHalo) * eo,
                              static_cast<size_t>(d.planes) * hout, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        return e == cudaSuccess ? SC5_OK : fail_cuda(e, "copy to host");
    }

    // Output bands of R rows (a multiple of the tile height, about 8 per plane).
    // The image's first and last band are split into bands of about R/4 rows, so
    // that the first kernel waits for a small copy and the last copy back is
    // small.  Each band's input rows are copied just ahead of it: only the rows
    // (band rows plus the 4-row halo) not yet on the device.
    const int th = p->shape.tile_h;
    const int R = std::max(th, (((Hv + 7) / 8) + th - 1) / th * th);
    const int Rs = std::max(th, ((R + 3) / 4 + th - 1) / th * th);
    const int nb = (Hv + R - 1) / R;
    const size_t need_ev = static_cast<size_t>(d.planes) * 2 * (nb + 2 * ((R + Rs - 1) / Rs));
    while (p->ev.size() < need_ev) {
        cudaEvent_t ev;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) return fail_cuda(e, "event create");
        p->ev.push_back(ev);
    }
    size_t evi = 0;
    const int64_t cap = static_cast<int64_t>(num_sms()) * p->ctas_per_sm;
    std::vector<std::pair<int, int>> bands;  // output rows [first, second) of one plane
    for (int pl = 0; pl < d.planes; ++pl) {
        bands.clear();
        for (int b = 0; b < nb; ++b) {
            const int y0 = b * R, y1 = std::min(Hv, y0 + R);
            const bool split = (pl == 0 && b == 0) || (pl == d.planes - 1 && b == nb - 1);
            for (int y = y0; y < y1; y += split ? Rs : R) bands.emplace_back(y, std::min(y1, y + (split ? Rs : R)));
        }
        const size_t in_plane = in_row * d.H * pl, out_plane = out_row * Hv * pl;
        int loaded = 0;  // input rows of this plane already copied
        cudaEvent_t in_ev = nullptr;
        for (const auto &band : bands) {
            const int y0 = band.first, rows_out = band.second - band.first;
            const int need = std::min(d.H, band.second + kHalo);
            if (need > loaded) {
                const size_t off = in_plane + in_row * loaded;
                e = cudaMemcpyAsync(din + off, hin + off, in_row * (need - loaded), cudaMemcpyHostToDevice, p->s_in);
                if (e != cudaSuccess) return fail_cuda(e, "band copy to device");
                in_ev = p->ev[evi++];
                cudaEventRecord(in_ev, p->s_in);
                loaded = need;
            }
            cudaStreamWaitEvent(s, in_ev, 0);
            ImgDesc desc;
            st = fill_desc(&desc, d.in_dtype, d.out_dtype, d.border, p->shape, din + in_plane + in_row * y0,
                           dout + out_plane + out_row * y0, 1, rows_out + kHalo, d.W, d.in_pitch, d.out_pitch, k,
                           in_scale, out_scale);
            if (st != SC5_OK) return st;
            const int64_t ntiles = static_cast<int64_t>(desc.tiles_x) * desc.tiles_y;
            const int grid = static_cast<int>(std::max<int64_t>(1, std::min(ntiles, cap)));
            e = launch_fused_single(d.in_dtype, d.out_dtype, p->shape_idx, desc, ntiles, grid, s);
            if (e != cudaSuccess) return fail_cuda(e, "band launch");
            cudaEvent_t kev = p->ev[evi++];
            cudaEventRecord(kev, s);
            cudaStreamWaitEvent(p->s_out, kev, 0);
            const size_t off = out_plane + out_row * y0;
            e = cudaMemcpy2DAsync(hout_c + off, out_row, dout + off, out_row, static_cast<size_t>(d.W - kHalo) * eo,
                                  rows_out, cudaMemcpyDeviceToHost, p->s_out);
            if (e != cudaSuccess) return fail_cuda(e, "band copy to host");
        }
    }
    e = cudaStreamSynchronize(p->s_out);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? SC5_OK : fail_cuda(e, "offload completion");
}

extern "C" sc5_status sepconv5_hpass(sc5_plan p, const void *in, float *T, int64_t t_pitch,
                                     const float k[5], void *stream)
{
    clear_error();
    if (!p || !in || !T || !k) return fail(SC5_EINVAL, "null argument");
    const sc5_plan_desc &d = p->d;
    if (is_reduce(d)) return fail(SC5_EINVAL, "a REDUCE plan runs through sepconv5_run only");
    if (d.layout != SC5_LAYOUT_PLANAR || taps_of(d) != kTaps)
        return fail(SC5_EINVAL, "the separate passes take planar images of width 5");
    if (t_pitch < d.W - kHalo || t_pitch % 4 || reinterpret_cast<uintptr_t>(T) % 16)
        return fail(SC5_EINVAL, "T needs t_pitch >= W-4, a multiple of 4, and 16-byte alignment");
    if (reinterpret_cast<uintptr_t>(in) % 16) return fail(SC5_EINVAL, "input must be 16-byte aligned");
    if (!taps_finite(k)) return fail(SC5_EINVAL, "taps must be finite");
    cudaError_t e = launch_hpass(d.in_dtype, in, d.planes, d.H, d.W, d.in_pitch, T, t_pitch, k,
                                 static_cast<cudaStream_t>(stream), in_plane_of(d));
    return e == cudaSuccess ? SC5_OK : fail_cuda(e, "hpass launch");
}

extern "C" sc5_status sepconv5_vpass(sc5_plan p, const float *T, int64_t t_pitch, void *out,
                                     const float k[5], float in_scale, float out_scale, void *stream)
{
    clear_error();
    if (!p || !out || !T || !k) return fail(SC5_EINVAL, "null argument");
    const sc5_plan_desc &d = p->d;
    if (is_reduce(d)) return fail(SC5_EINVAL, "a REDUCE plan runs through sepconv5_run only");
    if (d.layout != SC5_LAYOUT_PLANAR || taps_of(d) != kTaps)
        return fail(SC5_EINVAL, "the separate passes take planar images of width 5");
    if (t_pitch < d.W - kHalo || t_pitch % 4 || reinterpret_cast<uintptr_t>(T) % 16)
        return fail(SC5_EINVAL, "T needs t_pitch >= W-4, a multiple of 4, and 16-byte alignment");
    if (!(in_scale > 0.f) || !(out_scale > 0.f) || !std::isfinite(in_scale) || !std::isfinite(out_scale))
        return fail(SC5_EINVAL, "scales must be finite and > 0");
    if (!taps_finite(k)) return fail(SC5_EINVAL, "taps must be finite");
    const int eo = dtype_bytes(d.out_dtype);
    char *ob = static_cast<char *>(out);
    if (d.border == SC5_BORDER_KEEP) ob += (2 * d.out_pitch + 2) * eo;
    const int64_t op = out_plane_of(d);
    const bool vec = reinterpret_cast<uintptr_t>(ob) % (4 * eo) == 0 && d.out_pitch % 4 == 0 && op % 4 == 0;
    const float oscale = static_cast<float>(static_cast<double>(out_scale) / in_scale);
    cudaError_t e = launch_vpass(d.out_dtype, T, d.planes, d.H, d.W - kHalo, t_pitch, ob, d.out_pitch, op, k,
                                 oscale, vec, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? SC5_OK : fail_cuda(e, "vpass launch");
}

extern "C" sc5_status sepconv5_device_status(void *stream, int32_t *code)
{
    clear_error();
    if (!code) return fail(SC5_EINVAL, "null argument");
    cudaError_t e = read_and_clear_device_status(static_cast<cudaStream_t>(stream), code);
    if (e != cudaSuccess) return fail_cuda(e, "reading the device status word");
    return *code ? fail(SC5_EDEVICE, "a kernel reported device error %d", *code) : SC5_OK;
}

// ------------------------------------------------------------------ batches

namespace sc5 {

// Host-side build of a batch: one ImgDesc per image, tile records in image,
// plane, row, column order.  Returns the bytes of the device image
// (descriptors then tiles) in *blob.
sc5_status build_batch(const sc5_plan_desc &pd, int n, const sc5_image *imgs, const FusedShape &sh,
                       std::vector<unsigned char> *blob, int64_t *ntiles, size_t *tiles_off)
{
    if (n < 1 || !imgs) return fail(SC5_EINVAL, "empty batch");
    std::vector<ImgDesc> descs(n);
    int64_t nt = 0;
    for (int i = 0; i < n; ++i) {
        const sc5_image &im = imgs[i];
        sc5_status st = check_image(pd.in_dtype, pd.out_dtype, pd.border, im.in, im.out, pd.planes, im.H, im.W,
                                    im.in_pitch, im.out_pitch, im.in_scale, im.out_scale, true);
        if (st != SC5_OK) return fail(st, "image %d: %s", i, sepconv5_last_error());
        if (!taps_finite(im.k)) return fail(SC5_EINVAL, "image %d: taps must be finite", i);
        st = fill_desc(&descs[i], pd.in_dtype, pd.out_dtype, pd.border, sh, im.in, im.out, pd.planes, im.H,
                       im.W, im.in_pitch, im.out_pitch, im.k, im.in_scale, im.out_scale);
        if (st != SC5_OK) return st;
        nt += static_cast<int64_t>(pd.planes) * descs[i].tiles_x * descs[i].tiles_y;
    }
    const size_t dbytes = sizeof(ImgDesc) * n;
    const size_t toff = (dbytes + 255) / 256 * 256;
    blob->assign(toff + sizeof(TileRec) * nt, 0);
    std::memcpy(blob->data(), descs.data(), dbytes);
    TileRec *t = reinterpret_cast<TileRec *>(blob->data() + toff);
    for (int i = 0; i < n; ++i)
        for (int p = 0; p < pd.planes; ++p)
            for (int ty = 0; ty < descs[i].tiles_y; ++ty)
                for (int tx = 0; tx < descs[i].tiles_x; ++tx) *t++ = TileRec{i, p, ty, tx};
    *ntiles = nt;
    *tiles_off = toff;
    return SC5_OK;
}

sc5_status choose_batch_shape(int in_dtype, int out_dtype, int n, const sc5_image *imgs, int *idx, int *ctas)
{
    if (n < 1 || !imgs) return fail(SC5_EINVAL, "empty batch");
    tune_from_environment(in_dtype, out_dtype);
    double by_class[64] = {};
    for (int i = 0; i < n; ++i) {
        const double px = static_cast<double>(imgs[i].H) * imgs[i].W;
        const int c = std::min(63, std::max(0, static_cast<int>(std::log2(std::max(1.0, px)))));
        by_class[c] += px;
    }
    const int best = static_cast<int>(std::max_element(by_class, by_class + 64) - by_class);
    const int side = 1 << (best / 2);
    const int H = side, W = (best % 2) ? side * 2 : side;
    *idx = -1;
    return choose_shape(in_dtype, out_dtype, H, W, nullptr, idx, ctas, false, kTaps, true);
}

// Shape for a batch: the plan's override, else the tuned choice for the size
// class holding the most pixels.
sc5_status batch_shape(sc5_plan p, int n, const sc5_image *imgs, int *idx, int *ctas)
{
    const sc5_plan_desc &d = p->d;
    if (d.tile_h || d.tile_w || d.stages) {
        *idx = p->shape_idx;
        *ctas = p->ctas_per_sm;
        return SC5_OK;
    }
    sc5_status st = choose_batch_shape(d.in_dtype, d.out_dtype, n, imgs, idx, ctas);
    if (st == SC5_OK && d.ctas_per_sm > 0) *ctas = std::min(*ctas, d.ctas_per_sm);
    return st;
}

}  // namespace sc5

extern "C" sc5_status sepconv5_run_batch(sc5_plan p, int32_t n, const sc5_image *imgs, void *stream)
{
    clear_error();
    if (!p) return fail(SC5_EINVAL, "null plan");
    if (p->d.algo != SC5_ALGO_FUSED) return fail(SC5_EINVAL, "batches run the fused form only");
    if (taps_of(p->d) != kTaps || p->d.layout != SC5_LAYOUT_PLANAR)
        return fail(SC5_EINVAL, "batches are built for planar images of width 5");
    int idx = 0, ctas = 1;
    sc5_status st = batch_shape(p, n, imgs, &idx, &ctas);
    if (st != SC5_OK) return st;
    FusedShape sh;
    fused_shape(p->d.in_dtype, p->d.out_dtype, idx, &sh);
    std::vector<unsigned char> blob;
    int64_t ntiles = 0;
    size_t toff = 0;
    st = build_batch(p->d, n, imgs, sh, &blob, &ntiles, &toff);
    if (st != SC5_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the pinned staging buffer may still feed an earlier upload
    if (p->ws_pending) {
        cudaEventSynchronize(p->ws_done);
        p->ws_pending = false;
    }
    if (blob.size() > p->ws_cap) {
        cudaStreamSynchronize(s);
        cudaFree(p->ws_dev);
        p->ws_dev = nullptr;
        p->ws_cap = 0;
        cudaError_t e = cudaMalloc(&p->ws_dev, blob.size());
        if (e != cudaSuccess) return fail_cuda(e, "cudaMalloc of the batch work-list");
        p->ws_cap = blob.size();
    }
    if (blob.size() > p->ws_host_cap) {
        cudaFreeHost(p->ws_host);
        p->ws_host = nullptr;
        p->ws_host_cap = 0;
        cudaError_t e = cudaMallocHost(&p->ws_host, blob.size());
        if (e != cudaSuccess) return fail_cuda(e, "cudaMallocHost of the batch staging buffer");
        p->ws_host_cap = blob.size();
    }
    std::memcpy(p->ws_host, blob.data(), blob.size());
    cudaError_t e = cudaMemcpyAsync(p->ws_dev, p->ws_host, blob.size(), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail_cuda(e, "work-list upload");
    cudaEventRecord(p->ws_done, s);
    p->ws_pending = true;
    const int64_t cap = static_cast<int64_t>(num_sms()) * ctas;
    const int grid = static_cast<int>(std::max<int64_t>(1, std::min(ntiles, cap)));
    e = launch_fused_batch(p->d.in_dtype, p->d.out_dtype, idx, reinterpret_cast<const ImgDesc *>(p->ws_dev),
                           reinterpret_cast<const TileRec *>(p->ws_dev + toff), ntiles, grid, s);
    if (e != cudaSuccess) return fail_cuda(e, "batch launch");
    if (p->d.border == SC5_BORDER_KEEP) {
        for (int i = 0; i < n; ++i) {
            sc5_plan_desc fd = p->d;
            fd.H = imgs[i].H;
            fd.W = imgs[i].W;
            fd.in_pitch = imgs[i].in_pitch;
            fd.out_pitch = imgs[i].out_pitch;
            st = run_frame(fd, imgs[i].in, imgs[i].out, imgs[i].in_scale, imgs[i].out_scale, s);
            if (st != SC5_OK) return st;
        }
    }
    return SC5_OK;
}

struct sc5_batch_s {
    int device = 0;
    unsigned char *ws = nullptr;
    int64_t ntiles = 0;
    int grid = 0;
    FusedShape shape{};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

// CTAs per SM for a batch, measured on the batch itself: every feasible count,
// one warm-up and three timed launches each on a private stream, median kept
// (the launches write the batch's outputs, as its first replay would).
static cudaError_t time_batch_ctas(int in_dtype, int out_dtype, int idx, unsigned char *ws, size_t toff,
                                   int64_t ntiles, int *ctas, float *best_ms = nullptr)
{
    const int maxc = fused_max_ctas_per_sm(in_dtype, out_dtype, idx);
    if (maxc < 1) return cudaErrorInvalidConfiguration;
    cudaStream_t s = nullptr;
    cudaEvent_t a = nullptr, z = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&z);
    float best = 0.f;
    for (int c = 1; c <= maxc && e == cudaSuccess; ++c) {
        const int grid = static_cast<int>(std::max<int64_t>(1, std::min(ntiles, static_cast<int64_t>(num_sms()) * c)));
        std::vector<float> ts;
        for (int r = 0; r < 4 && e == cudaSuccess; ++r) {
            e = cudaEventRecord(a, s);
            if (e == cudaSuccess)
                e = launch_fused_batch(in_dtype, out_dtype, idx, reinterpret_cast<const ImgDesc *>(ws),
                                       reinterpret_cast<const TileRec *>(ws + toff), ntiles, grid, s);
            if (e == cudaSuccess) e = cudaEventRecord(z, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(z);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, z);
            if (r > 0) ts.push_back(ms);
        }
        if (e != cudaSuccess) break;
        std::sort(ts.begin(), ts.end());
        if (c == 1 || ts[1] < best) {
            best = ts[1];
            *ctas = c;
        }
    }
    if (best_ms) *best_ms = best;
    if (a) cudaEventDestroy(a);
    if (z) cudaEventDestroy(z);
    if (s) cudaStreamDestroy(s);
    return e;
}

// Every compiled shape of the plan's dtype pair, each at every feasible CTA
// count, timed on the batch itself (its own work-list per shape); the
// fastest (shape index, CTAs per SM).  The timing launches write the
// batch's outputs.
static sc5_status time_batch_shapes(const sc5_plan_desc &d, int n, const sc5_image *imgs, int *idx, int *ctas)
{
    float best = 0.f;
    int found = -1;
    for (int i = 0; i < fused_num_shapes(d.in_dtype, d.out_dtype); ++i) {
        FusedShape sh{};
        fused_shape(d.in_dtype, d.out_dtype, i, &sh);
        std::vector<unsigned char> blob;
        int64_t ntiles = 0;
        size_t toff = 0;
        sc5_status st = build_batch(d, n, imgs, sh, &blob, &ntiles, &toff);
        if (st != SC5_OK) return st;
        unsigned char *ws = nullptr;
        cudaError_t e = cudaMalloc(&ws, blob.size());
        if (e == cudaSuccess) e = cudaMemcpy(ws, blob.data(), blob.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = fused_prepare(d.in_dtype, d.out_dtype, i);
        int c = 1;
        float ms = 0.f;
        if (e == cudaSuccess) e = time_batch_ctas(d.in_dtype, d.out_dtype, i, ws, toff, ntiles, &c, &ms);
        cudaFree(ws);
        if (e != cudaSuccess) return fail_cuda(e, "timing the batch's shapes");
        if (found < 0 || ms < best) {
            best = ms;
            found = i;
            *ctas = c;
        }
    }
    if (found < 0) return fail(SC5_EINVAL, "no compiled shape for the dtype pair");
    *idx = found;
    return SC5_OK;
}

extern "C" sc5_status sepconv5_batch_create(sc5_plan p, int32_t n, const sc5_image *imgs, sc5_batch *out)
{
    clear_error();
    if (!p || !out) return fail(SC5_EINVAL, "null argument");
    *out = nullptr;
    if (p->d.algo != SC5_ALGO_FUSED) return fail(SC5_EINVAL, "batches run the fused form only");
    if (taps_of(p->d) != kTaps || p->d.layout != SC5_LAYOUT_PLANAR)
        return fail(SC5_EINVAL, "batches are built for planar images of width 5");
    int idx = 0, ctas = 1;
    sc5_status st = batch_shape(p, n, imgs, &idx, &ctas);
    if (st != SC5_OK) return st;
    const bool time_shapes = p->d.ctas_per_sm == -2 && !p->d.tile_h && !p->d.tile_w && !p->d.stages;
    if (time_shapes) {
        st = time_batch_shapes(p->d, n, imgs, &idx, &ctas);
        if (st != SC5_OK) return st;
    }
    sc5_batch b = new (std::nothrow) sc5_batch_s;
    if (!b) return fail(SC5_ENOMEM, "host allocation failed");
    cudaGetDevice(&b->device);
    fused_shape(p->d.in_dtype, p->d.out_dtype, idx, &b->shape);
    std::vector<unsigned char> blob;
    size_t toff = 0;
    st = build_batch(p->d, n, imgs, b->shape, &blob, &b->ntiles, &toff);
    if (st != SC5_OK) {
        delete b;
        return st;
    }
    cudaError_t e = cudaMalloc(&b->ws, blob.size());
    if (e == cudaSuccess) e = cudaMemcpy(b->ws, blob.data(), blob.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = fused_prepare(p->d.in_dtype, p->d.out_dtype, idx);
    if (e == cudaSuccess && p->d.ctas_per_sm < 0 && !time_shapes)
        e = time_batch_ctas(p->d.in_dtype, p->d.out_dtype, idx, b->ws, toff, b->ntiles, &ctas);
    const int64_t cap = static_cast<int64_t>(num_sms()) * ctas;
    b->grid = static_cast<int>(std::max<int64_t>(1, std::min(b->ntiles, cap)));
    cudaStream_t cs = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t le = launch_fused_batch(p->d.in_dtype, p->d.out_dtype, idx,
                                            reinterpret_cast<const ImgDesc *>(b->ws),
                                            reinterpret_cast<const TileRec *>(b->ws + toff), b->ntiles,
                                            b->grid, cs);
        if (le == cudaSuccess && p->d.border == SC5_BORDER_KEEP) {
            for (int i = 0; i < n && le == cudaSuccess; ++i) {
                const float ratio = static_cast<float>(static_cast<double>(imgs[i].out_scale) / imgs[i].in_scale);
                le = launch_keep_frame(p->d.in_dtype, p->d.out_dtype, imgs[i].in, p->d.planes, imgs[i].H,
                                       imgs[i].W, imgs[i].in_pitch, imgs[i].out, imgs[i].out_pitch, ratio, cs);
            }
        }
        e = cudaStreamEndCapture(cs, &b->graph);
        if (le != cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (cs) cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        if (b->graph) cudaGraphDestroy(b->graph);
        cudaFree(b->ws);
        delete b;
        return fail_cuda(e, "batch graph capture");
    }
    *out = b;
    return SC5_OK;
}

extern "C" sc5_status sepconv5_batch_launch(sc5_batch b, void *stream)
{
    clear_error();
    if (!b) return fail(SC5_EINVAL, "null batch");
    cudaError_t e = cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail_cuda(e, "graph launch");
    note_launches(1);
    return SC5_OK;
}

extern "C" sc5_status sepconv5_batch_info(sc5_batch b, int64_t *tiles, int32_t *ctas, int32_t *tile_h,
                                          int32_t *tile_w)
{
    clear_error();
    if (!b) return fail(SC5_EINVAL, "null batch");
    if (tiles) *tiles = b->ntiles;
    if (ctas) *ctas = b->grid;
    if (tile_h) *tile_h = b->shape.tile_h;
    if (tile_w) *tile_w = b->shape.tile_w;
    return SC5_OK;
}

extern "C" sc5_status sepconv5_batch_destroy(sc5_batch b)
{
    clear_error();
    if (!b) return SC5_OK;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    cudaFree(b->ws);
    delete b;
    return SC5_OK;
}

// ------------------------------------------------------------------ misc

extern "C" sc5_status sepconv5_fused_configs(int32_t in_dtype, int32_t out_dtype, int32_t *cfg, int32_t cap,
                                             int32_t *n)
{
    clear_error();
    if (!n) return fail(SC5_EINVAL, "null argument");
    const int m = fused_num_shapes(in_dtype, out_dtype);
    *n = m;
    for (int i = 0; i < m && i < cap && cfg; ++i) {
        FusedShape s;
        fused_shape(in_dtype, out_dtype, i, &s);
        cfg[3 * i] = s.tile_h;
        cfg[3 * i + 1] = s.tile_w;
        cfg[3 * i + 2] = s.stages;
    }
    return m ? SC5_OK : fail(SC5_EINVAL, "dtype pair not built");
}

extern "C" const char *sepconv5_last_error(void) { return t_err.c_str(); }

extern "C" sc5_status sepconv5_empty_launches(int32_t n, void *stream)
{
    clear_error();
    cudaError_t e = launch_empty(n, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? SC5_OK : fail_cuda(e, "empty launch");
}

extern "C" int64_t sepconv5_launch_count(void) { return g_launches.load(); }

extern "C" sc5_status sepconv5_selftest_wait_timeout(int32_t limit_us, void *stream)
{
    clear_error();
    if (limit_us < 1 || limit_us > 100000) return fail(SC5_EINVAL, "limit_us must be in [1, 100000]");
    cudaError_t e = launch_wait_selftest(limit_us, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? SC5_OK : fail_cuda(e, "self-test launch");
}
