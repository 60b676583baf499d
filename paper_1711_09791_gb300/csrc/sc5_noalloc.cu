// sc5_noalloc.cu -- the two-pass form for callers that cannot allocate device
// memory.
//
// Some callers of this library may not call cudaMalloc themselves and may not
// let a library do it on their behalf: code running under a framework whose
// caching allocator owns all of the GPU's memory, latency-bound loops that
// cannot absorb the device-wide synchronisation a cudaFree may cause, or
// plug-ins whose host application forbids allocation calls.  The regular
// two-pass path needs an FP32 intermediate image T, which sepconv5_plan
// allocates.  This entry point keeps T instead in a fixed array declared
// below, so a call allocates nothing; the caller still passes the input and
// output images.  The array is part of the library image: every GPU that
// loads the library holds SC5_NOALLOC_MAX_T_FLOATS * 4 bytes (16 MiB) until
// the process exits.
#include <cmath>
#include <mutex>

#include "sc5_internal.h"

namespace sc5 {

sc5_status fail(sc5_status st, const char *fmt, ...);
sc5_status fail_cuda(cudaError_t e, const char *what);
void clear_error();

// The shared intermediate.  Its name is only a host-side stand-in in host
// code; the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) float g_noalloc_T[SC5_NOALLOC_MAX_T_FLOATS];

// Device address of g_noalloc_T on the current device, looked up once per
// device (with that device current) and cached.
static sc5_status noalloc_scratch(float **out)
{
    static std::mutex mu;
    static float *addr[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_cuda(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(SC5_EINVAL, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_T);
        if (e != cudaSuccess) return fail_cuda(e, "cudaGetSymbolAddress of the no-allocation scratch");
        addr[dev] = static_cast<float *>(p);
    }
    *out = addr[dev];
    return SC5_OK;
}

}  // namespace sc5

using namespace sc5;

extern "C" sc5_status sepconv5_two_pass_noalloc(const void *in, void *out, int32_t planes, int32_t H, int32_t W,
                                                int64_t in_pitch, int64_t out_pitch, int32_t in_dtype,
                                                int32_t out_dtype, const float k[5], float in_scale,
                                                float out_scale, void *stream)
{
    clear_error();
    if (!in || !out || !k) return fail(SC5_EINVAL, "null argument");
    if (planes < 1 || H < 5 || W < 5) return fail(SC5_EINVAL, "need planes >= 1, H >= 5, W >= 5");
    if (H > 65535) return fail(SC5_EINVAL, "two-pass form needs H <= 65535");
    const int ei = dtype_bytes(in_dtype), eo = dtype_bytes(out_dtype);
    if (!ei || !eo || fused_num_shapes(in_dtype, out_dtype) == 0)
        return fail(SC5_EINVAL, "dtype pair (%d -> %d) not built: the output must be the input format or FP32",
                    in_dtype, out_dtype);
    const int Wv = W - kHalo, Hv = H - kHalo;
    if (in_pitch < W || out_pitch < Wv) return fail(SC5_EINVAL, "pitch smaller than the row width");
    if ((in_pitch * ei) % 16 || reinterpret_cast<uintptr_t>(in) % 16)
        return fail(SC5_EINVAL, "input must be 16-byte aligned with in_pitch * element size a multiple of 16");
    if (reinterpret_cast<uintptr_t>(out) % eo) return fail(SC5_EINVAL, "output not aligned to its element size");
    if (!(in_scale > 0.f) || !std::isfinite(in_scale) || !(out_scale > 0.f) || !std::isfinite(out_scale))
        return fail(SC5_EINVAL, "scales must be finite and > 0");
    for (int t = 0; t < kTaps; ++t)
        if (!std::isfinite(k[t])) return fail(SC5_EINVAL, "taps must be finite");
    const int64_t t_pitch = (static_cast<int64_t>(Wv) + 3) / 4 * 4;
    const double need = static_cast<double>(planes) * H * t_pitch;
    if (need > static_cast<double>(SC5_NOALLOC_MAX_T_FLOATS))
        return fail(SC5_EINVAL,
                    "image too large for the no-allocation scratch: planes * H * round_up(W-4, 4) = %.0f floats "
                    "> %d",
                    need, SC5_NOALLOC_MAX_T_FLOATS);
    const char *a = static_cast<const char *>(in), *b = static_cast<const char *>(out);
    if (a < b + static_cast<size_t>(planes) * Hv * out_pitch * eo && b < a + static_cast<size_t>(planes) * H * in_pitch * ei)
        return fail(SC5_EINVAL, "input and output overlap");
    float *T = nullptr;
    sc5_status st = noalloc_scratch(&T);
    if (st != SC5_OK) return st;
    // Every T element the vertical pass uses is written by the horizontal pass
    // of the same call, so nothing has to be cleared between calls.
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = launch_hpass(in_dtype, in, planes, H, W, in_pitch, T, t_pitch, k, s);
    if (e != cudaSuccess) return fail_cuda(e, "hpass launch");
    const bool vec = reinterpret_cast<uintptr_t>(out) % (4 * eo) == 0 && out_pitch % 4 == 0;
    const float oscale = static_cast<float>(static_cast<double>(out_scale) / in_scale);
    e = launch_vpass(out_dtype, T, planes, H, Wv, t_pitch, out, out_pitch, static_cast<int64_t>(Hv) * out_pitch, k,
                     oscale, vec, s);
    if (e != cudaSuccess) return fail_cuda(e, "vpass launch");
    return SC5_OK;
}
