// sc5_device.cuh -- device helpers shared by the kernels of libsepconv5:
// inline-PTX wrappers for mbarriers, TMA tensor loads and the global timer,
// and the storage-format traits (load 8 stored values as FP32, store 4 FP32
// results in a stored format).
#pragma once

#include <cuda.h>          // CUtensorMap (type only; no driver symbols are linked)
#include <cuda_runtime.h>
#include <stdint.h>

#include "sc5_internal.h"

namespace sc5 {

// ------------------------------------------------------------------ PTX wrappers

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_timer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Make the initialised barriers visible to the async (TMA) proxy.
__device__ __forceinline__ void fence_barrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}

// Wait for phase `parity` of a barrier, giving up after limit_ns of global
// time.  Returns false on time-out; the caller records the error and leaves.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t limit_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_timer_ns() - t0 > limit_ns) return false;
    }
    return true;
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap *m)
{
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(m)) : "memory");
}

// 3-D tiled TMA load of one box into shared memory; completion is signalled
// on `bar` as transaction bytes.  x is the innermost (column) coordinate.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *m, uint64_t *bar,
                                            int32_t x, int32_t y, int32_t z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(m)), "r"(smem_u32(bar)),
          "r"(x), "r"(y), "r"(z)
        : "memory");
}

// ------------------------------------------------------------------ formats

struct fp8e4m3_t { uint8_t v; };
struct bf16_t { uint16_t v; };
struct f16_t { uint16_t v; };

__device__ __forceinline__ float bf16_bits_to_f32(uint32_t b) { return __uint_as_float(b << 16); }

__device__ __forceinline__ void f16x2_to_f32(uint32_t h2, float &lo, float &hi)
{
    asm("{\n\t.reg .f16 a, b;\n\t"
        "mov.b32 {a, b}, %2;\n\t"
        "cvt.f32.f16 %0, a;\n\t"
        "cvt.f32.f16 %1, b;\n\t}"
        : "=f"(lo), "=f"(hi) : "r"(h2));
}

// two E4M3 codes (low byte first) -> f16x2 (exact), then -> two floats (exact)
__device__ __forceinline__ void e4m3x2_to_f32(uint32_t b16, float &lo, float &hi)
{
    uint32_t h2;
    asm("{\n\t.reg .b16 s;\n\t"
        "cvt.u16.u32 s, %1;\n\t"
        "cvt.rn.f16x2.e4m3x2 %0, s;\n\t}"
        : "=r"(h2) : "r"(b16));
    f16x2_to_f32(h2, lo, hi);
}

// pack two floats, `lo` into the low half
__device__ __forceinline__ uint32_t f32x2_to_bf16x2(float lo, float hi)
{
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

__device__ __forceinline__ uint32_t f32x2_to_f16x2(float lo, float hi)
{
    uint32_t r;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

__device__ __forceinline__ uint32_t f32x2_to_e4m3x2(float lo, float hi)
{
    uint32_t r;
    asm("{\n\t.reg .b16 s;\n\t"
        "cvt.rn.satfinite.e4m3x2.f32 s, %1, %2;\n\t"
        "cvt.u32.u16 %0, s;\n\t}"
        : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

// Storage traits.  load8 reads stored elements p[0..7] (p aligned to 4
// elements) and widens them exactly to float.  store4 narrows 4 floats.

// Pairings of the 8 widened inputs a0..a7 for the packed row pass:
//   adjacent  E = (a0,a1), (a2,a3), (a4,a5), (a6,a7) and shifted O = (a1,a2),
//             (a3,a4), (a5,a6) -- free for FP32 data, whose 16-byte loads
//             already fill register pairs;
//   stride 2  S_j = (a_j, a_{j+2}), j = 0..5 -- for narrow formats, where every
//             element is widened by one instruction anyway and can be widened
//             straight into its slot of a pair.
template <class T> struct Fmt;

template <> struct Fmt<float> {
    static constexpr int bytes = 4;
    static constexpr bool kStride2 = false;
    __device__ static __forceinline__ void load4(const float *p, float *a)
    {
        const float4 u = *reinterpret_cast<const float4 *>(p);
        a[0] = u.x; a[1] = u.y; a[2] = u.z; a[3] = u.w;
    }
    __device__ static __forceinline__ void load8(const float *p, float (&a)[8])
    {
        load4(p, a);
        load4(p + 4, a + 4);
    }
    __device__ static __forceinline__ float load1(const float *p) { return *p; }
    __device__ static __forceinline__ void store4(float *p, const float (&r)[4])
    {
        __stcs(reinterpret_cast<float4 *>(p), make_float4(r[0], r[1], r[2], r[3]));
    }
    __device__ static __forceinline__ void store1(float *p, float r) { __stcs(p, r); }
};

template <> struct Fmt<bf16_t> {
    static constexpr int bytes = 2;
    static constexpr bool kStride2 = true;
    __device__ static __forceinline__ void load8(const bf16_t *p, float (&a)[8])
    {
        load4(p, a);
        load4(p + 4, a + 4);
    }
    __device__ static __forceinline__ void load4(const bf16_t *p, float *a)
    {
        // a bfloat16 is the upper half of a binary32: one shift or mask per element
        const uint2 u = *reinterpret_cast<const uint2 *>(p);
        a[0] = __uint_as_float(u.x << 16); a[1] = __uint_as_float(u.x & 0xffff0000u);
        a[2] = __uint_as_float(u.y << 16); a[3] = __uint_as_float(u.y & 0xffff0000u);
    }
    // p[0..7] with one 16-byte load (p aligned to 8 elements)
    __device__ static __forceinline__ void load8a(const bf16_t *p, float *a)
    {
        const uint4 u = *reinterpret_cast<const uint4 *>(p);
        a[0] = __uint_as_float(u.x << 16); a[1] = __uint_as_float(u.x & 0xffff0000u);
        a[2] = __uint_as_float(u.y << 16); a[3] = __uint_as_float(u.y & 0xffff0000u);
        a[4] = __uint_as_float(u.z << 16); a[5] = __uint_as_float(u.z & 0xffff0000u);
        a[6] = __uint_as_float(u.w << 16); a[7] = __uint_as_float(u.w & 0xffff0000u);
    }
    __device__ static __forceinline__ float load1(const bf16_t *p) { return bf16_bits_to_f32(p->v); }
    __device__ static __forceinline__ void store4(bf16_t *p, const float (&r)[4])
    {
        uint2 w;
        w.x = f32x2_to_bf16x2(r[0], r[1]);
        w.y = f32x2_to_bf16x2(r[2], r[3]);
        __stcs(reinterpret_cast<uint2 *>(p), w);
    }
    __device__ static __forceinline__ void store1(bf16_t *p, float r)
    {
        p->v = static_cast<uint16_t>(f32x2_to_bf16x2(r, 0.f) & 0xffffu);
    }
};

template <> struct Fmt<f16_t> {
    static constexpr int bytes = 2;
    static constexpr bool kStride2 = true;
    __device__ static __forceinline__ void load8(const f16_t *p, float (&a)[8])
    {
        load4(p, a);
        load4(p + 4, a + 4);
    }
    __device__ static __forceinline__ void load4(const f16_t *p, float *a)
    {
        const uint2 u = *reinterpret_cast<const uint2 *>(p);
        f16x2_to_f32(u.x, a[0], a[1]);
        f16x2_to_f32(u.y, a[2], a[3]);
    }
    // p[0..7] with one 16-byte load (p aligned to 8 elements)
    __device__ static __forceinline__ void load8a(const f16_t *p, float *a)
    {
        const uint4 u = *reinterpret_cast<const uint4 *>(p);
        f16x2_to_f32(u.x, a[0], a[1]);
        f16x2_to_f32(u.y, a[2], a[3]);
        f16x2_to_f32(u.z, a[4], a[5]);
        f16x2_to_f32(u.w, a[6], a[7]);
    }
    __device__ static __forceinline__ float load1(const f16_t *p)
    {
        float lo, hi;
        f16x2_to_f32(p->v, lo, hi);
        return lo;
    }
    __device__ static __forceinline__ void store4(f16_t *p, const float (&r)[4])
    {
        uint2 w;
        w.x = f32x2_to_f16x2(r[0], r[1]);
        w.y = f32x2_to_f16x2(r[2], r[3]);
        __stcs(reinterpret_cast<uint2 *>(p), w);
    }
    __device__ static __forceinline__ void store1(f16_t *p, float r)
    {
        p->v = static_cast<uint16_t>(f32x2_to_f16x2(r, 0.f) & 0xffffu);
    }
};

template <> struct Fmt<fp8e4m3_t> {
    static constexpr int bytes = 1;
    static constexpr bool kStride2 = true;
    __device__ static __forceinline__ void load8(const fp8e4m3_t *p, float (&a)[8])
    {
        load4(p, a);
        load4(p + 4, a + 4);
    }
    __device__ static __forceinline__ void load4(const fp8e4m3_t *p, float *a)
    {
        const uint32_t u = *reinterpret_cast<const uint32_t *>(p);
        e4m3x2_to_f32(u & 0xffffu, a[0], a[1]);
        e4m3x2_to_f32(u >> 16, a[2], a[3]);
    }
    // p[0..7] with one 8-byte load (p aligned to 8 elements)
    __device__ static __forceinline__ void load8a(const fp8e4m3_t *p, float *a)
    {
        const uint2 u = *reinterpret_cast<const uint2 *>(p);
        e4m3x2_to_f32(u.x & 0xffffu, a[0], a[1]);
        e4m3x2_to_f32(u.x >> 16, a[2], a[3]);
        e4m3x2_to_f32(u.y & 0xffffu, a[4], a[5]);
        e4m3x2_to_f32(u.y >> 16, a[6], a[7]);
    }
    __device__ static __forceinline__ float load1(const fp8e4m3_t *p)
    {
        float lo, hi;
        e4m3x2_to_f32(p->v, lo, hi);
        return lo;
    }
    __device__ static __forceinline__ void store4(fp8e4m3_t *p, const float (&r)[4])
    {
        const uint32_t w = f32x2_to_e4m3x2(r[0], r[1]) | (f32x2_to_e4m3x2(r[2], r[3]) << 16);
        __stcs(reinterpret_cast<unsigned int *>(p), w);
    }
    __device__ static __forceinline__ void store1(fp8e4m3_t *p, float r)
    {
        p->v = static_cast<uint8_t>(f32x2_to_e4m3x2(r, 0.f) & 0xffu);
    }
};

// ------------------------------------------------------------------ packed FP32 pairs
// Blackwell executes two IEEE binary32 multiply-adds per instruction on a
// register pair (fma.rn.f32x2); each half is rounded exactly as the scalar
// fmaf would round it, so packed and scalar code give the same bits.

__device__ __forceinline__ uint64_t pack2(float lo, float hi)
{
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ void unpack2(uint64_t v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

// a * b + c, element-wise on pairs
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// ------------------------------------------------------------------ arithmetic
// The two 1D passes, with the taps applied in the fixed order t = 0..4
// (a plain product for t = 0, then fused multiply-adds), so that every kernel
// of the library produces bitwise the same FP32 values.

// horizontal: h = sum_t k[t] * a[c + t]
__device__ __forceinline__ float hdot(const float *k, const float *a)
{
    float s = __fmul_rn(k[0], a[0]);
    s = __fmaf_rn(k[1], a[1], s);
    s = __fmaf_rn(k[2], a[2], s);
    s = __fmaf_rn(k[3], a[3], s);
    s = __fmaf_rn(k[4], a[4], s);
    return s;
}

}  // namespace sc5
