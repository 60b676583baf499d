// sc5_fused.cu -- registry of the compiled fused-kernel shapes, their
// launchers, and the device status word that bounded waits report into.
#include <mutex>
#include <set>
#include <utility>

#include "sc5_fused_entry.cuh"

namespace sc5 {

int fused_entries_f32(int out_dtype, const FusedEntry **out);
int fused_entries_16(int in_dtype, int out_dtype, const FusedEntry **out);
int fused_entries_fp8(int out_dtype, const FusedEntry **out);
int fused_direct_entries_f32(int out_dtype, const FusedEntry **out);
int fused_direct_entries_16(int in_dtype, int out_dtype, const FusedEntry **out);
int fused_direct_entries_fp8(int out_dtype, const FusedEntry **out);
int fused_width_entries_f32(int out_dtype, int taps, const FusedEntry **out);
int fused_width_entries_16(int in_dtype, int out_dtype, int taps, const FusedEntry **out);
int fused_width_entries_fp8(int out_dtype, int taps, const FusedEntry **out);

// Device status word: 0 = no error; a kernel whose bounded wait ran out
// writes its error code here (first writer wins).
__device__ int g_status;

static int entries(int in_dtype, int out_dtype, const FusedEntry **e, bool direct = false, int taps = kTaps)
{
    if (taps != kTaps) {
        if (direct) return 0;
        switch (in_dtype) {
        case SC5_F32: return fused_width_entries_f32(out_dtype, taps, e);
        case SC5_BF16:
        case SC5_F16: return fused_width_entries_16(in_dtype, out_dtype, taps, e);
        case SC5_FP8E4M3: return fused_width_entries_fp8(out_dtype, taps, e);
        default: return 0;
        }
    }
    switch (in_dtype) {
    case SC5_F32: return direct ? fused_direct_entries_f32(out_dtype, e) : fused_entries_f32(out_dtype, e);
    case SC5_BF16:
    case SC5_F16:
        return direct ? fused_direct_entries_16(in_dtype, out_dtype, e) : fused_entries_16(in_dtype, out_dtype, e);
    case SC5_FP8E4M3: return direct ? fused_direct_entries_fp8(out_dtype, e) : fused_entries_fp8(out_dtype, e);
    default: return 0;
    }
}

int fused_num_shapes(int in_dtype, int out_dtype, bool direct, int taps)
{
    const FusedEntry *e;
    return entries(in_dtype, out_dtype, &e, direct, taps);
}

bool fused_shape(int in_dtype, int out_dtype, int idx, FusedShape *s, bool direct, int taps)
{
    const FusedEntry *e;
    const int n = entries(in_dtype, out_dtype, &e, direct, taps);
    if (idx < 0 || idx >= n) return false;
    *s = e[idx].shape;
    return true;
}

int fused_find_shape(int in_dtype, int out_dtype, int tile_h, int tile_w, int stages, bool direct, int taps)
{
    const FusedEntry *e;
    const int n = entries(in_dtype, out_dtype, &e, direct, taps);
    for (int i = 0; i < n; ++i)
        if (e[i].shape.tile_h == tile_h && e[i].shape.tile_w == tile_w &&
            (stages == 0 || e[i].shape.stages == stages))
            return i;
    return -1;
}

int fused_default_ctas(int in_dtype, int out_dtype, int idx, bool direct, int taps)
{
    const FusedEntry *e;
    const int n = entries(in_dtype, out_dtype, &e, direct, taps);
    return (idx >= 0 && idx < n) ? e[idx].ctas_default : 0;
}

int fused_threads(const FusedShape &s) { return 32 * (s.tile_h / s.rows_per_thread + 1); }

// cudaFuncSetAttribute for the dynamic shared memory once per (function, device).
static cudaError_t prepare_fn(const void *fn, int smem)
{
    static std::mutex mu;
    static std::set<std::pair<const void *, int>> done;
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    std::lock_guard<std::mutex> lk(mu);
    if (done.count({fn, dev})) return cudaSuccess;
    err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (err == cudaSuccess) done.insert({fn, dev});
    return err;
}

static int *status_ptr()
{
    static std::mutex mu;
    static int *ptrs[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!ptrs[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_status) != cudaSuccess) return nullptr;
        ptrs[dev] = static_cast<int *>(p);
    }
    return ptrs[dev];
}

int *status_word() { return status_ptr(); }

int fused_max_ctas_per_sm(int in_dtype, int out_dtype, int idx, bool direct, int taps)
{
    const FusedEntry *e;
    const int n = entries(in_dtype, out_dtype, &e, direct, taps);
    if (idx < 0 || idx >= n) return -1;
    if (prepare_fn(e[idx].single_fn, e[idx].smem) != cudaSuccess) return -1;
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, e[idx].single_fn, e[idx].threads,
                                                      e[idx].smem) != cudaSuccess)
        return -1;
    return blocks;
}

cudaError_t fused_prepare(int in_dtype, int out_dtype, int idx, bool direct, int taps)
{
    const FusedEntry *e;
    const int n = entries(in_dtype, out_dtype, &e, direct, taps);
    if (idx < 0 || idx >= n) return cudaErrorInvalidValue;
    cudaError_t err = prepare_fn(e[idx].single_fn, e[idx].smem);
    if (err == cudaSuccess) err = prepare_fn(e[idx].batch_fn, e[idx].smem);
    if (err == cudaSuccess && !status_ptr()) err = cudaErrorInvalidDevicePointer;
    return err;
}

cudaError_t launch_fused_single(int in_dtype, int out_dtype, int idx, const ImgDesc &d,
                                int64_t ntiles, int grid, cudaStream_t st, bool direct, int taps)
{
    const FusedEntry *e;
    const int n = entries(in_dtype, out_dtype, &e, direct, taps);
    if (idx < 0 || idx >= n || grid < 1) return cudaErrorInvalidValue;
    if (ntiles <= 0) return cudaSuccess;
    cudaError_t err = fused_prepare(in_dtype, out_dtype, idx, direct, taps);
    if (err != cudaSuccess) return err;
    int *status = status_ptr();
    const ImgDesc *no_descs = nullptr;
    const TileRec *no_tiles = nullptr;
    void *args[] = {const_cast<ImgDesc *>(&d), &no_descs, &no_tiles, &ntiles, &status};
    err = cudaLaunchKernel(e[idx].single_fn, dim3(grid), dim3(e[idx].threads), args,
                           e[idx].smem, st);
    if (err == cudaSuccess) note_launches(1);
    return err;
}

cudaError_t launch_fused_batch(int in_dtype, int out_dtype, int idx, const ImgDesc *descs,
                               const TileRec *tiles, int64_t ntiles, int grid, cudaStream_t st)
{
    const FusedEntry *e;
    const int n = entries(in_dtype, out_dtype, &e);
    if (idx < 0 || idx >= n || grid < 1) return cudaErrorInvalidValue;
    if (ntiles <= 0) return cudaSuccess;
    cudaError_t err = fused_prepare(in_dtype, out_dtype, idx);
    if (err != cudaSuccess) return err;
    int *status = status_ptr();
    static const ImgDesc zero_desc{};  // unused by the batch variant
    void *args[] = {const_cast<ImgDesc *>(&zero_desc), &descs, &tiles, &ntiles, &status};
    err = cudaLaunchKernel(e[idx].batch_fn, dim3(grid), dim3(e[idx].threads), args,
                           e[idx].smem, st);
    if (err == cudaSuccess) note_launches(1);
    return err;
}

// One warp waits, with the kernels' bounded wait, on a fresh barrier that
// nothing will ever complete; when the limit runs out it records the time-out
// code in the status word and returns.
__global__ void wait_selftest_kernel(uint64_t limit_ns, int *status)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bar, 0, limit_ns);
    if (!ok && threadIdx.x == 0) record_error(status, kDevErrTmaTimeout);
}

cudaError_t launch_wait_selftest(int limit_us, cudaStream_t st)
{
    int *status = status_ptr();
    if (!status) return cudaErrorInvalidDevicePointer;
    wait_selftest_kernel<<<1, 32, 0, st>>>(static_cast<uint64_t>(limit_us) * 1000ull, status);
    cudaError_t err = cudaGetLastError();
    if (err == cudaSuccess) note_launches(1);
    return err;
}

cudaError_t read_and_clear_device_status(cudaStream_t st, int32_t *code)
{
    int *p = status_ptr();
    if (!p) return cudaErrorInvalidDevicePointer;
    cudaError_t err = cudaStreamSynchronize(st);
    if (err != cudaSuccess) return err;
    int v = 0;
    err = cudaMemcpy(&v, p, sizeof v, cudaMemcpyDeviceToHost);
    if (err != cudaSuccess) return err;
    if (v != 0) {
        const int zero = 0;
        err = cudaMemcpy(p, &zero, sizeof zero, cudaMemcpyHostToDevice);
    }
    *code = v;
    return err;
}

}  // namespace sc5
