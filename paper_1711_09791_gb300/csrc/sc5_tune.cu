// sc5_tune.cu -- autotuner for the fused kernel (the GPU counterpart of the
// paper's tuning of the thread / task count, Sec. 4 and Sec. 7: 100 threads
// was the chosen "magic number", 120 helped some images).  For each size
// class of plane area, each dtype pair and each kernel kind it times every
// compiled tile shape at every feasible CTAs-per-SM count on synthetic images
// of that class and keeps the fastest: the batch kind on a batch of at least
// 512 MB of input replayed from a CUDA graph, the single-image kind on up to
// 32 separate plan runs over distinct images of the same set.  The table
// lives in the process and can be saved / loaded as JSON (one entry per
// line) keyed by GPU name.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <mutex>
#include <set>
#include <string>
#include <utility>
#include <vector>

#include "sc5_internal.h"
#include "sc5_tune.h"

namespace sc5 {

sc5_status fail(sc5_status st, const char *fmt, ...);
sc5_status fail_cuda(cudaError_t e, const char *what);
void clear_error();

struct TuneEntry {
    int in, out, kind, cls;
    int th, tw, stages, ctas;
    double us;
};

static std::mutex g_mu;
static std::vector<TuneEntry> g_table;

int size_class(double px)
{
    const double l = std::log2(std::max(px, 1.0));
    const int c = static_cast<int>(std::floor((l - 12.0) / 2.0));
    return std::min(kNumClasses - 1, std::max(0, c));
}

// Representative plane (H, W) of a class: area 2^(13 + 2c), nearly square.
static void class_shape(int c, int *H, int *W)
{
    const int e = 13 + 2 * c;
    *H = 1 << (e / 2);
    *W = 1 << (e - e / 2);
}

bool tune_lookup_internal(int in_dtype, int out_dtype, int H, int W, int kind, int *tile_h, int *tile_w,
                          int *stages, int *ctas_per_sm)
{
    const int c = size_class(static_cast<double>(H) * W);
    std::lock_guard<std::mutex> lk(g_mu);
    for (const auto &e : g_table)
        if (e.in == in_dtype && e.out == out_dtype && e.kind == kind && e.cls == c) {
            *tile_h = e.th;
            *tile_w = e.tw;
            *stages = e.stages;
            *ctas_per_sm = e.ctas;
            return true;
        }
    return false;
}

static std::string gpu_name()
{
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
        return "unknown";
    return prop.name;
}

// Median time in microseconds of `reps` repetitions of one configuration on
// n images of one size: one graph-replayed batch launch (batch kind), or one
// plan run per image for up to kSingleRuns images (single-image kind, time
// per run scaled to n images).
static sc5_status time_config(int in, int out, int H, int W, int n, int idx, int ctas, int kind,
                              unsigned char *din, unsigned char *dout, size_t in_img, size_t out_img, int reps,
                              double *us)
{
    constexpr int kSingleRuns = 32;
    FusedShape sh;
    fused_shape(in, out, idx, &sh);
    sc5_plan_desc d{};
    d.planes = 3;
    d.H = H;
    d.W = W;
    const int ei = dtype_bytes(in);
    d.in_pitch = (static_cast<int64_t>(W) * ei + 15) / 16 * 16 / ei;
    d.out_pitch = (W - 4 + 3) / 4 * 4;
    d.in_dtype = in;
    d.out_dtype = out;
    d.border = SC5_BORDER_VALID;
    d.algo = SC5_ALGO_FUSED;
    d.tile_h = sh.tile_h;
    d.tile_w = sh.tile_w;
    d.stages = sh.stages;
    d.ctas_per_sm = ctas;
    sc5_plan p = nullptr;
    sc5_status st = sepconv5_plan(&d, &p);
    if (st != SC5_OK) return st;
    std::vector<sc5_image> imgs(n);
    for (int i = 0; i < n; ++i) {
        sc5_image &im = imgs[i];
        im.in = din + i * in_img;
        im.out = dout + i * out_img;
        im.H = H;
        im.W = W;
        im.in_pitch = d.in_pitch;
        im.out_pitch = d.out_pitch;
        const float k[5] = {0.0625f, 0.25f, 0.375f, 0.25f, 0.0625f};
        for (int t = 0; t < 5; ++t) im.k[t] = k[t];
        im.in_scale = im.out_scale = 1.f;
    }
    sc5_batch b = nullptr;
    if (kind == kKindBatch) {
        st = sepconv5_batch_create(p, n, imgs.data(), &b);
        if (st != SC5_OK) {
            sepconv5_plan_destroy(p);
            return st;
        }
    }
    const int runs = std::min(n, kSingleRuns);
    cudaStream_t s = nullptr;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    cudaEvent_t a, e;
    cudaEventCreate(&a);
    cudaEventCreate(&e);
    std::vector<float> ts;
    for (int r = 0; r < reps + 2 && st == SC5_OK; ++r) {
        cudaEventRecord(a, s);
        if (kind == kKindBatch) {
            st = sepconv5_batch_launch(b, s);
        } else {
            for (int i = 0; i < runs && st == SC5_OK; ++i)
                st = sepconv5_run(p, imgs[i].in, imgs[i].out, imgs[i].k, 1.f, 1.f, s);
        }
        cudaEventRecord(e, s);
        cudaEventSynchronize(e);
        float ms = 0;
        cudaEventElapsedTime(&ms, a, e);
        if (kind != kKindBatch) ms *= static_cast<float>(n) / runs;
        if (r >= 2) ts.push_back(ms);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(e);
    cudaStreamDestroy(s);
    if (b) sepconv5_batch_destroy(b);
    sepconv5_plan_destroy(p);
    if (st != SC5_OK) return st;
    std::sort(ts.begin(), ts.end());
    *us = 1000.0 * ts[ts.size() / 2];
    return SC5_OK;
}

static sc5_status save_table(const char *path)
{
    FILE *f = std::fopen(path, "w");
    if (!f) return fail(SC5_EINVAL, "cannot write %s", path);
    const std::string name = gpu_name();
    std::fprintf(f, "{\"gpu\": \"%s\", \"entries\": [\n", name.c_str());
    std::lock_guard<std::mutex> lk(g_mu);
    for (size_t i = 0; i < g_table.size(); ++i) {
        const auto &e = g_table[i];
        std::fprintf(f,
                     "{\"in\": %d, \"out\": %d, \"kind\": %d, \"cls\": %d, \"tile_h\": %d, \"tile_w\": %d, "
                     "\"stages\": %d, \"ctas\": %d, \"us\": %.3f}%s\n",
                     e.in, e.out, e.kind, e.cls, e.th, e.tw, e.stages, e.ctas, e.us,
                     i + 1 < g_table.size() ? "," : "");
    }
    std::fprintf(f, "]}\n");
    std::fclose(f);
    return SC5_OK;
}

}  // namespace sc5

using namespace sc5;

extern "C" sc5_status sepconv5_autotune(int32_t mode, const int32_t *dtypes, int32_t n_pairs, const char *path)
{
    clear_error();
    if (mode == 0) {
        std::lock_guard<std::mutex> lk(g_mu);
        g_table.clear();
        return SC5_OK;
    }
    if (!dtypes || n_pairs < 1) return fail(SC5_EINVAL, "no dtype pairs given");
    const int reps = mode >= 2 ? 10 : 3;
    // Each class is tuned on a batch of images of its representative size
    // that together hold at least kTuneBytes of input: far more than the L2,
    // so the timings see the HBM-streaming behaviour of real batches.
    constexpr size_t kTuneBytes = 512ull << 20;
    std::vector<TuneEntry> found;
    for (int q = 0; q < n_pairs; ++q) {
        const int in = dtypes[2 * q], out = dtypes[2 * q + 1];
        const int nshapes = fused_num_shapes(in, out);
        if (!nshapes) return fail(SC5_EINVAL, "dtype pair (%d, %d) not built", in, out);
        for (int c = 0; c < kNumClasses; ++c) {
            int H, W;
            class_shape(c, &H, &W);
            const int ei = dtype_bytes(in), eo = dtype_bytes(out);
            const size_t in_pitch = (static_cast<size_t>(W) * ei + 15) / 16 * 16 / ei;
            const size_t out_pitch = (W - 4 + 3) / 4 * 4;
            const size_t in_img = (3 * H * in_pitch * ei + 255) / 256 * 256;
            const size_t out_img = (3 * (H - 4) * out_pitch * eo + 255) / 256 * 256;
            const int n = static_cast<int>(std::max<size_t>(1, (kTuneBytes + in_img - 1) / in_img));
            unsigned char *din = nullptr, *dout = nullptr;
            cudaError_t e = cudaMalloc(&din, n * in_img);
            if (e == cudaSuccess) e = cudaMalloc(&dout, n * out_img);
            if (e == cudaSuccess) e = cudaMemset(din, 0x3c, n * in_img);
            if (e != cudaSuccess) {
                cudaFree(din);
                cudaFree(dout);
                return fail_cuda(e, "autotune buffers");
            }
            for (int kind : {kKindSingle, kKindBatch}) {
                TuneEntry best{in, out, kind, c, 0, 0, 0, 0, 1e30};
                for (int idx = 0; idx < nshapes; ++idx) {
                    const int maxc = fused_max_ctas_per_sm(in, out, idx);
                    for (int ctas = 1; ctas <= maxc; ++ctas) {
                        double us = 0;
                        sc5_status st =
                            time_config(in, out, H, W, n, idx, ctas, kind, din, dout, in_img, out_img, reps, &us);
                        if (st != SC5_OK) {
                            cudaFree(din);
                            cudaFree(dout);
                            return st;
                        }
                        if (us < best.us) {
                            FusedShape sh;
                            fused_shape(in, out, idx, &sh);
                            best = TuneEntry{in, out, kind, c, sh.tile_h, sh.tile_w, sh.stages, ctas, us};
                        }
                    }
                }
                found.push_back(best);
            }
            cudaFree(din);
            cudaFree(dout);
        }
    }
    {
        std::lock_guard<std::mutex> lk(g_mu);
        for (const auto &f : found) {
            g_table.erase(std::remove_if(g_table.begin(), g_table.end(),
                                         [&](const TuneEntry &e) {
                                             return e.in == f.in && e.out == f.out && e.kind == f.kind &&
                                                    e.cls == f.cls;
                                         }),
                          g_table.end());
            g_table.push_back(f);
        }
    }
    return path ? save_table(path) : SC5_OK;
}

void sc5::tune_from_environment(int in_dtype, int out_dtype)
{
    const char *mode = std::getenv("SEPCONV5_TUNE");
    const char *file = std::getenv("SEPCONV5_TUNE_FILE");
    if (!mode && !file) return;
    static std::mutex mu;
    static bool file_loaded = false;
    static std::set<std::pair<int, int>> seen;
    {
        // Marked before tuning, so that the plans the tuner itself creates
        // (and plans made meanwhile on other threads) keep the defaults.
        std::lock_guard<std::mutex> lk(mu);
        if (!seen.insert({in_dtype, out_dtype}).second) return;
        if (file && !file_loaded) {
            file_loaded = true;
            sepconv5_tune_load(file);
        }
    }
    const int m = !mode ? 0 : std::strcmp(mode, "quick") == 0 ? 1 : std::strcmp(mode, "full") == 0 ? 2 : 0;
    if (m == 0) return;
    int have = 0;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        for (const auto &e : g_table) have += (e.in == in_dtype && e.out == out_dtype);
    }
    if (have >= 2 * kNumClasses) return;
    const int32_t pair[2] = {in_dtype, out_dtype};
    sepconv5_autotune(m, pair, 1, file);
}

extern "C" sc5_status sepconv5_tune_load(const char *path)
{
    clear_error();
    if (!path) return fail(SC5_EINVAL, "null path");
    FILE *f = std::fopen(path, "r");
    if (!f) return fail(SC5_ENOTFOUND, "cannot open %s", path);
    char line[512];
    std::string gpu;
    std::vector<TuneEntry> loaded;
    while (std::fgets(line, sizeof line, f)) {
        const char *g = std::strstr(line, "\"gpu\": \"");
        if (g) {
            g += 8;
            const char *e = std::strchr(g, '"');
            if (e) gpu.assign(g, e);
        }
        TuneEntry t;
        if (std::sscanf(line,
                        " {\"in\": %d, \"out\": %d, \"kind\": %d, \"cls\": %d, \"tile_h\": %d, \"tile_w\": %d, "
                        "\"stages\": %d, \"ctas\": %d, \"us\": %lf",
                        &t.in, &t.out, &t.kind, &t.cls, &t.th, &t.tw, &t.stages, &t.ctas, &t.us) == 9 &&
            (t.kind == kKindSingle || t.kind == kKindBatch))
            loaded.push_back(t);
    }
    std::fclose(f);
    if (gpu != gpu_name()) return fail(SC5_ENOTFOUND, "table is for GPU '%s'", gpu.c_str());
    std::lock_guard<std::mutex> lk(g_mu);
    for (const auto &t : loaded)
        if (fused_find_shape(t.in, t.out, t.th, t.tw, t.stages) >= 0 && t.cls >= 0 && t.cls < kNumClasses)
            g_table.push_back(t);
    return SC5_OK;
}

static sc5_status tune_lookup_kind(int32_t in_dtype, int32_t out_dtype, int32_t H, int32_t W, int kind,
                                   int32_t *tile_h, int32_t *tile_w, int32_t *stages, int32_t *ctas_per_sm)
{
    clear_error();
    if (!tile_h || !tile_w || !stages || !ctas_per_sm) return fail(SC5_EINVAL, "null argument");
    int th, tw, st, c;
    if (tune_lookup_internal(in_dtype, out_dtype, H, W, kind, &th, &tw, &st, &c)) {
        *tile_h = th;
        *tile_w = tw;
        *stages = st;
        *ctas_per_sm = c;
        return SC5_OK;
    }
    FusedShape s;
    if (!fused_shape(in_dtype, out_dtype, 0, &s)) return fail(SC5_EINVAL, "dtype pair not built");
    *tile_h = s.tile_h;
    *tile_w = s.tile_w;
    *stages = s.stages;
    *ctas_per_sm = 0;
    return SC5_ENOTFOUND;
}

extern "C" sc5_status sepconv5_tune_lookup(int32_t in_dtype, int32_t out_dtype, int32_t H, int32_t W,
                                           int32_t *tile_h, int32_t *tile_w, int32_t *stages,
                                           int32_t *ctas_per_sm)
{
    return tune_lookup_kind(in_dtype, out_dtype, H, W, kKindSingle, tile_h, tile_w, stages, ctas_per_sm);
}

extern "C" sc5_status sepconv5_tune_lookup_batch(int32_t in_dtype, int32_t out_dtype, int32_t H, int32_t W,
                                                 int32_t *tile_h, int32_t *tile_w, int32_t *stages,
                                                 int32_t *ctas_per_sm)
{
    return tune_lookup_kind(in_dtype, out_dtype, H, W, kKindBatch, tile_h, tile_w, stages, ctas_per_sm);
}
