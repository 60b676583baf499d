// sc5_serve.cpp -- serving runtime: continuous batching of convolution
// requests on one GPU.
//
// Requests (host images of any size, each with its own 5 taps) are queued by
// serve_submit.  A scheduler thread admits them in arrival order while the
// resident arena (a fixed device allocation of hbm_budget_bytes made at
// start) has room for their input and output and fewer than max_inflight
// are admitted; each admitted request's input is copied to the device on a
// copy stream.  What has been admitted and not yet launched is merged, up to
// max_merge requests at a time, into one persistent launch of the fused batch
// kernel (per-image descriptors + tile work-list), issued on the next of
// n_streams compute streams after the requests' copies have landed; the
// output values (not the rows' padding) are copied back to the requests' host
// buffers on a second copy stream.  At most two launches
// per compute stream are in flight: while they run, newly arriving requests
// are admitted and staged, and go out together in the next launch.  A
// completion thread retires launches as their last copy lands, frees their
// arena blocks (which lets waiting requests in) and time-stamps every
// request.  Each tile's arithmetic does not depend on what else is in the
// launch, so a request's result is the same alone and in any mix.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "sc5_internal.h"
#include "sc5_serve_host.h"

namespace sc5 {

using Clock = std::chrono::steady_clock;

namespace {

constexpr int kSlots = 8;                       // descriptor slots (launches in flight)
constexpr size_t kSlotBytes = 8u << 20;         // descriptors + tile list per launch
constexpr int kMaxQueued = 1 << 16;             // pending requests before back-pressure

struct Request {
    uint64_t id = 0;
    sc5_image img{};  // host pointers
    size_t in_bytes = 0, out_bytes = 0;
    size_t in_off = 0, out_off = 0;
    Clock::time_point t_submit, t_admit, t_launch, t_done;
    cudaEvent_t h2d = nullptr;
    bool done = false;
    sc5_status status = SC5_OK;
};

struct Launch {
    std::vector<std::shared_ptr<Request>> reqs;
    int slot = -1;
    int stream = 0;
    cudaEvent_t done = nullptr;
};

}  // namespace

}  // namespace sc5

using namespace sc5;

struct sc5_server_s {
    sc5_serve_cfg cfg{};
    int device = 0;
    unsigned char *arena_base = nullptr;
    Arena arena;
    cudaStream_t s_h2d = nullptr, s_d2h = nullptr;
    std::vector<cudaStream_t> s_comp;
    std::vector<int> inflight_per_stream;
    unsigned char *slot_dev = nullptr;
    unsigned char *slot_host = nullptr;
    std::vector<bool> slot_busy;
    std::vector<cudaEvent_t> event_pool;

    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::deque<std::shared_ptr<Request>> pending;   // submitted, not admitted
    std::vector<std::shared_ptr<Request>> staged;   // admitted, input copy issued, not launched
    Clock::time_point staged_since;                  // admission time of the oldest staged request
    std::deque<Launch> running;                      // launched, not retired
    std::unordered_map<uint64_t, std::shared_ptr<Request>> tickets;
    uint64_t next_id = 1;
    int admitted = 0;
    bool stop = false;
    sc5_serve_stats stats{};
    std::thread sched, compl_;
    int next_stream = 0;
    int fault_sched_delay_ms = 0;  // host-side fault injection (SC5_SERVE_FAULT)
    PhaseLog phases;

    cudaEvent_t get_event()
    {
        if (!event_pool.empty()) {
            cudaEvent_t e = event_pool.back();
            event_pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
        return e;
    }
    void put_event(cudaEvent_t e)
    {
        if (e) event_pool.push_back(e);
    }

    size_t need_bytes(const sc5_image &im) const
    {
        const int es = dtype_bytes(cfg.dtype);
        return round_up(static_cast<size_t>(cfg.planes) * im.H * im.in_pitch * es, kArenaAlign) +
               round_up(static_cast<size_t>(cfg.planes) * (im.H - 4) * im.out_pitch * es, kArenaAlign);
    }

    void scheduler_loop();
    void completion_loop();
    // Merge staged requests into one launch (called with mu held).
    void launch_staged(std::unique_lock<std::mutex> &lk);
};

void sc5_server_s::scheduler_loop()
{
    cudaSetDevice(device);
    const int es = dtype_bytes(cfg.dtype);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        // 1. admission, in arrival order
        if (fault_sched_delay_ms > 0 && !pending.empty()) {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::milliseconds(fault_sched_delay_ms));
            lk.lock();
        }
        while (!pending.empty() && admitted < cfg.max_inflight) {
            auto r = pending.front();
            size_t in_off = 0, out_off = 0;
            if (!arena.alloc(r->in_bytes, &in_off)) break;
            if (!arena.alloc(r->out_bytes, &out_off)) {
                arena.release(in_off, r->in_bytes);
                break;
            }
            pending.pop_front();
            r->in_off = in_off;
            r->out_off = out_off;
            r->t_admit = Clock::now();
            ++admitted;
            stats.resident_peak_bytes = std::max(stats.resident_peak_bytes, arena.used());
            r->h2d = get_event();
            cudaMemcpyAsync(arena_base + in_off, r->img.in,
                            static_cast<size_t>(cfg.planes) * r->img.H * r->img.in_pitch * es,
                            cudaMemcpyHostToDevice, s_h2d);
            cudaEventRecord(r->h2d, s_h2d);
            if (staged.empty()) staged_since = Clock::now();
            staged.push_back(r);
            if (!cfg.merge) break;  // one request per launch: launch it right away
        }
        // 2. merge what is staged into one launch when a stream slot is free
        if (!staged.empty()) {
            const int s = next_stream;
            const bool slot_free = std::find(slot_busy.begin(), slot_busy.end(), false) != slot_busy.end();
            const bool window_over =
                !cfg.merge || cfg.batch_window_us <= 0 || stop ||
                (cfg.max_merge > 0 && static_cast<int>(staged.size()) >= cfg.max_merge) ||
                Clock::now() - staged_since >= std::chrono::microseconds(cfg.batch_window_us);
            if (slot_free && inflight_per_stream[s] < 2 && window_over) {
                launch_staged(lk);
                if (!staged.empty()) staged_since = Clock::now();
                continue;
            }
        }
        if (stop && pending.empty() && staged.empty()) break;
        cv_sched.wait_for(lk, std::chrono::microseconds(200));
    }
}

void sc5_server_s::launch_staged(std::unique_lock<std::mutex> &)
{
    const int es = dtype_bytes(cfg.dtype);
    int slot = static_cast<int>(std::find(slot_busy.begin(), slot_busy.end(), false) - slot_busy.begin());
    // take requests while their work-list fits the descriptor slot
    std::vector<std::shared_ptr<Request>> group;
    std::vector<sc5_image> imgs;
    size_t bytes = 0;
    const size_t cap = !cfg.merge ? 1 : cfg.max_merge > 0 ? static_cast<size_t>(cfg.max_merge) : staged.size();
    size_t taken = 0;
    for (; taken < staged.size() && group.size() < cap; ++taken) {
        auto &r = staged[taken];
        // upper bound on this image's share: descriptor + smallest-tile work-list
        const size_t tiles = static_cast<size_t>(cfg.planes) * ((r->img.H - 4 + 31) / 32) * ((r->img.W - 4 + 127) / 128);
        const size_t add = sizeof(ImgDesc) + tiles * sizeof(TileRec);
        if (!group.empty() && bytes + add + kArenaAlign > kSlotBytes) break;
        bytes += add;
        sc5_image d = r->img;
        d.in = arena_base + r->in_off;
        d.out = arena_base + r->out_off;
        imgs.push_back(d);
        group.push_back(r);
    }
    staged.erase(staged.begin(), staged.begin() + taken);
    sc5_plan_desc pd{};
    pd.planes = cfg.planes;
    pd.in_dtype = pd.out_dtype = cfg.dtype;
    pd.border = SC5_BORDER_VALID;
    pd.algo = SC5_ALGO_FUSED;
    int idx = 0, ctas = 1;
    sc5_status st = choose_batch_shape(cfg.dtype, cfg.dtype, static_cast<int>(imgs.size()), imgs.data(), &idx, &ctas);
    FusedShape sh{};
    std::vector<unsigned char> blob;
    int64_t ntiles = 0;
    size_t toff = 0;
    if (st == SC5_OK) {
        fused_shape(cfg.dtype, cfg.dtype, idx, &sh);
        st = build_batch(pd, static_cast<int>(imgs.size()), imgs.data(), sh, &blob, &ntiles, &toff);
    }
    if (st == SC5_OK && blob.size() > kSlotBytes) st = SC5_ENOMEM;
    const int s = next_stream;
    next_stream = (next_stream + 1) % static_cast<int>(s_comp.size());
    Launch L;
    L.reqs = group;
    L.stream = s;
    L.slot = slot;
    L.done = get_event();
    cudaStream_t cs = s_comp[s];
    const auto t_launch = Clock::now();
    for (auto &r : group) r->t_launch = t_launch;
    if (st == SC5_OK) {
        slot_busy[slot] = true;
        unsigned char *hs = slot_host + static_cast<size_t>(slot) * kSlotBytes;
        unsigned char *ds = slot_dev + static_cast<size_t>(slot) * kSlotBytes;
        std::memcpy(hs, blob.data(), blob.size());
        cudaMemcpyAsync(ds, hs, blob.size(), cudaMemcpyHostToDevice, cs);
        for (auto &r : group) cudaStreamWaitEvent(cs, r->h2d, 0);
        const int64_t capc = static_cast<int64_t>(num_sms()) * ctas;
        const int grid = static_cast<int>(std::max<int64_t>(1, std::min(ntiles, capc)));
        cudaError_t e = launch_fused_batch(cfg.dtype, cfg.dtype, idx, reinterpret_cast<const ImgDesc *>(ds),
                                           reinterpret_cast<const TileRec *>(ds + toff), ntiles, grid, cs);
        if (e != cudaSuccess) st = SC5_ECUDA;
        cudaEvent_t kdone = get_event();
        cudaEventRecord(kdone, cs);
        cudaStreamWaitEvent(s_d2h, kdone, 0);
        // results go back as their W-4 valid values per row: the caller's row
        // padding is left as it was, as sepconv5_run leaves it
        for (auto &r : group) {
            const size_t pitch_b = static_cast<size_t>(r->img.out_pitch) * es;
            cudaMemcpy2DAsync(r->img.out, pitch_b, arena_base + r->out_off, pitch_b,
                              static_cast<size_t>(r->img.W - 4) * es,
                              static_cast<size_t>(cfg.planes) * (r->img.H - 4), cudaMemcpyDeviceToHost, s_d2h);
        }
        cudaEventRecord(L.done, s_d2h);
        put_event(kdone);  // its record/wait are already enqueued
    } else {
        L.slot = -1;
        cudaEventRecord(L.done, cs);
        for (auto &r : group) r->status = st;
    }
    ++inflight_per_stream[s];
    ++stats.launches;
    stats.merged_max = std::max<uint64_t>(stats.merged_max, group.size());
    running.push_back(std::move(L));
    cv_done.notify_all();
}

void sc5_server_s::completion_loop()
{
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        bool progressed = false;
        for (auto it = running.begin(); it != running.end();) {
            const cudaError_t q = cudaEventQuery(it->done);
            if (q == cudaErrorNotReady) {
                ++it;
                continue;
            }
            const auto now = Clock::now();
            for (auto &r : it->reqs) {
                if (q != cudaSuccess && r->status == SC5_OK) r->status = SC5_ECUDA;
                r->t_done = now;
                r->done = true;
                phases.add(r->t_admit - r->t_submit, r->t_launch - r->t_admit, now - r->t_launch);
                arena.release(r->in_off, r->in_bytes);
                arena.release(r->out_off, r->out_bytes);
                put_event(r->h2d);
                r->h2d = nullptr;
                --admitted;
                ++stats.completed;
            }
            if (it->slot >= 0) slot_busy[it->slot] = false;
            --inflight_per_stream[it->stream];
            put_event(it->done);
            it = running.erase(it);
            progressed = true;
        }
        if (progressed) {
            cv_done.notify_all();
            cv_sched.notify_all();
        }
        if (stop && running.empty() && pending.empty() && staged.empty()) break;
        if (!progressed) {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        }
    }
}

extern "C" sc5_status serve_create(const sc5_serve_cfg *cfg, sc5_server *out)
{
    clear_error();
    if (!cfg || !out) return fail(SC5_EINVAL, "null argument");
    *out = nullptr;
    if (!dtype_bytes(cfg->dtype) || fused_num_shapes(cfg->dtype, cfg->dtype) == 0)
        return fail(SC5_EINVAL, "unknown dtype %d", cfg->dtype);
    if (cfg->planes < 1 || cfg->hbm_budget_bytes < (1u << 20) || cfg->max_inflight < 1 || cfg->n_streams < 1)
        return fail(SC5_EINVAL, "need planes >= 1, budget >= 1 MiB, max_inflight >= 1, n_streams >= 1");
    std::unique_ptr<sc5_server_s> s(new (std::nothrow) sc5_server_s);
    if (!s) return fail(SC5_ENOMEM, "host allocation failed");
    s->cfg = *cfg;
    cudaGetDevice(&s->device);
    // Host-side fault injection for tests (never touches the GPU):
    //   SC5_SERVE_FAULT=arena_alloc       the arena allocation fails (SC5_ENOMEM)
    //   SC5_SERVE_FAULT=sched_delay_ms=N  the scheduler sleeps N ms before each admission round
    if (const char *f = std::getenv("SC5_SERVE_FAULT")) {
        if (std::strcmp(f, "arena_alloc") == 0) return fail(SC5_ENOMEM, "injected fault: arena allocation failed");
        if (std::strncmp(f, "sched_delay_ms=", 15) == 0) s->fault_sched_delay_ms = std::atoi(f + 15);
    }
    cudaError_t e = cudaMalloc(&s->arena_base, cfg->hbm_budget_bytes);
    if (e != cudaSuccess) return fail_cuda(e, "cudaMalloc of the serving arena");
    s->arena.reset(cfg->hbm_budget_bytes);
    e = cudaMalloc(&s->slot_dev, kSlots * kSlotBytes);
    if (e == cudaSuccess) e = cudaMallocHost(&s->slot_host, kSlots * kSlotBytes);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->s_h2d, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->s_d2h, cudaStreamNonBlocking);
    for (int i = 0; i < cfg->n_streams && e == cudaSuccess; ++i) {
        cudaStream_t st;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e == cudaSuccess) s->s_comp.push_back(st);
    }
    if (e != cudaSuccess) {
        cudaFree(s->arena_base);
        cudaFree(s->slot_dev);
        cudaFreeHost(s->slot_host);
        return fail_cuda(e, "serving set-up");
    }
    s->slot_busy.assign(kSlots, false);
    s->inflight_per_stream.assign(cfg->n_streams, 0);
    sc5_server_s *raw = s.get();
    s->sched = std::thread([raw] { raw->scheduler_loop(); });
    s->compl_ = std::thread([raw] { raw->completion_loop(); });
    *out = s.release();
    return SC5_OK;
}

extern "C" sc5_status serve_submit(sc5_server srv, const sc5_image *req, uint64_t *ticket)
{
    clear_error();
    if (!srv || !req || !ticket) return fail(SC5_EINVAL, "null argument");
    const sc5_image &im = *req;
    const int es = dtype_bytes(srv->cfg.dtype);
    if (!im.in || !im.out) return fail(SC5_EINVAL, "null image pointer");
    if (im.H < 5 || im.W < 5 || im.H > 65535 * 8 || im.W > (1 << 30) || im.in_pitch < im.W ||
        im.out_pitch < im.W - 4 || (im.in_pitch * es) % 16)
        return fail(SC5_EINVAL, "bad shape: 5 <= H <= 524280, 5 <= W <= 2^30, in_pitch >= W with in_pitch * "
                                "element size a multiple of 16, out_pitch >= W-4");
    if (!(im.in_scale > 0.f) || !std::isfinite(im.in_scale) || !(im.out_scale > 0.f) || !std::isfinite(im.out_scale))
        return fail(SC5_EINVAL, "scales must be finite and > 0");
    for (float t : im.k)
        if (!std::isfinite(t)) return fail(SC5_EINVAL, "taps must be finite");
    auto r = std::make_shared<Request>();
    r->img = im;
    r->in_bytes = static_cast<size_t>(srv->cfg.planes) * im.H * im.in_pitch * es;
    r->out_bytes = static_cast<size_t>(srv->cfg.planes) * (im.H - 4) * im.out_pitch * es;
    if (srv->need_bytes(im) > srv->cfg.hbm_budget_bytes)
        return fail(SC5_EINVAL, "request needs %zu bytes, more than the whole budget", srv->need_bytes(im));
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->stop) return fail(SC5_EINVAL, "server is shutting down");
    if (static_cast<int>(srv->pending.size()) >= kMaxQueued) {
        ++srv->stats.rejected;
        return fail(SC5_EAGAIN, "queue full (%d pending)", kMaxQueued);
    }
    r->id = srv->next_id++;
    r->t_submit = Clock::now();
    srv->pending.push_back(r);
    srv->tickets[r->id] = r;
    ++srv->stats.submitted;
    *ticket = r->id;
    srv->cv_sched.notify_one();
    return SC5_OK;
}

extern "C" sc5_status serve_poll(sc5_server srv, uint64_t ticket, int32_t timeout_us, double *latency_us)
{
    clear_error();
    if (!srv) return fail(SC5_EINVAL, "null server");
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->tickets.find(ticket);
    if (it == srv->tickets.end()) return fail(SC5_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    auto r = it->second;
    auto ready = [&] { return r->done; };
    if (timeout_us < 0) {
        srv->cv_done.wait(lk, ready);
    } else if (timeout_us > 0) {
        srv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready);
    }
    if (!r->done) return timeout_us == 0 ? SC5_EAGAIN : SC5_ETIMEDOUT;
    srv->tickets.erase(it);
    if (latency_us)
        *latency_us = std::chrono::duration<double, std::micro>(r->t_done - r->t_submit).count();
    if (r->status != SC5_OK) return fail(r->status, "request %llu failed", (unsigned long long)ticket);
    return SC5_OK;
}

extern "C" sc5_status serve_get_stats(sc5_server srv, sc5_serve_stats *stats)
{
    clear_error();
    if (!srv || !stats) return fail(SC5_EINVAL, "null argument");
    std::vector<float> q, s, r;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        *stats = srv->stats;
        q = srv->phases.q;
        s = srv->phases.s;
        r = srv->phases.r;
    }
    stats->queue_us_p50 = PhaseLog::pct(q, 50);
    stats->queue_us_p99 = PhaseLog::pct(q, 99);
    stats->stage_us_p50 = PhaseLog::pct(s, 50);
    stats->stage_us_p99 = PhaseLog::pct(s, 99);
    stats->run_us_p50 = PhaseLog::pct(r, 50);
    stats->run_us_p99 = PhaseLog::pct(r, 99);
    return SC5_OK;
}

extern "C" sc5_status serve_destroy(sc5_server srv)
{
    clear_error();
    if (!srv) return SC5_OK;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv_sched.notify_all();
    if (srv->sched.joinable()) srv->sched.join();
    if (srv->compl_.joinable()) srv->compl_.join();
    cudaSetDevice(srv->device);
    cudaStreamSynchronize(srv->s_d2h);
    for (auto st : srv->s_comp) cudaStreamDestroy(st);
    cudaStreamDestroy(srv->s_h2d);
    cudaStreamDestroy(srv->s_d2h);
    for (auto e : srv->event_pool) cudaEventDestroy(e);
    cudaFree(srv->arena_base);
    cudaFree(srv->slot_dev);
    cudaFreeHost(srv->slot_host);
    delete srv;
    return SC5_OK;
}
