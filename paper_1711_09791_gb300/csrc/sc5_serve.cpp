// sc5_serve.cpp -- serving runtime: continuous batching of convolution
// requests on one GPU.
//
// Requests (page-locked host images of any size, each with its own 5 taps)
// are queued by serve_submit.  A scheduler thread admits them in arrival
// order while the resident arena (one device allocation of hbm_budget_bytes
// made at start) has room for their input and output and fewer than
// max_inflight are admitted, and issues each admitted request's input copy
// on the copy stream at once.  Everything admitted in one pass of the
// scheduler (or, with a batching window, within the window) goes out as one
// persistent launch of the fused batch kernel (per-image descriptors + tile
// work-list, up to max_merge requests), issued on the next of n_streams
// compute streams behind device-side waits on those requests' input copies:
// the kernel starts the moment the last input lands, with no host round
// trip.  Behind the kernel, each request's output values (not the rows'
// padding) are copied back to its host buffer on a second copy stream,
// smallest request first, and an event is recorded after each copy.
//
// No lock is held while a CUDA call is issued.  A completion thread waits on
// those events in the order the copies were issued (blocking-sync events:
// the thread sleeps until the copy lands, there is no polling loop), and
// completes each request on its own: time stamp, arena blocks freed (which
// lets waiting requests in), ticket marked done.  A launch's descriptor
// block is freed with its last request.  Each tile's arithmetic does not
// depend on what else is in the launch, so a request's result is the same
// alone and in any mix.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "sc5_internal.h"
#include "sc5_serve_host.h"
#include "sc5_tune.h"

namespace sc5 {

using Clock = std::chrono::steady_clock;

namespace {

constexpr size_t kDescBytes = 64u << 20;       // descriptor + work-list area (device, pinned host mirror)
constexpr size_t kLaunchDescCap = 8u << 20;    // descriptor bytes one merged launch may take
constexpr int kMaxQueued = 1 << 16;            // pending requests before back-pressure

struct Launch {
    size_t desc_off = 0, desc_bytes = 0;  // block of the descriptor area (bytes 0: none)
    int remaining = 0;                    // requests of the launch not yet completed
};

struct Request {
    uint64_t id = 0;
    sc5_image img{};  // host pointers
    size_t in_bytes = 0, out_bytes = 0;
    size_t in_off = 0, out_off = 0;
    Clock::time_point t_submit, t_admit, t_launch, t_done;
    cudaEvent_t h2d = nullptr;   // the input copy has landed
    cudaEvent_t done_ev = nullptr;  // the output copy has landed (blocking sync)
    std::shared_ptr<Launch> launch;
    bool done = false;
    sc5_status status = SC5_OK;
};

bool is_page_locked(const void *p)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // clear the error the query may leave
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

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
    unsigned char *desc_dev = nullptr;
    unsigned char *desc_host = nullptr;
    Arena desc_arena;

    std::mutex ev_mu;  // event pools (scheduler and completion threads)
    std::vector<cudaEvent_t> plain_events, blocking_events;

    std::mutex mu;
    std::condition_variable cv_sched, cv_done, cv_compl;
    std::deque<std::shared_ptr<Request>> pending;      // submitted, not admitted
    std::deque<std::shared_ptr<Request>> issued;       // output copy issued, not completed (issue order)
    std::unordered_map<uint64_t, std::shared_ptr<Request>> tickets;
    uint64_t next_id = 1;
    int admitted = 0;
    bool stop = false, sched_done = false;
    sc5_serve_stats stats{};
    std::thread sched, compl_;
    int fault_sched_delay_ms = 0;  // host-side fault injection (SC5_SERVE_FAULT)
    PhaseLog phases;

    // scheduler-thread state (no lock)
    std::vector<std::shared_ptr<Request>> staged;  // input copy issued, not launched
    Clock::time_point staged_since;
    int next_stream = 0;

    cudaEvent_t get_event(bool blocking)
    {
        {
            std::lock_guard<std::mutex> lk(ev_mu);
            auto &pool = blocking ? blocking_events : plain_events;
            if (!pool.empty()) {
                cudaEvent_t e = pool.back();
                pool.pop_back();
                return e;
            }
        }
        cudaEvent_t e = nullptr;
        cudaEventCreateWithFlags(&e, cudaEventDisableTiming | (blocking ? cudaEventBlockingSync : 0));
        return e;
    }
    void put_event(cudaEvent_t e, bool blocking)
    {
        if (!e) return;
        std::lock_guard<std::mutex> lk(ev_mu);
        (blocking ? blocking_events : plain_events).push_back(e);
    }

    size_t need_bytes(const sc5_image &im) const
    {
        const int es = dtype_bytes(cfg.dtype);
        return round_up(static_cast<size_t>(cfg.planes) * im.H * im.in_pitch * es, kArenaAlign) +
               round_up(static_cast<size_t>(cfg.planes) * (im.H - 4) * im.out_pitch * es, kArenaAlign);
    }

    void scheduler_loop();
    void completion_loop();
    void launch_group(std::vector<std::shared_ptr<Request>> group);
};

void sc5_server_s::scheduler_loop()
{
    cudaSetDevice(device);
    const int es = dtype_bytes(cfg.dtype);
    for (;;) {
        // 1. admission, in arrival order (under the lock: no CUDA calls)
        std::vector<std::shared_ptr<Request>> admit;
        bool stopping = false;
        {
            std::unique_lock<std::mutex> lk(mu);
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
                admit.push_back(r);
            }
            stopping = stop;
            if (admit.empty() && staged.empty()) {
                if (stopping && pending.empty()) break;
                // nothing to do until a submit, a completion (arena space) or stop
                cv_sched.wait_for(lk, std::chrono::milliseconds(50));
                continue;
            }
        }
        // 2. input copies, issued at once on the copy stream
        for (auto &r : admit) {
            r->h2d = get_event(false);
            cudaMemcpyAsync(arena_base + r->in_off, r->img.in,
                            static_cast<size_t>(cfg.planes) * r->img.H * r->img.in_pitch * es,
                            cudaMemcpyHostToDevice, s_h2d);
            cudaEventRecord(r->h2d, s_h2d);
            if (staged.empty()) staged_since = Clock::now();
            staged.push_back(r);
        }
        // 3. merge what is staged into launches (all of it at once, up to
        // max_merge per launch), unless a batching window holds it a little
        // longer
        while (!staged.empty()) {
            const bool window_over =
                !cfg.merge || cfg.batch_window_us <= 0 || stopping ||
                (cfg.max_merge > 0 && static_cast<int>(staged.size()) >= cfg.max_merge) ||
                Clock::now() - staged_since >= std::chrono::microseconds(cfg.batch_window_us);
            if (!window_over) break;
            const size_t cap = !cfg.merge ? 1 : cfg.max_merge > 0 ? static_cast<size_t>(cfg.max_merge) : staged.size();
            std::vector<std::shared_ptr<Request>> group;
            size_t bytes = 0, taken = 0;
            for (; taken < staged.size() && group.size() < cap; ++taken) {
                const auto &r = staged[taken];
                // upper bound on this image's share: descriptor + smallest-tile work-list
                const size_t tiles =
                    static_cast<size_t>(cfg.planes) * ((r->img.H - 4 + 31) / 32) * ((r->img.W - 4 + 127) / 128);
                const size_t add = sizeof(ImgDesc) + tiles * sizeof(TileRec);
                if (!group.empty() && bytes + add + kArenaAlign > kLaunchDescCap) break;
                bytes += add;
                group.push_back(r);
            }
            staged.erase(staged.begin(), staged.begin() + static_cast<std::ptrdiff_t>(taken));
            if (!staged.empty()) staged_since = Clock::now();
            launch_group(std::move(group));
        }
        if (!staged.empty()) {
            // a batching window is open: come back when it closes (or earlier on a submit)
            std::unique_lock<std::mutex> lk(mu);
            const auto left = std::chrono::microseconds(cfg.batch_window_us) - (Clock::now() - staged_since);
            if (left > Clock::duration::zero() && !stop) cv_sched.wait_for(lk, left);
        }
    }
    std::lock_guard<std::mutex> lk(mu);
    sched_done = true;
    cv_compl.notify_all();
}

void sc5_server_s::launch_group(std::vector<std::shared_ptr<Request>> group)
{
    const int es = dtype_bytes(cfg.dtype);
    std::vector<sc5_image> imgs;
    imgs.reserve(group.size());
    for (auto &r : group) {
        sc5_image d = r->img;
        d.in = arena_base + r->in_off;
        d.out = arena_base + r->out_off;
        imgs.push_back(d);
    }
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
    if (st == SC5_OK && blob.size() > kLaunchDescCap) st = SC5_ENOMEM;
    auto L = std::make_shared<Launch>();
    L->remaining = static_cast<int>(group.size());
    if (st == SC5_OK) {
        // a block of the descriptor area: wait for earlier launches to retire if it is full
        std::unique_lock<std::mutex> lk(mu);
        while (!desc_arena.alloc(blob.size(), &L->desc_off)) {
            if (issued.empty()) {  // nothing in flight will free space: cannot happen below the cap
                st = SC5_ENOMEM;
                break;
            }
            cv_sched.wait_for(lk, std::chrono::milliseconds(1));
        }
        if (st == SC5_OK) L->desc_bytes = blob.size();
    }
    const int s = next_stream;
    next_stream = (next_stream + 1) % static_cast<int>(s_comp.size());
    cudaStream_t cs = s_comp[s];
    const auto t_launch = Clock::now();
    for (auto &r : group) {
        r->t_launch = t_launch;
        r->launch = L;
    }
    // outputs go back smallest first, so that small requests do not wait
    // behind a large one of the same launch
    std::stable_sort(group.begin(), group.end(),
                     [](const std::shared_ptr<Request> &a, const std::shared_ptr<Request> &b) {
                         return a->out_bytes < b->out_bytes;
                     });
    if (st == SC5_OK) {
        unsigned char *hs = desc_host + L->desc_off;
        unsigned char *ds = desc_dev + L->desc_off;
        std::memcpy(hs, blob.data(), blob.size());
        cudaMemcpyAsync(ds, hs, blob.size(), cudaMemcpyHostToDevice, cs);
        for (auto &r : group) cudaStreamWaitEvent(cs, r->h2d, 0);
        const int64_t capc = static_cast<int64_t>(num_sms()) * ctas;
        const int grid = static_cast<int>(std::max<int64_t>(1, std::min(ntiles, capc)));
        cudaError_t e = launch_fused_batch(cfg.dtype, cfg.dtype, idx, reinterpret_cast<const ImgDesc *>(ds),
                                           reinterpret_cast<const TileRec *>(ds + toff), ntiles, grid, cs);
        if (e != cudaSuccess) st = SC5_ECUDA;
    }
    if (st == SC5_OK) {
        cudaEvent_t kdone = get_event(false);
        cudaEventRecord(kdone, cs);
        cudaStreamWaitEvent(s_d2h, kdone, 0);
        // results go back as their W-4 valid values per row: the caller's row
        // padding is left as it was, as sepconv5_run leaves it
        for (auto &r : group) {
            const size_t pitch_b = static_cast<size_t>(r->img.out_pitch) * es;
            cudaMemcpy2DAsync(r->img.out, pitch_b, arena_base + r->out_off, pitch_b,
                              static_cast<size_t>(r->img.W - 4) * es,
                              static_cast<size_t>(cfg.planes) * (r->img.H - 4), cudaMemcpyDeviceToHost, s_d2h);
            r->done_ev = get_event(true);
            cudaEventRecord(r->done_ev, s_d2h);
        }
        put_event(kdone, false);  // its record and the wait on it are already enqueued
    } else {
        // nothing was launched: the requests complete with the error once
        // their input copies (which still write the arena) have landed
        for (auto &r : group) cudaStreamWaitEvent(cs, r->h2d, 0);
        for (auto &r : group) {
            r->status = st;
            r->done_ev = get_event(true);
            cudaEventRecord(r->done_ev, cs);
        }
    }
    for (auto &r : group) {  // the waits on the input copies are enqueued
        put_event(r->h2d, false);
        r->h2d = nullptr;
    }
    {
        std::lock_guard<std::mutex> lk(mu);
        for (auto &r : group) issued.push_back(r);
        ++stats.launches;
        stats.merged_max = std::max<uint64_t>(stats.merged_max, group.size());
    }
    cv_compl.notify_one();
}

void sc5_server_s::completion_loop()
{
    cudaSetDevice(device);
    for (;;) {
        std::shared_ptr<Request> r;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_compl.wait(lk, [&] { return !issued.empty() || sched_done; });
            if (issued.empty()) break;  // the scheduler has finished and everything completed
            r = issued.front();
        }
        // sleeps until the copy lands (blocking-sync event); outside the lock.
        // (Spinning on cudaEventQuery instead measured no shorter tail.)
        const cudaError_t q = cudaEventSynchronize(r->done_ev);
        const auto now = Clock::now();
        {
            std::lock_guard<std::mutex> lk(mu);
            issued.pop_front();
            if (q != cudaSuccess && r->status == SC5_OK) r->status = SC5_ECUDA;
            r->t_done = now;
            r->done = true;
            phases.add(r->t_admit - r->t_submit, r->t_launch - r->t_admit, now - r->t_launch);
            arena.release(r->in_off, r->in_bytes);
            arena.release(r->out_off, r->out_bytes);
            --admitted;
            ++stats.completed;
            if (--r->launch->remaining == 0 && r->launch->desc_bytes)
                desc_arena.release(r->launch->desc_off, r->launch->desc_bytes);
            r->launch.reset();
        }
        put_event(r->done_ev, true);
        r->done_ev = nullptr;
        cv_done.notify_all();
        cv_sched.notify_all();
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
    e = cudaMalloc(&s->desc_dev, kDescBytes);
    if (e == cudaSuccess) e = cudaMallocHost(&s->desc_host, kDescBytes);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->s_h2d, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->s_d2h, cudaStreamNonBlocking);
    for (int i = 0; i < cfg->n_streams && e == cudaSuccess; ++i) {
        cudaStream_t st;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e == cudaSuccess) s->s_comp.push_back(st);
    }
    if (e != cudaSuccess) {
        for (auto st : s->s_comp) cudaStreamDestroy(st);
        if (s->s_h2d) cudaStreamDestroy(s->s_h2d);
        if (s->s_d2h) cudaStreamDestroy(s->s_d2h);
        cudaFree(s->arena_base);
        cudaFree(s->desc_dev);
        cudaFreeHost(s->desc_host);
        return fail_cuda(e, "serving set-up");
    }
    s->desc_arena.reset(kDescBytes);
    // Warm-up, so that the first requests do not pay it: touch the arena and
    // the descriptor area once, load every compiled batch-kernel shape of the
    // dtype and set its attributes, and fill the event pools.
    e = cudaMemsetAsync(s->arena_base, 0, cfg->hbm_budget_bytes, s->s_h2d);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->desc_dev, 0, kDescBytes, s->s_h2d);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->s_h2d);
    tune_from_environment(cfg->dtype, cfg->dtype);  // here rather than on the scheduler thread
    for (int i = 0; i < fused_num_shapes(cfg->dtype, cfg->dtype) && e == cudaSuccess; ++i)
        e = fused_prepare(cfg->dtype, cfg->dtype, i);
    for (int i = 0; i < 2 * cfg->max_inflight && e == cudaSuccess; ++i) {
        cudaEvent_t a = nullptr, b = nullptr;
        e = cudaEventCreateWithFlags(&a, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b, cudaEventDisableTiming | cudaEventBlockingSync);
        if (a) s->plain_events.push_back(a);
        if (b) s->blocking_events.push_back(b);
    }
    if (e != cudaSuccess) {
        for (auto ev : s->plain_events) cudaEventDestroy(ev);
        for (auto ev : s->blocking_events) cudaEventDestroy(ev);
        for (auto st : s->s_comp) cudaStreamDestroy(st);
        cudaStreamDestroy(s->s_h2d);
        cudaStreamDestroy(s->s_d2h);
        cudaFree(s->arena_base);
        cudaFree(s->desc_dev);
        cudaFreeHost(s->desc_host);
        return fail_cuda(e, "serving warm-up");
    }
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
    if (!is_page_locked(im.in) || !is_page_locked(im.out))
        return fail(SC5_EINVAL, "host buffers must be page-locked (cudaMallocHost or cudaHostRegister): copies "
                                "from or to pageable memory block the scheduler");
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
    for (auto st : srv->s_comp) cudaStreamSynchronize(st);
    cudaStreamSynchronize(srv->s_h2d);
    cudaStreamSynchronize(srv->s_d2h);
    for (auto st : srv->s_comp) cudaStreamDestroy(st);
    cudaStreamDestroy(srv->s_h2d);
    cudaStreamDestroy(srv->s_d2h);
    for (auto e : srv->plain_events) cudaEventDestroy(e);
    for (auto e : srv->blocking_events) cudaEventDestroy(e);
    cudaFree(srv->arena_base);
    cudaFree(srv->desc_dev);
    cudaFreeHost(srv->desc_host);
    delete srv;
    return SC5_OK;
}
