// sc5_serve_host.h -- the host-only parts of the serving runtime: the
// first-fit allocator over the resident arena and the ring of per-request
// phase durations with its nearest-rank percentiles.  Plain C++17 with no
// CUDA dependency, so that the host tests compile and check them directly.
#pragma once

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstddef>
#include <map>
#include <vector>

namespace sc5 {

constexpr size_t kArenaAlign = 256;

inline size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// First-fit allocator over [0, size) in kArenaAlign units, with coalescing of
// adjacent free blocks on release.
class Arena {
public:
    void reset(size_t size)
    {
        free_.clear();
        free_[0] = size;
        used_ = 0;
        size_ = size;
    }
    bool alloc(size_t n, size_t *off)
    {
        n = round_up(n, kArenaAlign);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                const size_t rest = it->second - n;
                const size_t start = it->first + n;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_ += n;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t n)
    {
        n = round_up(n, kArenaAlign);
        used_ -= n;
        auto it = free_.emplace(off, n).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }
    size_t size() const { return size_; }
    size_t free_blocks() const { return free_.size(); }

private:
    std::map<size_t, size_t> free_;  // offset -> length of each free block
    size_t used_ = 0, size_ = 0;
};

// Phase durations of the last kPhaseLog completed requests (a ring).
struct PhaseLog {
    using Clock = std::chrono::steady_clock;
    static constexpr size_t kPhaseLog = size_t(1) << 20;
    std::vector<float> q, s, r;  // queue, stage, run (microseconds)
    size_t n = 0;
    static float us(Clock::duration d) { return std::chrono::duration<float, std::micro>(d).count(); }
    void add(Clock::duration dq, Clock::duration ds, Clock::duration dr)
    {
        if (q.size() < kPhaseLog) {
            q.push_back(us(dq));
            s.push_back(us(ds));
            r.push_back(us(dr));
        } else {
            const size_t i = n % kPhaseLog;
            q[i] = us(dq);
            s[i] = us(ds);
            r[i] = us(dr);
        }
        ++n;
    }
    // p-th percentile (nearest rank: the ceil(p/100 * n)-th smallest) of a
    // copy of v; 0 if empty.
    static double pct(std::vector<float> v, double p)
    {
        if (v.empty()) return 0.0;
        size_t k = static_cast<size_t>(std::ceil(p / 100.0 * v.size()));
        k = k ? k - 1 : 0;
        if (k >= v.size()) k = v.size() - 1;
        std::nth_element(v.begin(), v.begin() + static_cast<std::ptrdiff_t>(k), v.end());
        return v[k];
    }
};

}  // namespace sc5
