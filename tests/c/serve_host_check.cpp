// Checks of the serving runtime's host-only parts (sc5_serve_host.h), with no
// GPU: the arena allocator against a byte-level model of the arena under a
// seeded random sequence of allocations and releases, and the phase log's
// nearest-rank percentiles against a sorted copy.  Prints OK or the first
// failure; exit status 0 only on OK.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "sc5_serve_host.h"

using sc5::Arena;
using sc5::kArenaAlign;
using sc5::PhaseLog;

static int fails = 0;
#define CHECK(c, ...)                                  \
    do {                                               \
        if (!(c)) {                                    \
            if (!fails) std::printf(__VA_ARGS__);      \
            if (!fails) std::printf("\n");             \
            ++fails;                                   \
        }                                              \
    } while (0)

struct Block {
    size_t off, n;
};

// The model: one owner id per arena unit (0 = free).
static bool model_free(const std::vector<int> &owner, size_t off, size_t units)
{
    for (size_t u = off; u < off + units; ++u)
        if (u >= owner.size() || owner[u]) return false;
    return true;
}

static void check_arena(unsigned seed)
{
    const size_t units = 4096;
    Arena a;
    a.reset(units * kArenaAlign);
    std::vector<int> owner(units, 0);
    std::vector<Block> live;
    std::mt19937 g(seed);
    int id = 0;
    for (int step = 0; step < 20000 && !fails; ++step) {
        const bool do_alloc = live.empty() || (g() % 100) < 55;
        if (do_alloc) {
            // sizes of 1 byte to 300 units, not multiples of the alignment
            const size_t bytes = 1 + g() % (300 * kArenaAlign);
            const size_t need = (bytes + kArenaAlign - 1) / kArenaAlign;
            // first fit in the model: the lowest offset with `need` free units
            size_t first = units;
            for (size_t u = 0, run = 0; u < units; ++u) {
                run = owner[u] ? 0 : run + 1;
                if (run == need) {
                    first = u + 1 - need;
                    break;
                }
            }
            size_t off = 0;
            const bool ok = a.alloc(bytes, &off);
            if (first == units) {
                // no free run is long enough in the model: the arena must refuse
                CHECK(!ok, "seed %u step %d: alloc of %zu units succeeded with no free run", seed, step, need);
                continue;
            }
            CHECK(ok, "seed %u step %d: alloc of %zu units refused with a free run at %zu", seed, step, need, first);
            if (!ok) continue;
            CHECK(off % kArenaAlign == 0, "seed %u: offset %zu not aligned", seed, off);
            CHECK(off / kArenaAlign == first, "seed %u step %d: offset %zu is not the first fit %zu", seed, step,
                  off / kArenaAlign, first);
            CHECK(model_free(owner, off / kArenaAlign, need), "seed %u step %d: block overlaps a live one", seed,
                  step);
            ++id;
            for (size_t u = off / kArenaAlign; u < off / kArenaAlign + need && u < units; ++u) owner[u] = id;
            live.push_back({off, bytes});
        } else {
            const size_t i = g() % live.size();
            const Block b = live[i];
            live[i] = live.back();
            live.pop_back();
            a.release(b.off, b.n);
            const size_t need = (b.n + kArenaAlign - 1) / kArenaAlign;
            for (size_t u = b.off / kArenaAlign; u < b.off / kArenaAlign + need; ++u) owner[u] = 0;
        }
        size_t used_units = 0;
        for (int o : owner) used_units += o != 0;
        CHECK(a.used() == used_units * kArenaAlign, "seed %u step %d: used %zu, model %zu", seed, step, a.used(),
              used_units * kArenaAlign);
        // coalescing: the arena keeps exactly one block per maximal free run
        size_t runs = 0;
        for (size_t u = 0; u < units; ++u) runs += !owner[u] && (u == 0 || owner[u - 1]);
        CHECK(a.free_blocks() == runs, "seed %u step %d: %zu free blocks, model has %zu free runs", seed, step,
              a.free_blocks(), runs);
    }
    for (const Block &b : live) a.release(b.off, b.n);
    CHECK(a.used() == 0 && a.free_blocks() == 1, "seed %u: after releasing everything used=%zu blocks=%zu", seed,
          a.used(), a.free_blocks());
    size_t off = 1;
    CHECK(a.alloc(units * kArenaAlign, &off) && off == 0, "seed %u: the whole arena is not one block again", seed);
    CHECK(!a.alloc(1, &off), "seed %u: allocation from a full arena succeeded", seed);
}

static void check_percentiles()
{
    CHECK(PhaseLog::pct({}, 50) == 0.0, "empty percentile is not 0");
    // 1..100 in a shuffled order: the p-th percentile by nearest rank is p
    std::vector<float> v;
    for (int i = 1; i <= 100; ++i) v.push_back(static_cast<float>(i));
    std::shuffle(v.begin(), v.end(), std::mt19937(7));
    for (int p : {1, 50, 99, 100}) CHECK(PhaseLog::pct(v, p) == p, "pct(1..100, %d) = %g", p, PhaseLog::pct(v, p));
    // four values: p50 is the 2nd smallest, p99 and p100 the largest, p0 the smallest
    const std::vector<float> w = {40.f, 10.f, 30.f, 20.f};
    CHECK(PhaseLog::pct(w, 50) == 20.f, "pct(w, 50) = %g", PhaseLog::pct(w, 50));
    CHECK(PhaseLog::pct(w, 99) == 40.f, "pct(w, 99) = %g", PhaseLog::pct(w, 99));
    CHECK(PhaseLog::pct(w, 0) == 10.f, "pct(w, 0) = %g", PhaseLog::pct(w, 0));
    // the ring keeps the last kPhaseLog entries
    PhaseLog log;
    using us = std::chrono::microseconds;
    const size_t extra = 5;
    for (size_t i = 0; i < PhaseLog::kPhaseLog + extra; ++i) log.add(us(i), us(2 * i), us(3 * i));
    CHECK(log.q.size() == PhaseLog::kPhaseLog && log.n == PhaseLog::kPhaseLog + extra, "ring size %zu, n %zu",
          log.q.size(), log.n);
    CHECK(log.q[0] == static_cast<float>(PhaseLog::kPhaseLog) && log.r[extra - 1] == 3.f * (PhaseLog::kPhaseLog + extra - 1) &&
              log.s[extra] == 2.f * extra,
          "ring overwrote the wrong entries");
}

int main()
{
    for (unsigned seed : {1u, 2u, 3u}) check_arena(seed);
    check_percentiles();
    if (!fails) std::printf("OK\n");
    return fails ? 1 : 0;
}
