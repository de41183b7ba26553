/*
 * baseline_cpu.cpp -- CPU comparison sorts beside the oracle (test and
 * benchmark infrastructure only, as the rest of this directory).
 *
 *   oracle_stdsort_pairs     std::stable_sort of (key, payload) pairs by key,
 *                            one thread: the library stable sort the paper
 *                            compares zSort with (section "Experimental
 *                            Results", Table 1)
 *   oracle_zsort_segmented_mt
 *                            the oracle's zSort of every segment of a batch,
 *                            the segments shared out over a pool of
 *                            std::thread workers (a batch of independent
 *                            arrays is the one place where host threads help
 *                            a sequential sort)
 */
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <thread>
#include <vector>

extern "C" int oracle_zsort_pairs(uint64_t *keys, uint32_t *vals, uint64_t n, void *trace);

namespace {
struct Pair {
    uint64_t key;
    uint32_t val;
};
}  // namespace

extern "C" int oracle_stdsort_pairs(uint64_t *keys, uint32_t *vals, uint64_t n)
{
    std::vector<Pair> p(n);
    for (uint64_t i = 0; i < n; i++) p[i] = Pair{keys[i], vals[i]};
    std::stable_sort(p.begin(), p.end(), [](const Pair &a, const Pair &b) { return a.key < b.key; });
    for (uint64_t i = 0; i < n; i++) {
        keys[i] = p[i].key;
        vals[i] = p[i].val;
    }
    return 0;
}

// Segment i is [off[i], off[i+1]); threads <= 0 means one per host core.
// Returns the number of threads used, or a negative code (-5: decreasing
// offsets, -1: a segment's sort failed).
extern "C" int oracle_zsort_segmented_mt(uint64_t *keys, uint32_t *vals, const uint64_t *off, uint64_t nseg,
                                         int threads)
{
    for (uint64_t s = 0; s < nseg; s++)
        if (off[s + 1] < off[s]) return -5;
    int t = threads > 0 ? threads : (int)std::thread::hardware_concurrency();
    if (t < 1) t = 1;
    std::atomic<uint64_t> next{0};
    std::atomic<int> failed{0};
    auto work = [&]() {
        for (;;) {
            const uint64_t s = next.fetch_add(1);
            if (s >= nseg) return;
            const uint64_t a = off[s], b = off[s + 1];
            if (oracle_zsort_pairs(keys + a, vals + a, b - a, nullptr) != 0) failed.store(1);
        }
    };
    std::vector<std::thread> pool;
    for (int i = 0; i < t; i++) pool.emplace_back(work);
    for (auto &th : pool) th.join();
    return failed.load() ? -1 : t;
}
