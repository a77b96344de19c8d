// Randomised check of the device store's range allocator (host code of the
// batched and serving solvers) against a per-cell occupancy model: every
// allocation is the first aligned fit in address order, never overlaps a
// live range, and frees coalesce, so that after all releases the whole
// capacity is one free range again.  Links libadmm.so; needs no GPU.
#include <cstdint>
#include <cstdio>
#include <random>
#include <vector>

#include "store.h"

using admm_impl::RangeAlloc;

namespace {

int64_t first_fit(const std::vector<char> &used, int64_t len, int64_t align)
{
    const int64_t cap = (int64_t)used.size();
    int64_t s = 0;
    while (s < cap) {
        if (used[s]) { ++s; continue; }
        int64_t e = s;
        while (e < cap && !used[e]) ++e;            // maximal free run [s, e)
        const int64_t a = (s + align - 1) / align * align;
        if (a + len <= e) return a;
        s = e;
    }
    return -1;
}

void model_stats(const std::vector<char> &used, int64_t &free_cells, int64_t &longest)
{
    free_cells = longest = 0;
    int64_t run = 0;
    for (char u : used) {
        run = u ? 0 : run + 1;
        free_cells += !u;
        if (run > longest) longest = run;
    }
}

} // namespace

int main(int argc, char **argv)
{
    const unsigned seed = argc > 1 ? (unsigned)std::atoi(argv[1]) : 1u;
    std::mt19937_64 rng(seed);
    const int64_t cap = 4096;
    RangeAlloc ra;
    ra.init(cap);
    std::vector<char> used(cap, 0);
    struct Live { int64_t off, len; };
    std::vector<Live> live;
    int64_t fails = 0, allocs = 0;
    for (int op = 0; op < 20000; ++op) {
        const bool do_alloc = live.empty() || rng() % 100 < 55;
        if (do_alloc) {
            const int64_t len = 1 + (int64_t)(rng() % 300);
            const int64_t align = (rng() % 2) ? 4 : 1;
            const int64_t want = first_fit(used, len, align);
            const int64_t got = ra.alloc(len, align);
            if (got != want) {
                std::fprintf(stderr, "op %d: alloc(%lld, %lld) = %lld, first fit %lld\n", op, (long long)len,
                             (long long)align, (long long)got, (long long)want);
                return 1;
            }
            if (got < 0) { ++fails; continue; }
            ++allocs;
            for (int64_t t = got; t < got + len; ++t) used[t] = 1;
            live.push_back({got, len});
        } else {
            const size_t k = (size_t)(rng() % live.size());
            ra.release(live[k].off, live[k].len);
            for (int64_t t = live[k].off; t < live[k].off + live[k].len; ++t) used[t] = 0;
            live[k] = live.back();
            live.pop_back();
        }
        int64_t fc, lg;
        model_stats(used, fc, lg);
        if (ra.free_total() != fc || ra.largest_free() != lg) {
            std::fprintf(stderr, "op %d: free %lld / %lld, largest %lld / %lld\n", op, (long long)ra.free_total(),
                         (long long)fc, (long long)ra.largest_free(), (long long)lg);
            return 1;
        }
    }
    for (const Live &l : live) ra.release(l.off, l.len);
    if (ra.free_total() != cap || ra.largest_free() != cap) {
        std::fprintf(stderr, "not one free range after releasing everything\n");
        return 1;
    }
    if (fails == 0 || allocs < 1000) {
        std::fprintf(stderr, "the run did not exercise a full store (%lld fails, %lld allocs)\n", (long long)fails,
                     (long long)allocs);
        return 1;
    }
    std::printf("range allocator ok: %lld allocations, %lld refused\n", (long long)allocs, (long long)fails);
    return 0;
}
