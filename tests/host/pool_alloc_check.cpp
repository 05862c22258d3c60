// Randomised check of the serving loop's result-pool allocator against a
// brute-force model: a bitmap of units in which first fit is the lowest run of
// free units long enough.  Prints "ok" and exits 0, or prints the first
// disagreement and exits 1.
#include <cstdint>
#include <cstdio>
#include <random>
#include <vector>

#include "pool_alloc.h"

namespace {

struct Model {
    std::vector<bool> used;
    explicit Model(size_t n) : used(n, false) {}
    bool alloc(uint64_t len, uint64_t *off) {
        uint64_t run = 0;
        for (uint64_t i = 0; i < used.size(); ++i) {
            run = used[i] ? 0 : run + 1;
            if (run == len) {
                *off = i + 1 - len;
                for (uint64_t j = *off; j <= i; ++j) used[j] = true;
                return true;
            }
        }
        return false;
    }
    void release(uint64_t off, uint64_t len) {
        for (uint64_t j = off; j < off + len; ++j) used[j] = false;
    }
};

int fail(const char *what, long step) {
    std::printf("FAIL %s at step %ld\n", what, step);
    return 1;
}

}  // namespace

int main() {
    const uint64_t size = 4096;
    for (uint32_t seed = 1; seed <= 40; ++seed) {
        std::mt19937_64 rng(seed);
        bn::PoolAllocator pool(size);
        Model model(size);
        std::vector<std::pair<uint64_t, uint64_t>> live;  // (offset, length)
        for (long step = 0; step < 3000; ++step) {
            const bool do_alloc = live.empty() || rng() % 100 < 55;
            if (do_alloc) {
                const uint64_t len = 1 + rng() % (seed % 4 == 0 ? 600 : 97);
                uint64_t a = 0, b = 0;
                const bool ga = pool.alloc(len, &a), gb = model.alloc(len, &b);
                if (ga != gb) return fail("alloc success differs", step);
                if (ga) {
                    if (a != b) return fail("first-fit offset differs", step);
                    if (a + len > size) return fail("block beyond the pool", step);
                    live.push_back({a, len});
                }
            } else {
                const size_t k = rng() % live.size();
                pool.release(live[k].first, live[k].second);
                model.release(live[k].first, live[k].second);
                live[k] = live.back();
                live.pop_back();
            }
            uint64_t used = 0;
            for (auto &b : live) used += b.second;
            if (pool.used() != used) return fail("used bytes", step);
        }
        for (auto &b : live) pool.release(b.first, b.second);
        if (pool.used() != 0 || pool.free_blocks() != 1) return fail("free list not coalesced", -1);
        uint64_t off = 1;
        if (!pool.alloc(size, &off) || off != 0) return fail("whole pool after coalescing", -1);
        if (pool.high_water() != size) return fail("high water", -1);
    }
    bn::PoolAllocator empty(0);
    uint64_t off = 0;
    if (empty.alloc(1, &off)) return fail("empty pool", -1);
    bn::PoolAllocator one(8);
    if (one.alloc(0, &off)) return fail("zero-byte request", -1);
    std::printf("ok\n");
    return 0;
}
