// Host-only check of the request server's arena bookkeeping (tl_arena.h):
// random alloc/release sequences against a byte-map model.  Prints "ok" or
// the first violation and exits non-zero.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "tl_arena.h"

int main()
{
    const size_t cap = 1 << 20;
    tl::Arena a(cap + 100);  // capacity rounds down to the alignment
    if (a.capacity() != cap) { std::printf("capacity %zu\n", a.capacity()); return 1; }
    std::vector<int> owner(cap / tl::Arena::kAlign, -1);
    struct Blk { size_t off, bytes; bool live; };
    std::vector<Blk> blks;
    std::mt19937_64 g(7);
    for (int step = 0; step < 200000; ++step) {
        const bool do_alloc = blks.empty() || (g() % 100) < 55;
        if (do_alloc) {
            const size_t bytes = (g() % 3 == 0) ? g() % 300 : g() % 40000;
            const size_t off = a.alloc(bytes);
            const size_t len = tl::Arena::round_up(bytes ? bytes : 1);
            if (off == SIZE_MAX) {
                // refusal is only allowed when no free run of the model fits
                size_t run = 0, best = 0;
                for (int o : owner) { run = (o < 0) ? run + 1 : 0; best = run > best ? run : best; }
                if (best * tl::Arena::kAlign >= len) { std::printf("refused %zu with a %zu run\n", len, best); return 1; }
                if (a.largest_free() >= len) { std::printf("largest_free inconsistent\n"); return 1; }
                continue;
            }
            if (off % tl::Arena::kAlign || off + len > cap) { std::printf("bad range %zu+%zu\n", off, len); return 1; }
            for (size_t u = off / tl::Arena::kAlign; u < (off + len) / tl::Arena::kAlign; ++u) {
                if (owner[u] >= 0) { std::printf("overlap at %zu\n", u); return 1; }
                owner[u] = static_cast<int>(blks.size());
            }
            blks.push_back({off, bytes, true});
        } else {
            const size_t k = g() % blks.size();
            if (!blks[k].live) continue;
            const size_t len = tl::Arena::round_up(blks[k].bytes ? blks[k].bytes : 1);
            for (size_t u = blks[k].off / tl::Arena::kAlign; u < (blks[k].off + len) / tl::Arena::kAlign; ++u) owner[u] = -1;
            a.release(blks[k].off, blks[k].bytes);
            blks[k].live = false;
        }
        size_t used = 0;
        if (step % 997 == 0) {
            for (int o : owner) used += (o >= 0) ? tl::Arena::kAlign : 0;
            if (used != a.used()) { std::printf("used %zu vs %zu\n", a.used(), used); return 1; }
        }
    }
    for (auto &b : blks)
        if (b.live) a.release(b.off, b.bytes);
    if (a.used() != 0 || a.free_ranges() != 1 || a.largest_free() != cap) {
        std::printf("not coalesced: %zu ranges\n", a.free_ranges());
        return 1;
    }
    if (a.high_water() == 0 || a.high_water() > cap) { std::printf("high water %zu\n", a.high_water()); return 1; }
    std::printf("ok\n");
    return 0;
}
