// Randomised check of the server's first-fit allocator against a byte map:
// blocks never overlap, stay inside the range and are aligned; accounting
// matches; freeing everything coalesces back to one block.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>
#include "arena.h"

int main() {
    const size_t N = 1 << 20;
    supra::OffsetArena a;
    a.reset(N + 100);   // rounds down to a multiple of 256
    if (a.size() != N) return printf("size %zu\n", a.size()), 1;
    std::vector<int> owner(N / 256, -1);
    std::vector<std::pair<size_t, size_t>> live;   // offset, bytes (rounded)
    std::mt19937_64 rng(7);
    size_t used = 0, peak = 0;
    for (int it = 0; it < 200000; ++it) {
        if (live.empty() || rng() % 3 != 0) {
            const size_t want = 1 + rng() % 40000;
            const size_t off = a.alloc(want);
            const size_t len = (want + 255) / 256 * 256;
            // brute force: does any free run of len bytes exist?
            size_t run = 0, first_fit = SIZE_MAX;
            for (size_t b = 0; b < owner.size(); ++b) {
                run = owner[b] < 0 ? run + 256 : 0;
                if (run >= len) { first_fit = (b + 1) * 256 - len; break; }
            }
            if (off == supra::OffsetArena::kNone) {
                if (first_fit != SIZE_MAX) return printf("missed a fit at %d\n", it), 1;
                continue;
            }
            if (off != first_fit) return printf("not first fit at %d: %zu vs %zu\n", it, off, first_fit), 1;
            if (off % 256 || off + len > N) return printf("bad block at %d\n", it), 1;
            for (size_t b = off / 256; b < (off + len) / 256; ++b) {
                if (owner[b] >= 0) return printf("overlap at %d\n", it), 1;
                owner[b] = it;
            }
            live.push_back({off, len});
            used += len;
            peak = std::max(peak, used);
        } else {
            const size_t k = rng() % live.size();
            a.free(live[k].first);
            for (size_t b = live[k].first / 256; b < (live[k].first + live[k].second) / 256; ++b) owner[b] = -1;
            used -= live[k].second;
            live[k] = live.back();
            live.pop_back();
        }
        if (a.used() != used || a.peak() != peak) return printf("accounting at %d\n", it), 1;
    }
    for (auto &l : live) a.free(l.first);
    a.free(12345);   // unknown offset: ignored
    if (a.used() != 0 || a.free_blocks() != 1 || a.largest_free() != N) return printf("no coalesce\n"), 1;
    printf("ok\n");
    return 0;
}
