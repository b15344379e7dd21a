// Host check of the request server's first-fit arena (heget_arena.h) against
// a byte-occupancy model: random allocate / release sequences, after every
// operation
//   - live ranges are 256-aligned, inside the arena and pairwise disjoint;
//   - the free list covers exactly the bytes no live range holds, with no
//     two free ranges adjacent (freed neighbours merge);
//   - an allocation fails only when no free range is long enough, and
//     succeeds at the lowest such range (first fit);
// and releasing everything leaves one free range, the whole arena.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "heget_arena.h"

static int failures = 0;
#define CHECK(c, ...)                                  \
    do {                                               \
        if (!(c)) {                                    \
            if (failures < 20) std::printf(__VA_ARGS__); \
            ++failures;                                \
        }                                              \
    } while (0)

struct Live { size_t off, n; };

static size_t round256(size_t n) { return (n + 255) & ~(size_t)255; }

static void check_state(const heget::Arena& A, const std::vector<Live>& live, int step) {
    std::vector<char> used(A.size, 0);
    for (const Live& l : live) {
        CHECK(l.off % 256 == 0, "step %d: offset %zu not 256-aligned\n", step, l.off);
        CHECK(l.off + round256(l.n) <= A.size, "step %d: range %zu+%zu past the arena\n", step, l.off, l.n);
        for (size_t b = l.off; b < l.off + round256(l.n) && b < A.size; ++b) {
            CHECK(!used[b], "step %d: byte %zu held twice\n", step, b);
            used[b] = 1;
        }
    }
    size_t prev_end = (size_t)-1;
    std::vector<char> freeb(A.size, 0);
    for (const auto& f : A.free_) {
        CHECK(f.second > 0, "step %d: empty free range at %zu\n", step, f.first);
        CHECK(f.first != prev_end, "step %d: free ranges not merged at %zu\n", step, f.first);
        prev_end = f.first + f.second;
        for (size_t b = f.first; b < f.first + f.second && b < A.size; ++b) freeb[b] = 1;
    }
    for (size_t b = 0; b < A.size; ++b)
        CHECK(freeb[b] != used[b], "step %d: byte %zu is %s\n", step, b, used[b] ? "held and free" : "lost");
}

int main() {
    std::mt19937_64 rng(0x0908440300000A4Aull);
    for (int trial = 0; trial < 40; ++trial) {
        heget::Arena A;
        const size_t size = 256 * (8 + rng() % 200) + (trial % 3 == 0 ? rng() % 256 : 0);   // ragged sizes too
        A.init(size);
        std::vector<Live> live;
        for (int step = 0; step < 400; ++step) {
            if (!live.empty() && rng() % 5 < 2) {
                const size_t k = rng() % live.size();
                A.release(live[k].off, live[k].n);
                live.erase(live.begin() + (long)k);
            } else {
                const size_t n = 1 + rng() % (size / 6 + 1);
                // the first free range long enough, from the model's point of view
                size_t expect = (size_t)-1;
                for (const auto& f : A.free_)
                    if (f.second >= round256(n)) { expect = f.first; break; }
                size_t off = 0;
                const bool ok = A.alloc(n, &off);
                CHECK(ok == (expect != (size_t)-1), "trial %d step %d: alloc(%zu) returned %d\n", trial, step, n, ok);
                if (ok) {
                    CHECK(off == expect, "trial %d step %d: not first fit (%zu vs %zu)\n", trial, step, off, expect);
                    live.push_back({off, n});
                }
            }
            check_state(A, live, step);
        }
        for (const Live& l : live) A.release(l.off, l.n);
        live.clear();
        check_state(A, live, -1);
        CHECK(A.free_.size() == 1 && A.free_.begin()->first == 0 && A.free_.begin()->second == size,
              "trial %d: arena not whole after releasing everything\n", trial);
    }
    std::printf("arena checks: %d failures\n", failures);
    return failures ? 1 : 0;
}
