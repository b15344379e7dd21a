// Host-side checks of the kernels' index tables and shared-memory layouts
// (compiled and run by tests/test_layout.py; no GPU needed).  Exit status 0
// when every check holds; each failure prints one line.
#include <cstdio>

#include "heget_kernels.cuh"

using namespace heget;

static int failures = 0;
#define CHECK(cond, ...)                  \
    do {                                  \
        if (!(cond)) {                    \
            std::printf("FAIL: " __VA_ARGS__); \
            std::printf("\n");            \
            ++failures;                   \
        }                                 \
    } while (0)

static int popcount(unsigned x) { return __builtin_popcount(x); }

// pair / child index tables: consistent, ordered by set size, and every
// attach of the walk (sets of at most n - 2 photons with the two-ended
// finish) lands in the part of the table the rounds hold
static void check_tree_tables() {
    const TreeTables t = make_tree_tables();
    for (int n = kMinN; n <= kMaxN; ++n) {
        const int K = num_pairs(n), po = pair_offset(n), co = child_offset(n);
        int prev = 0;
        for (int idx = 0; idx < K; ++idx) {
            const int T = t.pair[po + idx] & 0xFF, j = t.pair[po + idx] >> 8;
            CHECK((T >> j) & 1, "n=%d pair %d: photon %d not in set %d", n, idx, j, T);
            CHECK(popcount(T) >= prev, "n=%d pair %d: not ordered by set size", n, idx);
            prev = popcount(T);
            CHECK(t.child[co + (T & ~(1 << j)) * n + j] == idx, "n=%d pair %d: child mismatch", n, idx);
        }
        const int KW = n >= 4 ? K - n * (n - 1) : K;
        for (int S = 0; S < (1 << n); ++S)
            for (int j = 0; j < n; ++j)
                if (!((S >> j) & 1) && popcount(S) <= n - 3)
                    CHECK(t.child[co + S * n + j] < KW, "n=%d: attach (%d, %d) beyond the held tables", n, S, j);
    }
}

// pair columns: the index of every (a, b, point, lambdas) entry lies in the table
template <class R, int N, int HB, int G, int BLOCK>
static void check_pair_columns() {
    using RT = RoundTables<R, N, BLOCK, HB, G>;
    if constexpr (tree_two_ended<R, N>()) {
        size_t hi = 0;
        for (int a = 0; a < N; ++a)
            for (int b = 0; b < N; ++b)
                if (a != b)
                    for (int p = 0; p < RT::P; ++p)
                        for (int l = 0; l < 4; ++l) {
                            const size_t e = ((size_t)pair_slot<N>(a, b) * RT::P + p) * 4 + l;
                            hi = e > hi ? e : hi;
                        }
        CHECK(hi < RT::p_elems, "n=%d: pair column index %zu of %zu", N, hi, RT::p_elems);
    }
}

static size_t resident_blocks(size_t smem_per_block) {
    const size_t per_sm = 228 * 1024, reserved = 1024;
    return per_sm / (smem_per_block + reserved);
}

int main() {
    check_tree_tables();
    check_pair_columns<float, 4, 0, 1, 256>();
    check_pair_columns<float, 5, 0, 1, 256>();
    check_pair_columns<float, 6, 1, 2, 128>();
    check_pair_columns<float, 7, 1, 2, 256>();
    check_pair_columns<float, 8, 1, 2, 256>();
    check_pair_columns<double, 4, 0, 1, 256>();
    check_pair_columns<double, 8, 0, 1, 256>();
    // occupancy the tuned launch shapes rely on
    const size_t draws4 = 2 * ws_stage(4) * sizeof(SampleDraw) + 256;
    const size_t ws4 = ws_smem_bytes<float, 4, kAlgTree>() + draws4;
    CHECK(resident_blocks(ws4) >= 2, "warp-specialised n=4 tree: %zu bytes, fewer than 2 blocks per SM", ws4);
    const size_t ws4s = ws_smem_bytes<float, 4, kAlgSubset>() + draws4;
    CHECK(resident_blocks(ws4s) >= 2, "warp-specialised n=4 subset: %zu bytes, fewer than 2 blocks per SM", ws4s);
    const size_t ws4e = ws_smem_bytes<float, 4, table_alg<kAlgTree, true>()>() + draws4;
    CHECK(resident_blocks(ws4e) >= 2, "warp-specialised n=4 tree with escalation: %zu bytes", ws4e);
    const size_t ws5 = ws_smem_bytes<float, 5, kAlgTree>() + 2 * ws_stage(5) * sizeof(SampleDraw) + 256;
    CHECK(resident_blocks(ws5) >= 2, "warp-specialised n=5 tree: %zu bytes", ws5);
    const size_t t6 = xsec_smem_bytes<float, 6, 128, kAlgTree>(32);
    CHECK(resident_blocks(t6) >= 5, "tile n=6 tree (128 threads): %zu bytes, fewer than 5 blocks per SM", t6);
    const size_t t7 = xsec_smem_bytes<float, 7, 256, kAlgTree>(8);
    CHECK(resident_blocks(t7) >= 3, "tile n=7 tree: %zu bytes, fewer than 3 blocks per SM", t7);
    CHECK(sizeof(SampleDraw) == 16, "SampleDraw is %zu bytes", sizeof(SampleDraw));
    std::printf("layout checks: %d failures\n", failures);
    return failures ? 1 : 0;
}
