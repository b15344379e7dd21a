// Host-side checks of the kernels' index tables and shared-memory layouts
// (compiled and run by tests/test_layout.py; no GPU needed).  Exit status 0
// when every check holds; each failure prints one line.
#include <cstdio>
#include <vector>

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

// prefix decoding of the walk: every ordered prefix of depth 2 and 3 exactly
// once, in lexicographic order, with distinct photons
template <int N>
static void check_prefixes() {
    int last = -1;
    for (int k = 0; k < N * (N - 1); ++k) {
        int a, b, c;
        tree_prefix<N, 2>(k, a, b, c);
        const int key = a * N + b;
        CHECK(a >= 0 && a < N && b >= 0 && b < N && a != b && key > last, "n=%d depth-2 prefix %d = (%d, %d)", N, k, a, b);
        last = key;
    }
    last = -1;
    for (int k = 0; k < N * (N - 1) * (N - 2); ++k) {
        int a, b, c;
        tree_prefix<N, 3>(k, a, b, c);
        const int key = (a * N + b) * N + c;
        CHECK(a >= 0 && b >= 0 && c >= 0 && a < N && b < N && c < N && a != b && a != c && b != c && key > last,
              "n=%d depth-3 prefix %d = (%d, %d, %d)", N, k, a, b, c);
        last = key;
    }
}

// lane layout of a shape: every (group, point slot, helicity bits) once per
// block, groups warp-aligned, units of work shared out evenly where the
// block's default allows it; pair units decode to every pair p < q once and
// spread a lane's bits over the other photons
template <class R, int N, int BLOCK>
static void check_shape(bool even) {
    using SH = DefaultShape<R, N, BLOCK>;
    using S = TreeShape<N, BLOCK, SH::HB, SH::G>;
    CHECK(SH::G * S::P * S::NSL == BLOCK, "n=%d block %d: lanes do not tile the block", N, BLOCK);
    CHECK(SH::G == 1 || S::GL % 32 == 0, "n=%d block %d: group of %d lanes", N, BLOCK, S::GL);
    if (even) CHECK(S::NPRE % SH::G == 0, "n=%d block %d: %d prefixes over %d groups", N, BLOCK, S::NPRE, SH::G);
    if (S::PAIRS) {
        int u = 0;
        for (int p = 0; p < N; ++p)
            for (int q = p + 1; q < N; ++q, ++u) {
                int a, b;
                pair_of_unit<N>(u, a, b);
                CHECK(a == p && b == q, "n=%d unit %d -> (%d, %d), expected (%d, %d)", N, u, a, b, p, q);
                for (unsigned hl = 0; hl < (1u << (N - 2)); ++hl) {
                    const unsigned h = spread_pair_bits(hl, p, q);
                    // the other photons' bits in order, zeros at p and q
                    unsigned back = 0;
                    int k = 0;
                    for (int i = 0; i < N; ++i)
                        if (i != p && i != q) back |= ((h >> i) & 1u) << k++;
                    CHECK(!((h >> p) & 1u) && !((h >> q) & 1u) && back == hl, "n=%d spread (%d, %d) %u", N, p, q, hl);
                }
            }
        CHECK(u == S::NPRE, "n=%d: %d pair units", N, u);
    }
}

// Met-in-the-middle currents: every buffer holds its sizes' rows; the row an
// item reads for photon position pos of set S, helicities lambda, is row
// (S - i, lambda without bit pos) of the size below, helicity-major
// (lambda' C(n, k-1) + rank(S - i)), inside that level; the contraction's
// rows for set T and configuration lambda are J(T, pext(lambda, T)) and
// R(all - T, pext(lambda, all - T)).
static int host_rank(unsigned S, int n) {
    int r = 0;
    for (unsigned u = 0; u < S; ++u)
        if (popcount(u) == popcount(S) && u < (1u << n)) ++r;
    return r;
}
static int host_pext(int x, unsigned m) {
    int o = 0, k = 0;
    for (int b = 0; b < 8; ++b)
        if ((m >> b) & 1u) o |= ((x >> b) & 1) << k++;
    return o;
}
template <class R, int N, int BLOCK>
static void check_meet() {
    using MT = MeetTables<R, N, BLOCK>;
    auto in_buf = [&](int k, int buf) {
        CHECK(meet_rows(N, k) <= buf, "n=%d: size-%d currents (%d rows) in a buffer of %d", N, k, meet_rows(N, k), buf);
    };
    for (int k = 1; k <= MT::M - 1; ++k) in_buf(k, ((MT::M - k) & 1) ? MT::J1 : MT::J0);
    for (int k = 1; k <= MT::MK - 1; ++k) in_buf(k, ((MT::MK - 1 - k) & 1) ? MT::K1 : MT::K0);
    CHECK((MT::CH << MT::M) <= MT::J0 && (MT::CH << MT::MK) <= MT::RR, "n=%d: chunk buffers", N);
    CHECK(MT::M > 1 || MT::CH == MT::CM, "n=%d: one-photon J read in place needs one chunk", N);
    CHECK(MT::G * MT::GTH <= BLOCK && MT::PG * MT::CT * MT::GT <= MT::GTH, "n=%d: group shape", N);
    CHECK(MT::G == 1 || 8 + MT::G <= 16, "n=%d: %d groups exceed the named barriers", N, MT::G);
    CHECK(!MT::XA_OVER || MT::XAB <= (size_t)(MT::J1 + MT::K0 + MT::K1) * sizeof(Row<R>), "n=%d: overlaid amplitudes", N);
    for (int k = 2; k <= MT::MK; ++k) {
        const int B = meet_block(k), LB = meet_lb(k), NB = (1 << k) / B;
        const int CK1 = set_binom(N, k - 1);
        for (unsigned S = 0; S < (1u << N); ++S) {
            if (popcount(S) != k) continue;
            for (int blk = 0; blk < NB; ++blk) {
                unsigned s = S;
                for (int pos = 0; pos < k; ++pos) {
                    const int i = __builtin_ctz(s);
                    s &= s - 1;
                    const int ri = host_rank(S ^ (1u << i), N);
                    for (int b = 0; b < B; ++b) {
                        const int lam = blk * B + b;
                        int got;
                        if ((1 << pos) < B) {
                            const int d = meet_drop(b, pos);
                            CHECK(meet_insert(d, pos, (b >> pos) & 1) == b, "n=%d insert/drop", N);
                            got = blk * (B / 2) * CK1 + ri + d * CK1;
                        } else {
                            got = meet_drop(blk, pos - LB) * B * CK1 + ri + b * CK1;
                        }
                        const int want = meet_drop(lam, pos) * CK1 + ri;
                        CHECK(got == want && got < meet_rows(N, k - 1), "n=%d k=%d S=%u blk=%d pos=%d b=%d: row %d, want %d",
                              N, k, S, blk, pos, b, got, want);
                    }
                }
            }
        }
    }
    // chunk rows: one row per (place, assignment), inside the buffer
    for (int LOGK : {MT::M, MT::MK}) {
        std::vector<int> seen((size_t)MT::CH << LOGK, 0);
        for (int t = 0; t < MT::CH; ++t)
            for (int lam = 0; lam < (1 << LOGK); ++lam) {
                const int rr = LOGK == MT::M ? meet_chunk_row<MT::M>(t, lam, MT::CH) : meet_chunk_row<MT::MK>(t, lam, MT::CH);
                CHECK(rr >= 0 && rr < (MT::CH << LOGK) && !seen[rr]++, "n=%d chunk row (%d, %d) -> %d", N, t, lam, rr);
            }
    }
    // contraction rows in the chunk buffers, as meet_contract forms them
    const int M = MT::M, CB = MT::CB, CH = MT::CH;
    const unsigned FULL = (1u << N) - 1;
    for (unsigned T = 0; T < (1u << N); ++T) {
        if (popcount(T) != M) continue;
        const unsigned V = FULL & ~T;
        const int r = host_rank(T, N), t = r % CH;
        const int TL = (int)(T & ((1u << CB) - 1)), VL = ((1 << CB) - 1) & ~TL, a = popcount((unsigned)TL);
        for (int lam = 0; lam < (1 << N); ++lam) {
            const int hi = lam >> CB, b = lam & ((1 << CB) - 1);
            const int lt = (host_pext(hi, T >> CB) << a) | host_pext(b, (unsigned)TL);
            const int lv = (host_pext(hi, V >> CB) << (CB - a)) | host_pext(b, (unsigned)VL);
            CHECK(lt == host_pext(lam, T) && lv == host_pext(lam, V), "n=%d T=%u lambda=%d: helicities", N, T, lam);
            const int jrow = meet_chunk_row<MT::M>(t, lt, CH), rrow = meet_chunk_row<MT::MK>(t, lv, CH);
            CHECK(jrow >= 0 && jrow < (CH << M) && rrow >= 0 && rrow < (CH << MT::MK), "n=%d T=%u lambda=%d: rows %d %d", N,
                  T, lam, jrow, rrow);
        }
    }
}

static size_t resident_blocks(size_t smem_per_block) {
    const size_t per_sm = 228 * 1024, reserved = 1024;
    return per_sm / (smem_per_block + reserved);
}

int main() {
    check_tree_tables();
    check_prefixes<4>();
    check_prefixes<5>();
    check_prefixes<6>();
    check_prefixes<7>();
    check_prefixes<8>();
    check_shape<float, 5, 256>(true);
    check_shape<double, 8, 256>(true);
    check_shape<float, 6, 160>(true);
    check_shape<float, 6, 256>(false);
    check_shape<float, 7, 224>(true);
    check_shape<float, 7, 256>(false);
    check_shape<float, 8, 256>(true);
    check_pair_columns<float, 4, 0, 1, 256>();
    check_pair_columns<float, 5, 0, 1, 256>();
    check_pair_columns<float, 6, 2, 5, 160>();
    check_pair_columns<float, 6, 2, 8, 256>();
    check_pair_columns<float, 7, 2, 7, 224>();
    check_pair_columns<float, 7, 2, 4, 256>();
    check_pair_columns<float, 8, 2, 4, 256>();
    check_pair_columns<double, 4, 0, 1, 256>();
    check_pair_columns<double, 8, 0, 1, 256>();
    // occupancy the tuned launch shapes rely on
    const size_t draws4 = 2 * ws_stage(4, kAlgTree) * sizeof(SampleDraw) + 256;
    const size_t ws4 = ws_smem_bytes<float, 4, kAlgTree>() + draws4;
    CHECK(resident_blocks(ws4) >= 2, "warp-specialised n=4 tree: %zu bytes, fewer than 2 blocks per SM", ws4);
    const size_t ws4s = ws_smem_bytes<float, 4, kAlgSubset>() + draws4;
    CHECK(resident_blocks(ws4s) >= 2, "warp-specialised n=4 subset: %zu bytes, fewer than 2 blocks per SM", ws4s);
    // the escalating kernel keeps 256 consumers (its FP32 bound runs on them)
    constexpr int ws4_esc_threads = ws_threads<4, kAlgTree, true>(), ws4_threads = ws_threads<4, kAlgTree, false>();
    CHECK(ws4_esc_threads == 384 && ws4_threads == 256, "n=4 tree block shapes %d %d", ws4_esc_threads, ws4_threads);
    const size_t ws4e = ws_smem_bytes<float, 4, kAlgTree, table_alg<kAlgTree, true>()>() + draws4;
    CHECK(resident_blocks(ws4e) >= 2, "warp-specialised n=4 tree with escalation: %zu bytes", ws4e);
    const size_t ws5 = ws_smem_bytes<float, 5, kAlgTree>() + 2 * ws_stage(5, kAlgTree) * sizeof(SampleDraw) + 256;
    CHECK(resident_blocks(ws5) >= 2, "warp-specialised n=5 tree: %zu bytes", ws5);
    const size_t ws6 = ws_smem_bytes<float, 6, kAlgTree>() + 2 * ws_stage(6, kAlgTree) * sizeof(SampleDraw) + 256;
    CHECK(resident_blocks(ws6) >= 2, "warp-specialised n=6 tree: %zu bytes", ws6);
    check_shape<float, 6, ws_consumers(6, kAlgTree, false)>(true);
    const size_t t6 = xsec_smem_bytes<float, 6, 160, kAlgTree>(64);
    CHECK(resident_blocks(t6) >= 3, "tile n=6 tree (160 threads): %zu bytes, fewer than 3 blocks per SM", t6);
    const size_t t7 = xsec_smem_bytes<float, 7, 224, kAlgTree>(32);
    CHECK(resident_blocks(t7) >= 2, "tile n=7 tree (224 threads): %zu bytes, fewer than 2 blocks per SM", t7);
    const size_t t8 = xsec_smem_bytes<float, 8, 256, kAlgTree>(8);
    CHECK(resident_blocks(t8) >= 2, "tile n=8 tree: %zu bytes, fewer than 2 blocks per SM", t8);
    check_meet<float, 2, 256>();
    check_meet<float, 3, 256>();
    check_meet<float, 4, 256>();
    check_meet<float, 5, 256>();
    check_meet<float, 6, 256>();
    check_meet<float, 7, 256>();
    check_meet<float, 8, 256>();
    check_meet<double, 6, 256>();
    check_meet<double, 8, 256>();
    check_meet<float, 7, ws_consumers(7, kAlgSubset, false)>();
    check_meet<float, 8, ws_consumers(8, kAlgSubset, false)>();
    const size_t ws8s = ws_smem_bytes<float, 8, kAlgSubset>() + 2 * ws_stage(8, kAlgSubset) * sizeof(SampleDraw) + 256;
    CHECK(resident_blocks(ws8s) >= 1, "warp-specialised n=8 subset: %zu bytes", ws8s);
    const size_t ws7s = ws_smem_bytes<float, 7, kAlgSubset>() + 2 * ws_stage(7, kAlgSubset) * sizeof(SampleDraw) + 256;
    CHECK(resident_blocks(ws7s) >= 1, "warp-specialised n=7 subset: %zu bytes", ws7s);
    const size_t ws6s = ws_smem_bytes<float, 6, kAlgSubset>() + 2 * ws_stage(6, kAlgSubset) * sizeof(SampleDraw) + 256;
    CHECK(resident_blocks(ws6s) >= 2, "warp-specialised n=6 subset: %zu bytes, fewer than 2 blocks per SM", ws6s);
    CHECK(sizeof(SampleDraw) == 16, "SampleDraw is %zu bytes", sizeof(SampleDraw));
    std::printf("layout checks: %d failures\n", failures);
    return failures ? 1 : 0;
}
