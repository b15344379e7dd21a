// heget_meet.cuh -- the ordering sum as a recursion over photon sets, met in
// the middle (the amplitude rounds of the subset algorithm).
//
// Every ordering's chain is  vbar E_{pi1} Q_{T1} E_{pi2} Q_{T2} ... Q_{T(n-1)}
// E_{pin} u_R  with E_i = eps*_i . sigma for the photon's helicity and
// Q_T = (q_T . sigmabar) / q_T^2 for the set T of photons attached from the
// vbar end (the prefix tree's step matrix is M(i, T) = E_i Q_T).  Cutting each
// chain after its m-th photon (m = floor(n/2)) and summing the orderings on
// each side of the cut first (distributivity; the grouping by photon set of
// the sum over permutations in Sec. 2.1 eqs. (6)-(8)):
//   J(S) = [sum_{i in S} J(S - i) E_i] Q_S,            J({i}) = vbar E_i Q_{i},
//   K(W) = Q_{all - W} [sum_{i in W} E_i K(W - i)],    K({i}) = Q_{all - i} E_i u_R,
//   R(V) = sum_{i in V} E_i K(V - i)                   (|V| = n - m; R = E u_R at n = 2),
//   A    = sum_{|T| = m} J(T) . R(all - T),
// each current for every assignment of its own photons' helicities.  J is a
// row 2-spinor (vbar side), K and R are columns (u side).  E has the form
// [[e00, e01], [e10, -e00]] with e00 real and Q the form [[A, B*], [B, D]]
// with A, D real, so one term of a current costs 12 fused multiply-adds and
// its Q product 12 more.  This is the same sum of products as the prefix
// tree, rounded in another order, with about 3.2e5 multiply-adds per point at
// n = 8 (the tree walk: about 5e6).
//
// Work: the block's threads form G groups of GTH threads; each group takes
// its own points, PG at a time, through phases separated by the group's own
// named barrier, so that the phases of different groups overlap: photon and
// set data, E and the one-photon currents; one phase per current size k =
// 2 .. n-m-1 (J of size k < m, K of size k); then, chunk by chunk over the
// sets T of size m (CH at a time; all at once below n = 8), J(T) and R(all -
// T) followed by their contraction (2^CB helicity configurations per thread,
// the chunk's sets shared out over thread groups); a fixed-order sum of the
// groups and of w_h |A_h|^2 per point.  Every sum runs in an order fixed by
// the launch shape, so results are reproducible bit for bit.  The chunks
// bound a point's tables at n = 8 to 28 KB (57 KB with every J and R of size
// 4 held at once), so that more points share an SM.
//
// Layout: the currents of size k < m sit helicity-major, row(S, lambda) =
// lambda C(n, k) + rank(S) (rank among the sets of size k in numeric
// order), so that an item's rows for its helicity block lie at constant
// strides from one base (immediate load offsets) and the threads of a warp,
// taking consecutive sets, store consecutive rows.  The chunks' J and R go
// set-major with an XOR swizzle (meet_chunk_row), which keeps both their
// stores and the contraction's loads nearly free of bank conflicts; E sits
// photon-minor.  Index work that does not depend on the point (which photon
// sits at which position of a set, the rank of the set without it, the
// complement's rank, the helicity bits at a set's positions) comes from
// tables built once per call.
#pragma once

#include <type_traits>

#include "heget_amp.cuh"

namespace heget {

// currents of the sets of size k, each with its 2^k helicity assignments
__host__ __device__ constexpr int meet_rows(int n, int k) { return k < 1 ? 0 : set_binom(n, k) << k; }

// Helicity block of a size-k item: B = min(2^k, 2^kMeetLB) assignments of
// the set's helicities, the low log2(B) bits varying, the block index giving
// the others.  An input row of a photon whose helicity varies inside the
// block feeds two outputs (24 multiply-adds per row loaded, else 12); four
// rows keep the accumulators within the register budget of two 288-thread
// blocks per SM.
constexpr int kMeetLB = 2;
__host__ __device__ constexpr int meet_lb(int k) { return k >= kMeetLB ? kMeetLB : k; }
__host__ __device__ constexpr int meet_block(int k) { return 1 << meet_lb(k); }

// Contraction: 2^CB helicity configurations per thread (photons 0 .. CB-1
// free).  From n = 6 the 2^(n-CB) threads of a point and set T fill exactly
// one warp (CB = n - 5), so that every lane of a warp contracts the same T:
// the code path chosen by T's lower photons is then uniform, and lanes that
// need the same J or R row read it in one broadcast.
__host__ __device__ constexpr int meet_cb(int n) { return n >= 6 ? n - 5 : n >= 3 ? 3 : n; }

// Input-table entries of the sizes 2 .. k-1 (one per set and position).
__host__ __device__ constexpr int meet_in_offset(int n, int k) {
    int o = 0;
    for (int j = 2; j < k; ++j) o += set_binom(n, j) * j;
    return o;
}

// Group shape: threads per group (two to four warps from n = 6, the whole
// block below), points a group takes per round, sets T of size m per chunk.
template <class R>
__host__ __device__ constexpr int meet_group_threads(int n, int block) {
    const int want = n <= 5 ? block : n == 6 ? 64 : 128;
    return want < block ? want : block;
}
// (FP64 at n = 6: two points per group, whose longer FP64 phases then
// share each barrier; in FP32 one point per group is faster.)
template <class R>
__host__ __device__ constexpr int meet_group_points(int n, int gth) {
    const int p = n <= 5 ? gth / 16 : n == 6 && sizeof(R) != sizeof(float) ? 2 : 1;
    const int q = n <= 5 && sizeof(R) != sizeof(float) ? p / 2 : p;
    return q > 0 ? q : 1;
}
__host__ __device__ constexpr int meet_chunk(int n) { return n == 8 ? 14 : set_binom(n, n / 2); }

template <class R, int N, int BLOCK>
struct MeetTables {
    static constexpr int NS = 1 << N;
    static constexpr int M = N / 2;       // vbar side: J of sizes 1 .. M
    static constexpr int MK = N - M;      // u side: K of sizes 1 .. MK-1, R of size MK
    static constexpr int GTH = meet_group_threads<R>(N, BLOCK);
    static constexpr int G = BLOCK / GTH;
    static constexpr int PG = meet_group_points<R>(N, GTH);
    static constexpr int CM = set_binom(N, M), CMK = set_binom(N, MK);
    static constexpr int CH = meet_chunk(N);
    // rows per point: two buffers per side, alternating by size: J of size
    // M-2 (M-4, ...) and then the chunk's J of size M in the first, M-1
    // (M-3, ...) in the second; K of size MK-1 (MK-3, ...), MK-2 (...); the
    // chunk's R
    static constexpr int JA = meet_rows(N, M - 2), JB = CH << M;
    static constexpr int J0 = JA > JB ? JA : JB, J1 = meet_rows(N, M - 1);
    static constexpr int K0 = meet_rows(N, MK - 1), K1 = meet_rows(N, MK - 2);
    static constexpr int RR = CH << MK;
    static constexpr int PL = J0 + J1 + K0 + K1 + RR;
    static constexpr int PT = N + NS + 4 * N + PL;       // rows per point with PH, SD, E
    // contraction: threads per point (2^CB configurations each), groups over T
    static constexpr int CB = meet_cb(N);
    static constexpr int CT = NS >> CB;
    static constexpr int GT = GTH / (PG * CT) > 0 ? GTH / (PG * CT) : 1;
    static constexpr int HM = 1 << (N - CB);             // values of the helicity bits above CB
    static constexpr int NIN = meet_in_offset(N, MK + 1);
    // the groups' amplitudes overlay J1, K0, K1 of the group's point once the
    // last chunk's currents are formed (one point per group), else follow
    static constexpr size_t XAB = (size_t)GT * PG * NS * 2 * sizeof(R);
    static constexpr bool XA_OVER = PG == 1 && XAB <= (size_t)(J1 + K0 + K1) * sizeof(Row<R>);
    static constexpr size_t GB = (size_t)PG * PT * sizeof(Row<R>) + (XA_OVER ? 0 : XAB);   // bytes per group
    static_assert(N >= 2 && PG * CT * GT <= GTH, "group shape");
    static constexpr size_t align4(size_t x) { return (x + 3) & ~(size_t)3; }
    static constexpr size_t bytes = (size_t)G * GB + align4((size_t)NIN * 2) + 2 * (size_t)NS + (size_t)HM * HM + 80;
    unsigned char* base;
    unsigned short* IN;    // size k, set rank r, position pos: rank(S - i) | i << 8
    unsigned char* RANK;   // [2^N]: rank of S among the sets of its size
    unsigned char* LIST;   // [2^N]: sets by size, then rank
    unsigned char* PXH;    // [HM][HM]: bits of h at the set bits of m, packed
    unsigned char* CR;     // [C(n, M)]: rank of the complement of the size-M set of rank r
    __device__ __forceinline__ explicit MeetTables(unsigned char* b) : base(b) {
        IN = reinterpret_cast<unsigned short*>(b + (size_t)G * GB);
        RANK = reinterpret_cast<unsigned char*>(IN) + align4((size_t)NIN * 2);
        LIST = RANK + NS;
        PXH = LIST + NS;
        CR = PXH + HM * HM;
    }
    // per group g and point slot p (< PG)
    __device__ __forceinline__ Row<R>* pt(int g, int p) const {
        return reinterpret_cast<Row<R>*>(base + (size_t)g * GB) + (size_t)p * PT;
    }
    __device__ __forceinline__ Row<R>* PH(int g, int p) const { return pt(g, p); }
    __device__ __forceinline__ Row<R>* SD(int g, int p) const { return pt(g, p) + N; }
    __device__ __forceinline__ Row<R>* E(int g, int p) const { return pt(g, p) + N + NS; }
    __device__ __forceinline__ Row<R>* LV(int g, int p) const { return pt(g, p) + N + NS + 4 * N; }
    __device__ __forceinline__ Row<R>* J(int g, int p, int k) const { return LV(g, p) + (((M - k) & 1) ? J0 : 0); }
    __device__ __forceinline__ Row<R>* K(int g, int p, int k) const {
        return LV(g, p) + J0 + J1 + (((MK - 1 - k) & 1) ? K0 : 0);
    }
    __device__ __forceinline__ Row<R>* RV(int g, int p) const { return LV(g, p) + J0 + J1 + K0 + K1; }
    __device__ __forceinline__ R* XA(int g) const {
        return XA_OVER ? reinterpret_cast<R*>(LV(g, 0) + J0)
                       : reinterpret_cast<R*>(base + (size_t)g * GB + (size_t)PG * PT * sizeof(Row<R>));
    }
};

// E = eps*(k, lambda) . sigma = [[e00, e01], [e10, -e00]]: the step matrix
// without the propagator.
template <class R>
struct EMat {
    R e00, e01r, e01i, e10r, e10i;
};

// E of photon i, helicity lam from a point's table (rows (2 lam + r) N + i,
// r = 0: (e00, e01, Re e10), r = 1: (Im e10, -, -, -)): the photons of a
// warp's items lie in consecutive rows
template <class R, int N>
__device__ __forceinline__ EMat<R> load_e(const Row<R>* em, int i, int lam) {
    const Row<R> a = ld_row(em + 2 * lam * N + i);
    return EMat<R>{a.ar, a.ai, a.br, a.bi, em[(2 * lam + 1) * N + i].ar};
}

// E for photon direction ph (sin theta, cos theta, cos phi, sin phi) and
// helicity lam_bit (1: +, 0: -), as in step_matrix:
//   E = (1/sqrt2) [[-l s, -(1 - l c) e^{-i phi}], [(1 + l c) e^{i phi}, l s]].
template <class R>
__device__ __forceinline__ EMat<R> e_matrix(const Row<R>& ph, int lam_bit) {
    const R rs2 = R(0.70710678118654752440);
    const R l = lam_bit ? R(1) : R(-1);
    const R am = (R(1) - l * ph.ai) * rs2, ap = (R(1) + l * ph.ai) * rs2;
    return EMat<R>{-l * ph.ar * rs2, -am * ph.br, am * ph.bi, ap * ph.br, ap * ph.bi};
}

// acc += r . E (r a row)
template <class R>
__device__ __forceinline__ void row_e_acc(Row<R>& acc, const Row<R>& r, const EMat<R>& E) {
    acc.ar = fmad<R>(r.ar, E.e00, fmad<R>(r.br, E.e10r, fmad<R>(-r.bi, E.e10i, acc.ar)));
    acc.ai = fmad<R>(r.ai, E.e00, fmad<R>(r.br, E.e10i, fmad<R>(r.bi, E.e10r, acc.ai)));
    acc.br = fmad<R>(r.ar, E.e01r, fmad<R>(-r.ai, E.e01i, fmad<R>(-r.br, E.e00, acc.br)));
    acc.bi = fmad<R>(r.ar, E.e01i, fmad<R>(r.ai, E.e01r, fmad<R>(-r.bi, E.e00, acc.bi)));
}

// acc += E . c (c a column)
template <class R>
__device__ __forceinline__ void e_col_acc(Row<R>& acc, const EMat<R>& E, const Row<R>& c) {
    acc.ar = fmad<R>(E.e00, c.ar, fmad<R>(E.e01r, c.br, fmad<R>(-E.e01i, c.bi, acc.ar)));
    acc.ai = fmad<R>(E.e00, c.ai, fmad<R>(E.e01r, c.bi, fmad<R>(E.e01i, c.br, acc.ai)));
    acc.br = fmad<R>(E.e10r, c.ar, fmad<R>(-E.e10i, c.ai, fmad<R>(-E.e00, c.br, acc.br)));
    acc.bi = fmad<R>(E.e10r, c.ai, fmad<R>(E.e10i, c.ar, fmad<R>(-E.e00, c.bi, acc.bi)));
}

// r . Q and Q . c for Q = [[A, B*], [B, D]] stored as (A, D, Re B, Im B)
template <class R>
__device__ __forceinline__ Row<R> row_q(const Row<R>& r, const Row<R>& q) {
    const R A = q.ar, D = q.ai, Br = q.br, Bi = q.bi;
    Row<R> o;
    o.ar = fmad<R>(r.ar, A, fmad<R>(r.br, Br, -r.bi * Bi));
    o.ai = fmad<R>(r.ai, A, fmad<R>(r.br, Bi, r.bi * Br));
    o.br = fmad<R>(r.ar, Br, fmad<R>(r.ai, Bi, r.br * D));
    o.bi = fmad<R>(-r.ar, Bi, fmad<R>(r.ai, Br, r.bi * D));
    return o;
}
template <class R>
__device__ __forceinline__ Row<R> q_col(const Row<R>& q, const Row<R>& c) {
    const R A = q.ar, D = q.ai, Br = q.br, Bi = q.bi;
    Row<R> o;
    o.ar = fmad<R>(A, c.ar, fmad<R>(Br, c.br, Bi * c.bi));
    o.ai = fmad<R>(A, c.ai, fmad<R>(Br, c.bi, -Bi * c.br));
    o.br = fmad<R>(Br, c.ar, fmad<R>(-Bi, c.ai, D * c.br));
    o.bi = fmad<R>(Br, c.ai, fmad<R>(Bi, c.ar, D * c.bi));
    return o;
}

// x with bit `pos` removed (the helicities of S - i from those of S), and
// with a bit of value v inserted at `pos`
__host__ __device__ constexpr int meet_drop(int x, int pos) {
    return (x & ((1 << pos) - 1)) | ((x >> (pos + 1)) << pos);
}
__host__ __device__ constexpr int meet_insert(int x, int pos, int v) {
    return (x & ((1 << pos) - 1)) | (v << pos) | ((x >> pos) << (pos + 1));
}
__host__ __device__ constexpr int meet_popc(int x) { return x ? (x & 1) + meet_popc(x >> 1) : 0; }
// bits of x at the set bits of m, packed
__host__ __device__ constexpr int meet_pext(int x, int m) {
    int o = 0, k = 0;
    for (int b = 0; b < 8; ++b)
        if ((m >> b) & 1) o |= ((x >> b) & 1) << k++;
    return o;
}

// The point-independent tables of MeetTables (lists and ranks of the sets,
// input table, pext table, complement ranks), by the block's threads.
template <class R, int N, int BLOCK>
__device__ __forceinline__ void meet_build_tables(const MeetTables<R, N, BLOCK>& tb) {
    using MT = MeetTables<R, N, BLOCK>;
    const int tid = threadIdx.x;
    build_set_list<N>(tb.LIST, tb.RANK, tid, BLOCK);
    for (int v = tid; v < MT::HM * MT::HM; v += BLOCK) tb.PXH[v] = (unsigned char)meet_pext(v / MT::HM, v % MT::HM);
    // input table: for each size k = 2 .. n-m, set S (by rank) and position pos,
    // the pos-th photon i of S and rank(S - i); complement ranks of size m
    for (int S = tid; S < MT::NS; S += BLOCK) {
        const int k = __popc(S);
        if (k == MT::M) tb.CR[set_rank<N>((unsigned)S)] = (unsigned char)set_rank<N>((unsigned)(MT::NS - 1) & ~(unsigned)S);
        if (k < 2 || k > MT::MK) continue;
        unsigned short* e = tb.IN + meet_in_offset(N, k) + set_rank<N>((unsigned)S) * k;
        unsigned s = (unsigned)S;
        for (int pos = 0; pos < k; ++pos) {
            const int i = __ffs(s) - 1;
            s &= s - 1;
            e[pos] = (unsigned short)(set_rank<N>((unsigned)S ^ (1u << i)) | (i << 8));
        }
    }
}

// Row of helicity assignment lam of the t-th set of a chunk (2^LOG rows per
// set): set-major with the assignment XOR-ed by t mod 8 when a set has at
// least eight rows (the items, taking consecutive sets, store in different
// banks; the contraction, reading one set's rows, meets at most two-way
// conflicts), else helicity-major with stride ch.
template <int LOG>
__host__ __device__ __forceinline__ int meet_chunk_row(int t, int lam, int ch) {
    if constexpr (LOG >= 3) return (t << LOG) + (lam ^ (t & 7));
    else return lam * ch + t;
}

// Named barrier of group g (GTH threads), or the block's when it is one group.
template <int BAR, int BLOCK, int GBAR0, int GTH, int G>
__device__ __forceinline__ void meet_sync(int g) {
    if constexpr (G == 1 && GTH == BLOCK) {
        group_sync<BAR, BLOCK>();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(GBAR0 + g), "n"(GTH) : "memory");
    }
}

// One item of size K: the currents of set S (rank rS among the sets of size
// K) for the helicity assignments blk B .. blk B + B - 1, from the size-(K-1)
// currents in src (helicity-major) into dst at rows lambda OS + oi.  COL: the
// u side (columns, E on the left; with WITHQ the complement's Q after the
// sum: K; without: R); else the vbar side (rows, E on the right, Q_S after:
// J).  em: the point's E table, sd: its set data.
template <class R, int N, int BLOCK, int K, bool COL, bool WITHQ, bool CHUNK = false>
__device__ __forceinline__ void meet_item(const MeetTables<R, N, BLOCK>& tb, const Row<R>* em, const Row<R>* sd, int rS,
                                          int blk, const Row<R>* src, Row<R>* dst, int OS, int oi) {
    constexpr int B = meet_block(K), LB = meet_lb(K);
    constexpr int CK1 = set_binom(N, K - 1);
    constexpr unsigned FULL = (1u << N) - 1;
    const unsigned short* in = tb.IN + meet_in_offset(N, K) + rS * K;
    Row<R> acc[B];
#pragma unroll
    for (int b = 0; b < B; ++b) acc[b] = Row<R>{R(0), R(0), R(0), R(0)};
#pragma unroll
    for (int pos = 0; pos < K; ++pos) {
        const unsigned v = in[pos];
        const int ri = (int)(v & 0xFFu), i = (int)(v >> 8);
        if ((1 << pos) < B) {   // (pos is a constant once the loop is unrolled)
            // this photon's helicity varies inside the block: each input feeds two outputs
            const EMat<R> E0 = load_e<R, N>(em, i, 0), E1 = load_e<R, N>(em, i, 1);
            const Row<R>* x0 = src + blk * (B / 2) * CK1 + ri;
#pragma unroll
            for (int d = 0; d < B / 2; ++d) {
                const Row<R> x = ld_row(x0 + d * CK1);
                const int b0 = meet_insert(d, pos, 0), b1 = meet_insert(d, pos, 1);
                if constexpr (COL) {
                    e_col_acc(acc[b0], E0, x);
                    e_col_acc(acc[b1], E1, x);
                } else {
                    row_e_acc(acc[b0], x, E0);
                    row_e_acc(acc[b1], x, E1);
                }
            }
        } else {
            const int sh = pos >= LB ? pos - LB : 0;
            const EMat<R> E = load_e<R, N>(em, i, (blk >> sh) & 1);
            const Row<R>* x0 = src + meet_drop(blk, sh) * B * CK1 + ri;
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const Row<R> x = ld_row(x0 + b * CK1);
                if constexpr (COL) e_col_acc(acc[b], E, x);
                else row_e_acc(acc[b], x, E);
            }
        }
    }
    // rows: lambda OS + oi, or for a chunk meet_chunk_row (oi the place in the chunk, OS its size)
    auto row = [&](int b) { return CHUNK ? meet_chunk_row<K>(oi, blk * B + b, OS) : (blk * B + b) * OS + oi; };
    if constexpr (!WITHQ) {
#pragma unroll
        for (int b = 0; b < B; ++b) st_row(dst + row(b), acc[b]);
    } else {
        const unsigned S = tb.LIST[set_level_offset(N, K) + rS];
        const Row<R> q = ld_row(sd + (COL ? (FULL & ~S) : S));
#pragma unroll
        for (int b = 0; b < B; ++b) st_row(dst + row(b), COL ? q_col<R>(q, acc[b]) : row_q<R>(acc[b], q));
    }
}

// Phase of size K (2 <= K < n - m) of group g: J of size K (K < m), K of
// size K; items ordered set fastest, then helicity block, then point.
template <class R, int N, int BLOCK, int BAR, int GBAR0, int K>
__device__ __forceinline__ void meet_phase(const MeetTables<R, N, BLOCK>& tb, int g, int lid, const PointRec<R, N>* rb,
                                           int cnt) {
    using MT = MeetTables<R, N, BLOCK>;
    constexpr int PG = MT::PG, M = MT::M, MK = MT::MK;
    constexpr int CK = set_binom(N, K), NB = (1 << K) / meet_block(K);
    constexpr int NJ = K < M ? PG * CK * NB : 0;
    constexpr int NK = PG * CK * NB;
    // the K items start at a warp boundary, so that no warp runs both kinds
    constexpr int NJP = (NJ + 31) / 32 * 32;
    for (int it = lid; it < NJP + NK; it += MT::GTH) {
        const bool col = it >= NJP;
        const int q = col ? it - NJP : it;
        if (!col && q >= NJ) continue;
        const int rS = q % CK, blk = (q / CK) % NB, p = q / (NB * CK);
        if (p >= cnt || !rb[p].valid) continue;
        if (!col) {
            if constexpr (K < M)
                meet_item<R, N, BLOCK, K, false, true>(tb, tb.E(g, p), tb.SD(g, p), rS, blk, tb.J(g, p, K - 1),
                                                       tb.J(g, p, K), CK, rS);
        } else {
            meet_item<R, N, BLOCK, K, true, true>(tb, tb.E(g, p), tb.SD(g, p), rS, blk, tb.K(g, p, K - 1), tb.K(g, p, K),
                                                  CK, rS);
        }
    }
    meet_sync<BAR, BLOCK, GBAR0, MT::GTH, MT::G>(g);
    if constexpr (K + 1 < MK) meet_phase<R, N, BLOCK, BAR, GBAR0, K + 1>(tb, g, lid, rb, cnt);
}

// Chunk phase of group g: J of size m for the sets of rank c0 .. c0+nc-1 and
// R of their complements, into the chunk buffers (rows lambda CH + t).
template <class R, int N, int BLOCK>
__device__ __forceinline__ void meet_chunk_items(const MeetTables<R, N, BLOCK>& tb, int g, int lid,
                                                 const PointRec<R, N>* rb, int cnt, int c0, int nc) {
    using MT = MeetTables<R, N, BLOCK>;
    constexpr int PG = MT::PG, M = MT::M, MK = MT::MK, CH = MT::CH;
    constexpr int NBJ = M >= 2 ? (1 << M) / meet_block(M) : 0, NBR = MK >= 2 ? (1 << MK) / meet_block(MK) : 0;
    const int NJ = PG * nc * NBJ, NR = PG * nc * NBR;
    const int NJP = (NJ + 31) / 32 * 32;   // R items from a warp boundary on
    for (int it = lid; it < NJP + NR; it += MT::GTH) {
        const bool col = it >= NJP;
        const int q = col ? it - NJP : it;
        if (!col && q >= NJ) continue;
        const int nb = col ? NBR : NBJ;
        const int t = q % nc, blk = (q / nc) % nb, p = q / (nb * nc);
        if (p >= cnt || !rb[p].valid) continue;
        if (!col) {
            if constexpr (M >= 2)
                meet_item<R, N, BLOCK, M, false, true, true>(tb, tb.E(g, p), tb.SD(g, p), c0 + t, blk, tb.J(g, p, M - 1),
                                                       tb.J(g, p, M), CH, t);
        } else {
            if constexpr (MK >= 2)
                meet_item<R, N, BLOCK, MK, true, false, true>(tb, tb.E(g, p), tb.SD(g, p), tb.CR[c0 + t], blk,
                                                        tb.K(g, p, MK - 1), tb.RV(g, p), CH, t);
        }
    }
}

// Contraction of the t-th set T of a chunk whose photons below CB are TL (a
// compile-time case): the thread's 2^CB configurations lambda = (hi << CB) |
// b add J(T, lambda_T) . R(V, lambda_V), V = all - T; phT, phV: the bits of hi
// at the upper photons of T and of V, packed (they sit above the |TL| and
// CB - |TL| lower ones).
template <class R, int N, int CB, int M, int MK, int CH, int TL>
__device__ __forceinline__ void meet_contract_case(const Row<R>* J, const Row<R>* RV, int t, int phT, int phV,
                                                   R (&are)[1 << CB], R (&aim)[1 << CB]) {
    constexpr int VL = ((1 << CB) - 1) & ~TL;
    constexpr int a = meet_popc(TL), av = meet_popc(VL);
    Row<R> jr[1 << a], rr[1 << av];
#pragma unroll
    for (int j = 0; j < (1 << a); ++j) jr[j] = ld_row(J + meet_chunk_row<M>(t, (phT << a) | j, CH));
#pragma unroll
    for (int j = 0; j < (1 << av); ++j) rr[j] = ld_row(RV + meet_chunk_row<MK>(t, (phV << av) | j, CH));
#pragma unroll
    for (int b = 0; b < (1 << CB); ++b) close_row(jr[meet_pext(b, TL)], rr[meet_pext(b, VL)], are[b], aim[b]);
}

template <class R, int N, int CB, int M, int MK, int CH>
__device__ __forceinline__ void meet_contract(int TL, const Row<R>* J, const Row<R>* RV, int t, int phT, int phV,
                                              R (&are)[1 << CB], R (&aim)[1 << CB]) {
#define HEGET_MEET_CASE(c)                                                                 \
    case c:                                                                                \
        if constexpr (c < (1 << CB)) meet_contract_case<R, N, CB, M, MK, CH, c>(J, RV, t, phT, phV, are, aim); \
        break;
    switch (TL) {
        HEGET_MEET_CASE(0)
        HEGET_MEET_CASE(1)
        HEGET_MEET_CASE(2)
        HEGET_MEET_CASE(3)
        HEGET_MEET_CASE(4)
        HEGET_MEET_CASE(5)
        HEGET_MEET_CASE(6)
        HEGET_MEET_CASE(7)
        default:
            break;
    }
#undef HEGET_MEET_CASE
}

// Amplitude rounds over recs[0 .. cnt-1] by the met-in-the-middle recursion:
// the same contract as amplitude_rounds (recs[p].ssum = sum_h w_h |A_h|^2 in
// the scaled units of the records; mask: helicity mask, NULL = all).  All
// threads must call it; BAR: the block barrier of the caller's threads, the
// groups' own barriers counting from GBAR0 (1 with __syncthreads, else 8).
template <class R, int N, int BLOCK, int BAR = 0>
__device__ __noinline__ void amplitude_rounds_meet(unsigned char* table_smem, PointRec<R, N>* recs, int cnt,
                                                   const uint32_t* mask) {
    using MT = MeetTables<R, N, BLOCK>;
    constexpr int NS = MT::NS, M = MT::M, MK = MT::MK, CT = MT::CT, GT = MT::GT, CB = MT::CB, PG = MT::PG;
    constexpr int GTH = MT::GTH, G = MT::G, CM = MT::CM, CH = MT::CH;
    constexpr int GBAR0 = BAR == 0 ? 1 : 8;
    static_assert(G == 1 || GBAR0 + G <= 16, "named barriers of the groups");
    constexpr unsigned FULL = NS - 1;
    const MT tb(table_smem);
    meet_build_tables(tb);
    group_sync<BAR, BLOCK>();
    const int g = threadIdx.x / GTH, lid = threadIdx.x % GTH;
    if (g < G) {
        for (int base = g * PG; base < cnt; base += G * PG) {
            const int rc = min(PG, cnt - base);
            const PointRec<R, N>* rb = recs + base;
            // photon and set data; E and the one-photon currents (helicity-major,
            // row lambda N + i): J({i}) = n2 (e10, -e00) Q_{i}, E u_R = n1 (e00, e10),
            // K({i}) = Q_{all - i} E u_R (or R = E u_R at n = 2), from the record
            for (int it = lid; it < PG * (N + NS + 2 * N); it += GTH) {
                const int p = it / (N + NS + 2 * N), e = it - p * (N + NS + 2 * N);
                if (p >= rc) continue;
                const PointRec<R, N>& rc_ = rb[p];
                if (e < N) {
                    tb.PH(g, p)[e] = photon_row<R>(rc_.k[e]);
                } else if (e < N + NS) {
                    const unsigned T = tb.LIST[e - N];
                    if (T != 0u && T != FULL) tb.SD(g, p)[T] = set_row<R, N>(rc_, T);
                } else if (rc_.valid) {
                    const int q = e - N - NS, lam = q & 1, i = q >> 1;
                    const EMat<R> E = e_matrix<R>(photon_row<R>(rc_.k[i]), lam);
                    Row<R>* em = tb.E(g, p) + 2 * lam * N + i;
                    st_row(em, Row<R>{E.e00, E.e01r, E.e01i, E.e10r});
                    st_row(em + N, Row<R>{E.e10i, R(0), R(0), R(0)});
                    const R n1 = rc_.n1, n2 = rc_.n2;
                    const int x = lam * N + i;
                    st_row(tb.J(g, p, 1) + x,
                           row_q<R>(Row<R>{n2 * E.e10r, n2 * E.e10i, -n2 * E.e00, R(0)}, set_row<R, N>(rc_, 1u << i)));
                    const Row<R> cl{n1 * E.e00, R(0), n1 * E.e10r, n1 * E.e10i};
                    if constexpr (MK >= 2) st_row(tb.K(g, p, 1) + x, q_col<R>(set_row<R, N>(rc_, FULL & ~(1u << i)), cl));
                    else st_row(tb.RV(g, p) + lam * N + (N - 1 - i), cl);   // n = 2: at the place of T = all - {i}
                }
            }
            meet_sync<BAR, BLOCK, GBAR0, GTH, G>(g);
            if constexpr (MK >= 3) meet_phase<R, N, BLOCK, BAR, GBAR0, 2>(tb, g, lid, rb, rc);
            // chunks of the sets T of size m: their J and the R of their
            // complements, then the contraction A(lambda) += J(T) . R(all - T)
            // by 2^CB configurations per thread (photons below CB free, hi
            // the others), the chunk's sets shared out over GT groups
            const int gt = lid / (PG * CT), rem = lid % (PG * CT);
            const int p = rem / CT, hi = rem % CT;
            const bool mine = gt < GT && p < rc && rb[p].valid;
            R are[1 << CB], aim[1 << CB];
#pragma unroll
            for (int b = 0; b < (1 << CB); ++b) are[b] = aim[b] = R(0);
            const unsigned char* px = tb.PXH + hi * MT::HM;
#pragma unroll 1
            for (int c0 = 0; c0 < CM; c0 += CH) {
                const int nc = min(CH, CM - c0);
                meet_chunk_items(tb, g, lid, rb, rc, c0, nc);
                meet_sync<BAR, BLOCK, GBAR0, GTH, G>(g);
                if (mine) {
                    const Row<R>* Jm = tb.J(g, p, M);
                    const Row<R>* RV = tb.RV(g, p);
#pragma unroll 1
                    for (int t = gt; t < nc; t += GT) {
                        const unsigned T = tb.LIST[set_level_offset(N, M) + c0 + t], V = FULL & ~T;
                        meet_contract<R, N, CB, M, MK, CH>((int)(T & ((1u << CB) - 1)), Jm, RV, t, px[T >> CB],
                                                           px[V >> CB], are, aim);
                    }
                }
                if (c0 + CH < CM) meet_sync<BAR, BLOCK, GBAR0, GTH, G>(g);   // before the next chunk's currents
            }
            // the groups' amplitudes, configuration-major (entry ((u PG + p) 2^CB
            // + b) CT + hi for lambda = (hi << CB) | b): a warp's lanes store
            // consecutive words
            if (mine) {
                R* xa = tb.XA(g) + (((size_t)gt * PG + p) << CB) * CT * 2 + (size_t)hi * 2;
#pragma unroll
                for (int b = 0; b < (1 << CB); ++b) {
                    using V2 = typename std::conditional<sizeof(R) == sizeof(float), float2, double2>::type;
                    V2 v2;
                    v2.x = are[b];
                    v2.y = aim[b];
                    *reinterpret_cast<V2*>(xa + (size_t)b * CT * 2) = v2;
                }
            }
            meet_sync<BAR, BLOCK, GBAR0, GTH, G>(g);
            // one warp per point: groups added in order, w_h |A_h|^2 summed
            // over h (lane order: hi fastest, as stored)
            for (int q = lid >> 5; q < rc; q += GTH / 32) {
                const int lane = lid & 31;
                const bool valid = rb[q].valid;
                const int hsel = valid ? rb[q].hsel : -1;
                R v = R(0);
                if (valid)
                    for (int x = lane; x < NS; x += 32) {
                        const int hh = x % CT, b = x / CT;
                        const unsigned h = ((unsigned)hh << CB) | (unsigned)b;
                        R ar = R(0), ai = R(0);
#pragma unroll
                        for (int u = 0; u < GT; ++u) {
                            const R* a = tb.XA(g) + ((((size_t)u * PG + q) << CB) + b) * CT * 2 + (size_t)hh * 2;
                            ar += a[0];
                            ai += a[1];
                        }
                        v += (ar * ar + ai * ai) * R(sel_weight<N>(hsel, h, lane_weight<N>(mask, h)));
                    }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
                if (lane == 0) recs[base + q].ssum = valid ? v : R(0);
            }
            meet_sync<BAR, BLOCK, GBAR0, GTH, G>(g);
        }
    }
    group_sync<BAR, BLOCK>();
}

}  // namespace heget
