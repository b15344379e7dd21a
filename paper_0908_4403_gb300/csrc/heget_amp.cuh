// heget_amp.cuh -- helicity amplitudes of u ubar -> n photons on the
// prefix-shared ordering tree (Sec. 2.1 eqs. (6)-(8); the permutation program
// of Appendix A.2 and the unrolled loop of Appendix C, re-designed).
//
// Chiral (Weyl) basis, gamma5 = diag(-1,-1,+1,+1) (the block convention of
// Sec. 4 / Appendix B.3).  For massless quarks the chain keeps chirality, so
// with s1 = + only the lower (right-handed) block of u(p1) and the upper
// block of vbar(p2) survive (s2 = -s1 is forced; s1 = s2 amplitudes are
// exact zeros).  Reading the chain from the vbar end, every step
//     r <- r . (eps*_j . sigma) (q_T . sigmabar) / q_T^2,
//     q_T = sum_{i in T} k_i - p2,   T = photons attached so far,
// maps an upper-block row 2-spinor (2 complex numbers) to another one: the
// massless off-shell fermion of fvoxx0 (Appendix B.3.3) in two components.
// The vertex closure with the photon next to u(p1) is iovxx0 (Appendix
// B.3.1): A = r . (eps*_j . sigma) . u_R.
//
// Prefix sharing: the current after an ordered prefix is computed once and
// extended by every remaining photon (depth-first, registers hold the stack),
// so the tree does sum_{l=1}^{n-1} n!/(n-l)! steps and n! closures per
// helicity instead of n! (n-1) steps.  The step matrices M(j, T) depend on
// (j, T, lambda_j) only and are precomputed per point in shared memory.  From
// n = 4 the walk also shares the suffix of the last two photons (the
// two-ended finish below), which removes the level of n! steps.
//
// Lanes: each lane carries one to four photon-helicity configurations h in
// [0, 2^n) with s1 = + (TreeShape); the lanes of a warp walk the same
// subtrees (uniform control flow), reading the same table entries up to the
// lambda_j bit (broadcast loads).  The s1 = - configurations follow from
// parity, |M_{-h}|^2 = |M_h|^2 (checked against the oracle), folded into a
// per-configuration weight w_h = [mask(+,-,h)] + [mask(-,+,~h)].
#pragma once

#include "heget_ps.cuh"

namespace heget {

// a complex pair (a, b): a row 2-spinor, or one row of a 2x2 matrix
template <class R>
struct alignas(16) Row {
    R ar, ai, br, bi;
};

__device__ __forceinline__ Row<float> ld_row(const Row<float>* p) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    return Row<float>{v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ Row<double> ld_row(const Row<double>* p) {
    const double2 a = reinterpret_cast<const double2*>(p)[0];
    const double2 b = reinterpret_cast<const double2*>(p)[1];
    return Row<double>{a.x, a.y, b.x, b.y};
}
__device__ __forceinline__ void st_row(Row<float>* p, const Row<float>& r) {
    *reinterpret_cast<float4*>(p) = make_float4(r.ar, r.ai, r.br, r.bi);
}
__device__ __forceinline__ void st_row(Row<double>* p, const Row<double>& r) {
    reinterpret_cast<double2*>(p)[0] = make_double2(r.ar, r.ai);
    reinterpret_cast<double2*>(p)[1] = make_double2(r.br, r.bi);
}

// r . M with M given by its rows m0 = (M00, M01), m1 = (M10, M11)
template <class R>
__device__ __forceinline__ Row<R> row_times(const Row<R>& r, const Row<R>& m0, const Row<R>& m1) {
    Row<R> o;
    o.ar = r.ar * m0.ar - r.ai * m0.ai + r.br * m1.ar - r.bi * m1.ai;
    o.ai = r.ar * m0.ai + r.ai * m0.ar + r.br * m1.ai + r.bi * m1.ar;
    o.br = r.ar * m0.br - r.ai * m0.bi + r.br * m1.br - r.bi * m1.bi;
    o.bi = r.ar * m0.bi + r.ai * m0.br + r.br * m1.bi + r.bi * m1.br;
    return o;
}

// Barrier of the threads that run the amplitude rounds: the whole block
// (BAR = 0, __syncthreads) or, in a warp-specialised block, the BLOCK
// consumer threads on named barrier BAR.
template <int BAR, int BLOCK>
__device__ __forceinline__ void group_sync() {
    if constexpr (BAR == 0) {
        __syncthreads();
    } else {
        asm volatile("bar.sync %0, %1;" ::"n"(BAR), "n"(BLOCK) : "memory");
    }
}

template <class R> __device__ __forceinline__ R recip(R x);
template <> __device__ __forceinline__ float recip<float>(float x) { return __frcp_rn(x); }
template <> __device__ __forceinline__ double recip<double>(double x) { return 1.0 / x; }
template <class R> __device__ __forceinline__ R rsq(R x);
template <> __device__ __forceinline__ float rsq<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rsq<double>(double x) { return rsqrt(x); }

template <class R> __device__ __forceinline__ R fmad(R a, R b, R c);
template <> __device__ __forceinline__ float fmad<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <> __device__ __forceinline__ double fmad<double>(double a, double b, double c) { return __fma_rn(a, b, c); }

// Lane layout of the tree (a compile-time shape HB, G):
//   * HB = 0: one photon-helicity configuration per lane; the 2^n lanes of a
//     point are contiguous, and G groups (whole warps) split the ordered
//     prefixes of depth D0 between them (prefix k goes to group k % G) and add
//     their partial amplitudes before squaring.
//   * HB = 2 ("pair units"): the orderings are cut into units, one per
//     unordered photon pair {p, q}: those that start with p, q or with q, p.
//     A lane carries the four configurations of (lambda_p, lambda_q) as rows
//     and its 2^(n-2) lanes per point the helicities of the other photons.
//     Below the first two levels every photon the walk attaches is one of the
//     others, so all rows of a lane read the same table entry and a single
//     code path serves every step; the table loads and the index work of a
//     step are spread over four row updates.  G slots (whole warps holding
//     P points) take the units u = g, g + G, ...; a slot adds its units'
//     amplitudes into its own accumulator per absolute helicity, and the
//     slots are added in a fixed order after the walk.
//   * thread t: group or slot g = t / (P 2^NB), point slot (t / 2^NB) % P,
//     lane bits hl = t % 2^NB (NB = n - HB).
// The walk below depth D0 keeps one row set per level in registers; at n = 8
// the pair units recompute the top of the stack (two steps) per depth-3
// prefix instead of holding it.
template <int N, int BLOCK, int HB, int G>
struct TreeShape {
    static constexpr int H = 1 << HB;
    static constexpr int NB = N - HB;
    static constexpr int NSL = 1 << NB;      // lanes of one point
    static constexpr int GL = BLOCK / G;     // lanes of a group
    static constexpr int P = GL / NSL;       // points per round
    static constexpr bool PAIRS = HB == 2;
    static constexpr int D0 = PAIRS ? (N == 8 ? 3 : 2) : N >= 3 ? 2 : 1;
    // units of work shared out over the groups: pairs, or ordered prefixes
    static constexpr int NPRE = PAIRS ? N * (N - 1) / 2 : D0 == 2 ? N * (N - 1) : N;
    static_assert(HB == 0 || (HB == 2 && N >= 4), "one configuration per lane, or pair units");
    static_assert(BLOCK % G == 0 && GL % NSL == 0 && P >= 1, "a round holds whole points");
    static_assert(G == 1 || GL % 32 == 0, "groups fill whole warps");
};

// Two-ended finish of the tree (sub-current reuse from the u side): with two
// photons a, b left after an ordered prefix, the two remaining orderings are
//   r . M(a, all - {b}) . cl_b  +  r . M(b, all - {a}) . cl_a,
// and the pair columns PC(a -> b) = M(a, all - {b}) . cl_b depend only on
// (a, b, lambda_a, lambda_b), not on the prefix: computed once per point,
// they turn the last level of steps (n! per lane) into closures.  The walk
// then never uses the step matrices of the sets of n - 1 photons; the pair
// columns form theirs directly, and the round tables leave them out, which
// costs about what the pair columns take.  Compiled in for n >= 4 (at n = 3
// the extra table phase costs more than the level it saves).
// -DHEGET_TWO_ENDED=0 turns it off.
#ifndef HEGET_TWO_ENDED
#define HEGET_TWO_ENDED 1
#endif
template <class R, int N>
__host__ __device__ constexpr bool tree_two_ended() {
    return HEGET_TWO_ENDED && N >= 4;
}

// Ordered pair (a, b), a != b, as an index in [0, n(n-1)).
template <int N>
__host__ __device__ __forceinline__ int pair_slot(int a, int b) {
    return a * (N - 1) + b - (b > a);
}

// Unordered pair u (lexicographic over p < q) -> (p, q).
template <int N>
__host__ __device__ __forceinline__ void pair_of_unit(int u, int& p, int& q) {
    p = 0;
    while (u >= N - 1 - p) {
        u -= N - 1 - p;
        ++p;
    }
    q = p + 1 + u;
}

// The n - 2 helicity bits of a pair unit's lane spread over the photons other
// than p < q (zeros at p and q).
__host__ __device__ __forceinline__ unsigned spread_pair_bits(unsigned hl, int p, int q) {
    const unsigned x = (hl & ((1u << p) - 1u)) | ((hl >> p) << (p + 1));
    return (x & ((1u << q) - 1u)) | ((x >> q) << (q + 1));
}

// Shared-memory tables of one round.  Every lane of a point reads one index
// for its point and one lambda, so entries are laid out [index][point][lambda]
// (plus the two rows of a step matrix next to each other): the lanes of a
// warp hit a few consecutive 16-byte rows.
template <class R, int N, int BLOCK, int HB = 0, int G = 1>
struct RoundTables {
    using S = TreeShape<N, BLOCK, HB, G>;
    static constexpr int P = S::P;
    static constexpr int K = num_pairs(N);
    // step matrices held: with the two-ended finish, those of sets of at
    // most n - 2 photons (the pair index lists them first)
    static constexpr int KW = tree_two_ended<R, N>() ? K - N * (N - 1) : K;
    static constexpr int NS = 1 << N;
    static constexpr size_t m_elems = (size_t)KW * P * 4;   // [idx][p][lambda][row 0, row 1]
    static constexpr size_t c_elems = (size_t)N * P * 2;    // [j][p][lambda]
    // group exchange: partial amplitudes per lane (ordered-prefix groups), or
    // the slots' accumulators per absolute helicity (pair units)
    static constexpr size_t x_elems = S::PAIRS ? (size_t)G * P * NS * 2 : G > 1 ? (size_t)BLOCK * 2 : 0;
    static constexpr size_t p_elems = tree_two_ended<R, N>() ? (size_t)N * (N - 1) * P * 4 : 0;
    static constexpr size_t bytes = (m_elems + 2 * c_elems + p_elems) * sizeof(Row<R>)   // MT, CL, R1, PC
                                  + (size_t)P * N * sizeof(Row<R>)                      // photon data
                                  + (size_t)P * NS * sizeof(Row<R>)                     // set data
                                  + x_elems * sizeof(R)                                 // exchange
                                  + (size_t)(BLOCK / 32) * sizeof(R) + 16;              // reduction
    Row<R>* MT;   // step matrices M(j, T)^lambda
    Row<R>* CL;   // closures (eps*_j . sigma) u_R
    Row<R>* R1;   // first rows vbar(p2) . M(j, {j})
    Row<R>* PC;   // [pair_slot(a, b)][P][lambda_a 2 + lambda_b]: pair columns (two-ended finish)
    Row<R>* PH;   // [P][N]: (sin th, cos th, cos ph, sin ph)
    Row<R>* SD;   // [P][2^N]: (A, D, Bre, Bim) = ((q0+q3), (q0-q3), q1, q2) / q^2
    R* XCH;       // [BLOCK][2], or [G][P][2^N][2] with pair units
    R* RED;       // [BLOCK/32]
    __device__ __forceinline__ explicit RoundTables(unsigned char* base) {
        MT = reinterpret_cast<Row<R>*>(base);
        CL = MT + m_elems;
        R1 = CL + c_elems;
        PC = R1 + c_elems;
        PH = PC + p_elems;
        SD = PH + (size_t)P * N;
        XCH = reinterpret_cast<R*>(SD + (size_t)P * NS);
        RED = XCH + x_elems;
    }
};

// Photon direction (sin th, cos th, cos ph, sin ph) of momentum k.
template <class R>
__device__ __forceinline__ Row<R> photon_row(const R* k) {
    const R pt2 = k[1] * k[1] + k[2] * k[2];
    const R ka2 = pt2 + k[3] * k[3];
    const R rk = rsq<R>(ka2);
    Row<R> d;
    d.ai = k[3] * rk;                        // cos theta
    if (pt2 > R(1e-24) * ka2) {
        const R rpt = rsq<R>(pt2);
        d.ar = pt2 * rpt * rk;               // sin theta
        d.br = k[1] * rpt;                   // cos phi
        d.bi = k[2] * rpt;                   // sin phi
    } else {  // photon along z: the phi -> 0 limit of the polarisation
        d.ar = R(0);
        d.br = R(1);
        d.bi = R(0);
    }
    return d;
}

// Set data (q0+q3, q0-q3, q1, q2) / t_T of set T (0 < T < 2^N - 1), q_T =
// sum_{i in T} k_i - p2, from a record: t_T as the record holds it (from
// FP64, rounded once) or as the float-float sum of its invariants.
template <class R, int N>
__device__ __forceinline__ Row<R> set_row(const PointRec<R, N>& rc, unsigned T) {
    R q0 = -rc.e2, q1 = R(0), q2 = R(0), q3 = rc.e2;
#pragma unroll
    for (int i = 0; i < N; ++i)
        if (T >> i & 1) {
            q0 += rc.k[i][0];
            q1 += rc.k[i][1];
            q2 += rc.k[i][2];
            q3 += rc.k[i][3];
        }
    R tT;
    if constexpr (rec_invariants<R, N>()) tT = rec_denominator<N>(rc.inv, T);
    else tT = rc.t[T];
    const R it_ = recip<R>(tT);
    return Row<R>{(q0 + q3) * it_, (q0 - q3) * it_, q1 * it_, q2 * it_};
}

// Photon data PH[p][j] (photon_row) and set data SD[p][T] (set_row) for the
// points recs[0 .. cnt-1] (P slots).  Everything runs in R: the records hold
// t_T from FP64, or the FP64 invariants it is a float-float sum of.  list
// (optional): the sets by size (build_set_list), the order in which the
// threads take them, so that the float-float sums of a warp's lanes share
// their loop counts.
template <class R, int N, int BLOCK, int P>
__device__ __forceinline__ void setup_photons_and_sets(Row<R>* PH, Row<R>* SD, const PointRec<R, N>* recs, int cnt,
                                                       const unsigned char* list = nullptr) {
    constexpr int NS = 1 << N;
    const int tid = threadIdx.x;
    constexpr int n_ph = P * N, n_sd = P * NS;
    for (int it = tid; it < n_ph + n_sd; it += BLOCK) {
        if (it < n_ph) {
            const int p = it / N, j = it - p * N;
            if (p >= cnt) continue;
            PH[p * N + j] = photon_row<R>(recs[p].k[j]);
        } else {
            const int r = it - n_ph;
            const int p = r / NS, e = r - p * NS;
            const int T = list ? (int)list[e] : e;
            if (p >= cnt || T == 0 || T == NS - 1) continue;
            SD[p * NS + T] = set_row<R, N>(recs[p], (unsigned)T);
        }
    }
}

// Step matrix M = E Qbar of photon (ph) into set (sd) for lambda = +-1
// (lam_bit 1/0), with E = eps*(k, lambda) . sigma, or (k/k^0) . sigma for the
// gauge check; also returns E's first column (the closure against u_R).
template <class R>
struct StepMat {
    Row<R> m0, m1;   // rows (M00, M01), (M10, M11)
    R e00, e10r, e10i;
};

template <class R>
__device__ __forceinline__ StepMat<R> step_matrix(const Row<R>& ph, const Row<R>& sd, int lam_bit, bool ward) {
    const R rs2 = R(0.70710678118654752440);
    const R lam = lam_bit ? R(1) : R(-1);
    // E = eps*(k, lambda) . sigma = (1/sqrt2) [[-l s, -(1 - l c) e^{-i phi}],
    //                                         [(1 + l c) e^{i phi}, l s]]
    R e00 = -lam * ph.ar * rs2;
    R e11 = -e00;
    const R am = (R(1) - lam * ph.ai) * rs2, ap = (R(1) + lam * ph.ai) * rs2;
    R e01r = -am * ph.br, e01i = am * ph.bi;   // -(1 - l c) e^{-i phi}
    R e10r = ap * ph.br, e10i = ap * ph.bi;    //  (1 + l c) e^{+i phi}
    if (ward) {
        // (k/k^0) . sigma = [[1 - c, -s e^{-i phi}], [-s e^{i phi}, 1 + c]]
        e00 = R(1) - ph.ai;
        e11 = R(1) + ph.ai;
        e01r = -ph.ar * ph.br;
        e01i = ph.ar * ph.bi;
        e10r = -ph.ar * ph.br;
        e10i = -ph.ar * ph.bi;
    }
    // Qbar = [[A, B*], [B, D]], B = Bre + i Bim
    const R A = sd.ar, D = sd.ai, Br = sd.br, Bi = sd.bi;
    StepMat<R> o;
    o.m0.ar = e00 * A + e01r * Br - e01i * Bi;   // M00 = e00 A + e01 B
    o.m0.ai = e01r * Bi + e01i * Br;
    o.m0.br = e00 * Br + e01r * D;               // M01 = e00 B* + e01 D
    o.m0.bi = -e00 * Bi + e01i * D;
    o.m1.ar = e10r * A + e11 * Br;               // M10 = e10 A + e11 B
    o.m1.ai = e10i * A + e11 * Bi;
    o.m1.br = e10r * Br + e10i * Bi + e11 * D;   // M11 = e10 B* + e11 D
    o.m1.bi = e10i * Br - e10r * Bi;
    o.e00 = e00;
    o.e10r = e10r;
    o.e10i = e10i;
    return o;
}

// acc += r . c, c = (ca, cb) a column 2-spinor: a chain of fused
// multiply-adds into the accumulator (8 per closure)
template <class R>
__device__ __forceinline__ void close_row(const Row<R>& r, const Row<R>& c, R& are, R& aim) {
    are = fmad<R>(r.ar, c.ar, are);
    are = fmad<R>(-r.ai, c.ai, are);
    are = fmad<R>(r.br, c.br, are);
    are = fmad<R>(-r.bi, c.bi, are);
    aim = fmad<R>(r.ar, c.ai, aim);
    aim = fmad<R>(r.ai, c.ar, aim);
    aim = fmad<R>(r.br, c.bi, aim);
    aim = fmad<R>(r.bi, c.br, aim);
}

// Fill the round tables for points recs[0 .. cnt-1] (cnt <= P).  Phases
// separated by barriers; all threads of the block must call it.  Everything
// here runs in R: the FP64 content (invariants) is already in the records.
// ward >= 0 replaces the polarisation of that photon by k/k^0 in every step,
// closure and first row (the gauge check; both lambda entries then agree).
template <class R, int N, int BLOCK, int BAR = 0, int HB = 0, int G = 1>
__device__ __forceinline__ void setup_round(const RoundTables<R, N, BLOCK, HB, G>& tb, const PointRec<R, N>* recs,
                                            int cnt, int ward = -1) {
    using RT = RoundTables<R, N, BLOCK, HB, G>;
    constexpr int P = RT::P, K = RT::KW, NS = RT::NS;
    const int tid = threadIdx.x;
    setup_photons_and_sets<R, N, BLOCK, P>(tb.PH, tb.SD, recs, cnt);
    group_sync<BAR, BLOCK>();
    // (b) step matrices M(j, T) = E_j^lambda Qbar_T, closures and first rows
    for (int it = tid; it < P * K * 2; it += BLOCK) {
        const int lam_bit = it & 1;
        const int q = it >> 1;
        const int p = q % P;
        const int idx = q / P;
        if (p >= cnt) continue;
        const uint16_t pr = c_tables.pair[pair_offset(N) + idx];
        const int T = pr & 0xFF, j = pr >> 8;
        const StepMat<R> sm = step_matrix<R>(tb.PH[p * N + j], tb.SD[p * NS + T], lam_bit, j == ward);
        const Row<R>& m1 = sm.m1;
        const size_t o = (((size_t)idx * P + p) * 2 + lam_bit) * 2;
        st_row(tb.MT + o, sm.m0);
        st_row(tb.MT + o + 1, m1);
        if (T == (1 << j)) {
            const size_t oc = ((size_t)j * P + p) * 2 + lam_bit;
            const R n1 = recs[p].n1;
            const R n2 = recs[p].n2;
            st_row(tb.CL + oc, Row<R>{n1 * sm.e00, R(0), n1 * sm.e10r, n1 * sm.e10i});
            st_row(tb.R1 + oc, Row<R>{n2 * m1.ar, n2 * m1.ai, n2 * m1.br, n2 * m1.bi});
        }
    }
    group_sync<BAR, BLOCK>();
    if constexpr (tree_two_ended<R, N>()) {
        // (c) pair columns PC(a -> b) = M(a, all - {b}) . cl_b
        constexpr unsigned FULL = (1u << N) - 1;
        for (int it = tid; it < N * (N - 1) * P * 2; it += BLOCK) {
            const int la = it & 1, q = it >> 1;
            const int p = q % P, k = q / P;
            if (p >= cnt) continue;
            const int a = k / (N - 1), t = k - a * (N - 1), b = t + (t >= a);
            // M(a, all - {b}), not held in the step tables, once for both lambda_b
            const StepMat<R> sm = step_matrix<R>(tb.PH[p * N + a], tb.SD[p * NS + (FULL & ~(1u << b))], la, a == ward);
#pragma unroll
            for (int lb = 0; lb < 2; ++lb) {
                const Row<R> c = ld_row(tb.CL + ((size_t)b * P + p) * 2 + lb);
                Row<R> pc{R(0), R(0), R(0), R(0)};
                // (M c)_0 = m0 . c, (M c)_1 = m1 . c, as a column (a, b)
                close_row(sm.m0, c, pc.ar, pc.ai);
                close_row(sm.m1, c, pc.br, pc.bi);
                st_row(tb.PC + ((size_t)k * P + p) * 4 + la * 2 + lb, pc);
            }
        }
        group_sync<BAR, BLOCK>();
    }
}

// Per-lane view of the round tables: pointers already offset to the lane's
// point slot; per table index the step matrices advance by 4P rows, the
// closures and first rows by 2P per photon, the pair columns by 4P per pair.
template <class R, int N, int BLOCK, int HB = 0, int G = 1>
struct LaneTables {
    const Row<R>* mt;
    const Row<R>* cl;
    const Row<R>* r1;
    const Row<R>* pc;
    unsigned hl;  // lambda bits of the photons the walk attaches (bit set -> +1)
};

template <class R, int N, int BLOCK, int HB, int G>
__device__ __forceinline__ LaneTables<R, N, BLOCK, HB, G> lane_tables(const RoundTables<R, N, BLOCK, HB, G>& tb,
                                                                      int slot, unsigned hl) {
    return LaneTables<R, N, BLOCK, HB, G>{tb.MT + 4 * slot, tb.CL + 2 * slot, tb.R1 + 2 * slot, tb.PC + 4 * slot,
                                          hl};
}

// Rows r[b] . M: every row of the lane takes the same step matrix.
template <class R, int H>
__device__ __forceinline__ void step_same(Row<R> (&o)[H], const Row<R> (&r)[H], const Row<R>& m0, const Row<R>& m1) {
#pragma unroll
    for (int b = 0; b < H; ++b) o[b] = row_times(r[b], m0, m1);
}

// Attach photon j to the rows (table entry index idx).
template <class R, int N, int BLOCK, int HB, int G>
__device__ __forceinline__ void attach(const LaneTables<R, N, BLOCK, HB, G>& L, int j, int idx,
                                       const Row<R> (&r)[1 << HB], Row<R> (&o)[1 << HB]) {
    constexpr int P = TreeShape<N, BLOCK, HB, G>::P;
    const Row<R>* e = L.mt + idx * (4 * P) + ((L.hl >> j) & 1) * 2;
    step_same<R, 1 << HB>(o, r, ld_row(e), ld_row(e + 1));
}

// Closure with the last photon j (iovxx0 against u(p1)).
template <class R, int N, int BLOCK, int HB, int G>
__device__ __forceinline__ void close_rows(const LaneTables<R, N, BLOCK, HB, G>& L, int j, const Row<R> (&r)[1 << HB],
                                           R (&are)[1 << HB], R (&aim)[1 << HB]) {
    constexpr int P = TreeShape<N, BLOCK, HB, G>::P;
    const Row<R> c = ld_row(L.cl + j * (2 * P) + ((L.hl >> j) & 1));
#pragma unroll
    for (int b = 0; b < (1 << HB); ++b) close_row(r[b], c, are[b], aim[b]);
}

// The two orderings left below a node of depth n - 2 by the pair columns:
// acc += r . PC(a -> b) + r . PC(b -> a) (s_ab, s_ba: the ordered pair slots).
template <class R, int N, int BLOCK, int HB, int G>
__device__ __forceinline__ void close_pair_slots(const LaneTables<R, N, BLOCK, HB, G>& L, int a, int b, int s_ab,
                                                 int s_ba, const Row<R> (&r)[1 << HB], R (&are)[1 << HB],
                                                 R (&aim)[1 << HB]) {
    constexpr int P = TreeShape<N, BLOCK, HB, G>::P;
    const int la = (L.hl >> a) & 1, lb = (L.hl >> b) & 1;
    const Row<R> c1 = ld_row(L.pc + s_ab * (4 * P) + la * 2 + lb);
    const Row<R> c2 = ld_row(L.pc + s_ba * (4 * P) + lb * 2 + la);
#pragma unroll
    for (int row = 0; row < (1 << HB); ++row) {
        close_row(r[row], c1, are[row], aim[row]);
        close_row(r[row], c2, are[row], aim[row]);
    }
}

template <class R, int N, int BLOCK, int HB, int G>
__device__ __forceinline__ void close_pair(const LaneTables<R, N, BLOCK, HB, G>& L, int a, int b,
                                           const Row<R> (&r)[1 << HB], R (&are)[1 << HB], R (&aim)[1 << HB]) {
    close_pair_slots<R, N, BLOCK, HB, G>(L, a, b, pair_slot<N>(a, b), pair_slot<N>(b, a), r, are, aim);
}

// First rows vbar(p2) . M(j, {j}) for the lane's helicities.
template <class R, int N, int BLOCK, int HB, int G>
__device__ __forceinline__ void first_rows(const LaneTables<R, N, BLOCK, HB, G>& L, int j, Row<R> (&r)[1 << HB]) {
    constexpr int P = TreeShape<N, BLOCK, HB, G>::P;
    const Row<R> a = ld_row(L.r1 + j * (2 * P) + ((L.hl >> j) & 1));
#pragma unroll
    for (int b = 0; b < (1 << HB); ++b) r[b] = a;
}

__device__ __forceinline__ int tree_child(int n, unsigned T, int j) {
    return c_tables.child[child_offset(n) + T * n + j];
}

// The bottom three levels of the walk, written out from the per-set index
// entry (Bottom3): below a node with rows r and three photons a < b < c
// left, attach each of them and close the two orderings of the other two by
// the pair columns.
template <class R, int N, int BLOCK, int HB, int G>
__device__ __forceinline__ void bottom3(const LaneTables<R, N, BLOCK, HB, G>& L, const Row<R> (&r)[1 << HB],
                                        unsigned T, R (&are)[1 << HB], R (&aim)[1 << HB]) {
    constexpr int P = TreeShape<N, BLOCK, HB, G>::P, H = 1 << HB;
    constexpr unsigned FULL = (1u << N) - 1;
    const unsigned rem = FULL & ~T, rem2 = rem & (rem - 1);
    const int x[3] = {__ffs(rem) - 1, __ffs(rem2) - 1, __ffs(rem2 & (rem2 - 1)) - 1};
    const Bottom3& e = c_bottom.e[bottom_offset(N) + T];
#pragma unroll
    for (int u = 0; u < 3; ++u) {
        const int j = x[u], y = x[u == 0 ? 1 : 0], z = x[u == 2 ? 1 : 2];
        Row<R> r2[H];
        const Row<R>* m = L.mt + e.st[u] * (4 * P) + ((L.hl >> j) & 1) * 2;
        step_same<R, H>(r2, r, ld_row(m), ld_row(m + 1));
        close_pair_slots<R, N, BLOCK, HB, G>(L, y, z, e.pc[2 * u], e.pc[2 * u + 1], r2, are, aim);
    }
}

// Depth-first walk of the ordering tree below a node at depth D (D photons
// attached, set T, current rows r), adding the closures to acc.  The last
// three levels are written out (bottom3); above them the loop stays rolled.
template <class R, int N, int D, int BLOCK, int HB, int G>
__device__ __forceinline__ void descend(const LaneTables<R, N, BLOCK, HB, G>& L, const Row<R> (&r)[1 << HB],
                                        unsigned T, R (&are)[1 << HB], R (&aim)[1 << HB]) {
    constexpr unsigned FULL = (1u << N) - 1;
    if constexpr (D == N - 1) {
        close_rows<R, N, BLOCK, HB, G>(L, __ffs(FULL & ~T) - 1, r, are, aim);
    } else if constexpr (D == N - 2 && tree_two_ended<R, N>()) {
        const unsigned rem = FULL & ~T;
        close_pair<R, N, BLOCK, HB, G>(L, __ffs(rem) - 1, __ffs(rem & (rem - 1)) - 1, r, are, aim);
    } else if constexpr (D == N - 3 && tree_two_ended<R, N>() && N >= 5) {
        bottom3<R, N, BLOCK, HB, G>(L, r, T, are, aim);
    } else {
        unsigned rem = FULL & ~T;
#pragma unroll 1
        while (rem) {
            const int j = __ffs(rem) - 1;
            rem &= rem - 1;
            Row<R> r2[1 << HB];
            attach<R, N, BLOCK, HB, G>(L, j, tree_child(N, T, j), r, r2);
            descend<R, N, D + 1, BLOCK, HB, G>(L, r2, T | (1u << j), are, aim);
        }
    }
}

// Ordered prefix k (lexicographic) of depth D = 2 or 3: photons j1, j2 (, j3).
template <int N, int D>
__host__ __device__ __forceinline__ void tree_prefix(int k, int& j1, int& j2, int& j3) {
    if constexpr (D == 2) {
        j1 = k / (N - 1);
        const int t = k - j1 * (N - 1);
        j2 = t + (t >= j1);
        j3 = -1;
    } else {
        constexpr int W2 = (N - 1) * (N - 2);
        j1 = k / W2;
        const int t = k - j1 * W2;
        const int t2 = t / (N - 2), t3 = t - t2 * (N - 2);
        j2 = t2 + (t2 >= j1);
        // j3: the t3-th photon (in order) other than j1 and j2
        const int lo = j1 < j2 ? j1 : j2, hi = j1 < j2 ? j2 : j1;
        j3 = t3 + (t3 >= lo);
        j3 += j3 >= hi;
    }
}

// The orderings of group g for one lane with one configuration per lane: the
// subtrees below the ordered prefixes k = g, g + G, ... of depth D0
// (lexicographic), each prefix's row formed from the first row by one step.
// Sums the helicity amplitude (up to normalisation) for s1 = +.  g is the
// same for every lane of a warp, so every loop bound and table index below is
// warp-uniform.
template <class R, int N, int BLOCK, int G>
__device__ __forceinline__ void tree_amplitude(const LaneTables<R, N, BLOCK, 0, G>& L, int g, R (&are)[1],
                                               R (&aim)[1]) {
    using S = TreeShape<N, BLOCK, 0, G>;
    are[0] = aim[0] = R(0);
#pragma unroll 1
    for (int k = g; k < S::NPRE; k += G) {
        if constexpr (S::D0 == 1) {
            Row<R> r1[1];
            first_rows<R, N, BLOCK, 0, G>(L, k, r1);
            descend<R, N, 1, BLOCK, 0, G>(L, r1, 1u << k, are, aim);
        } else {
            int j1, j2, j3;
            tree_prefix<N, 2>(k, j1, j2, j3);
            Row<R> r1[1], r2[1];
            first_rows<R, N, BLOCK, 0, G>(L, j1, r1);
            attach<R, N, BLOCK, 0, G>(L, j2, tree_child(N, 1u << j1, j2), r1, r2);
            descend<R, N, 2, BLOCK, 0, G>(L, r2, (1u << j1) | (1u << j2), are, aim);
        }
    }
}

// The rows (lambda_p, lambda_q) = (bit 0, bit 1 of the row) after the first
// two photons j1, j2 of the ordering, {j1, j2} = {p, q}: the first row of j1
// and the step of j2, each row with its own lambdas (sh1: the row bit of j1).
template <class R, int N, int BLOCK, int G>
__device__ __forceinline__ void pair_top(const LaneTables<R, N, BLOCK, 2, G>& L, int j1, int j2, int sh1,
                                         Row<R> (&r2)[4]) {
    constexpr int P = TreeShape<N, BLOCK, 2, G>::P;
    const Row<R>* f = L.r1 + j1 * (2 * P);
    const Row<R>* m = L.mt + tree_child(N, 1u << j1, j2) * (4 * P);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const int l1 = (b >> sh1) & 1, l2 = (b >> (1 - sh1)) & 1;
        r2[b] = row_times(ld_row(f + l1), ld_row(m + 2 * l2), ld_row(m + 2 * l2 + 1));
    }
}

// One pair unit {p, q} for one lane: the orderings that start with (p, q) or
// (q, p), every row with its (lambda_p, lambda_q); the lane's view L carries
// the other photons' lambdas (zeros at p and q).
template <class R, int N, int BLOCK, int G>
__device__ __forceinline__ void pair_unit(const LaneTables<R, N, BLOCK, 2, G>& L, int p, int q, R (&are)[4],
                                          R (&aim)[4]) {
    const unsigned T2 = (1u << p) | (1u << q);
#pragma unroll 1
    for (int o = 0; o < 2; ++o) {
        const int j1 = o ? q : p, j2 = o ? p : q;
        if constexpr (TreeShape<N, BLOCK, 2, G>::D0 == 2) {
            Row<R> r2[4];
            pair_top<R, N, BLOCK, G>(L, j1, j2, o, r2);
            descend<R, N, 2, BLOCK, 2, G>(L, r2, T2, are, aim);
        } else {
            // depth-3 prefixes: the two top levels recomputed per third photon
            unsigned rem = ((1u << N) - 1) & ~T2;
#pragma unroll 1
            while (rem) {
                const int j3 = __ffs(rem) - 1;
                rem &= rem - 1;
                Row<R> r2[4], r3[4];
                pair_top<R, N, BLOCK, G>(L, j1, j2, o, r2);
                attach<R, N, BLOCK, 2, G>(L, j3, tree_child(N, T2, j3), r2, r3);
                descend<R, N, 3, BLOCK, 2, G>(L, r3, T2 | (1u << j3), are, aim);
            }
        }
    }
}

// Parity-folded helicity weight of photon-helicity configuration h (see file
// comment): w_h = [mask(+,-,h)] + [mask(-,+,~h)], 2 without a mask.
template <int N>
__device__ __forceinline__ float lane_weight(const uint32_t* mask, unsigned h) {
    if (!mask) return 2.0f;
    const unsigned full = (1u << N) - 1;
    const unsigned hp = 1u | (h << 2);
    const unsigned hm = 2u | ((~h & full) << 2);
    const unsigned bp = (__ldg(mask + (hp >> 5)) >> (hp & 31)) & 1u;
    const unsigned bm = (__ldg(mask + (hm >> 5)) >> (hm & 31)) & 1u;
    return (float)(bp + bm);
}

// Weight of lane lam for a point whose record selects `hsel` (PointRec):
// w (the mask's) for every lane when hsel = -1, else 2^(n+2) for the selected
// lane only (a sampled helicity counts for all 2^(n+2)).
template <int N>
__device__ __forceinline__ float sel_weight(int hsel, unsigned lam, float w) {
    return hsel == -1 ? w : (int)lam == hsel ? (float)(1 << (N + 2)) : 0.0f;
}


// Lane coordinates in a round: group or slot, point slot, lane bits.
template <int N, int BLOCK, int HB, int G>
struct LaneId {
    using S = TreeShape<N, BLOCK, HB, G>;
    int g, slot, hl;
    __device__ __forceinline__ explicit LaneId(int tid)
        : g(tid / S::GL), slot((tid % S::GL) / S::NSL), hl(tid % S::NSL) {}
};

// One configuration per lane, several groups: every group leaves its partial
// sums in shared memory and group 0 adds them in group order (the other
// groups' amplitudes become 0).  All threads must call it.
template <class R, int N, int BLOCK, int BAR, int G>
__device__ __forceinline__ void combine_groups(const RoundTables<R, N, BLOCK, 0, G>& tb, const LaneId<N, BLOCK, 0, G>& id,
                                               R (&are)[1], R (&aim)[1]) {
    if constexpr (G > 1) {
        using S = TreeShape<N, BLOCK, 0, G>;
        R* x = tb.XCH + (size_t)threadIdx.x * 2;
        x[0] = are[0];
        x[1] = aim[0];
        group_sync<BAR, BLOCK>();
        if (id.g == 0) {
#pragma unroll 1
            for (int gg = 1; gg < G; ++gg) {
                const R* y = tb.XCH + (size_t)(threadIdx.x + gg * S::GL) * 2;
                are[0] += y[0];
                aim[0] += y[1];
            }
        } else {
            are[0] = aim[0] = R(0);
        }
    }
}

// Sum (MAX = false) or maximum (MAX = true) of v over the point lanes of
// group 0 (the other groups hold zeros); the result is valid in the point's
// first lane of group 0.  All threads must call it.
template <class R, int N, int BLOCK, int BAR, int G, bool MAX>
__device__ __forceinline__ R point_reduce(const RoundTables<R, N, BLOCK, 0, G>& tb, R v) {
    using S = TreeShape<N, BLOCK, 0, G>;
    constexpr int W = S::NSL < 32 ? S::NSL : 32;
#pragma unroll
    for (int off = 1; off < W; off <<= 1) {
        const R o = __shfl_xor_sync(0xffffffffu, v, off);
        v = MAX ? fmax(v, o) : v + o;
    }
    if constexpr (S::NSL > 32) {
        const int tid = threadIdx.x;
        if ((tid & 31) == 0) tb.RED[tid >> 5] = v;
        group_sync<BAR, BLOCK>();
        if (tid < S::GL && tid % S::NSL == 0)
            for (int w = 1; w < S::NSL / 32; ++w) {
                const R o = tb.RED[(tid >> 5) + w];
                v = MAX ? fmax(v, o) : v + o;
            }
    }
    return v;
}

// Amplitude rounds over recs[0 .. cnt-1], one configuration per lane.  For
// each point the lanes' reduction yields S = sum_h w_h |A_h|^2 (scaled
// units), stored by the point's first lane in recs[p].ssum; the FP64
// normalisation and the accumulation are left to whole warps afterwards (one
// lane per point), so no FP64 instruction here runs with one or two active
// lanes.  mask: helicity mask (NULL = all).
template <class R, int N, int BLOCK, int BAR, int G>
__device__ __forceinline__ void amplitude_rounds_lanes(unsigned char* table_smem, PointRec<R, N>* recs, int cnt,
                                                       const uint32_t* mask) {
    using RT = RoundTables<R, N, BLOCK, 0, G>;
    using S = TreeShape<N, BLOCK, 0, G>;
    constexpr int P = S::P;
    const RT tb(table_smem);
    const LaneId<N, BLOCK, 0, G> id(threadIdx.x);
    const LaneTables<R, N, BLOCK, 0, G> L = lane_tables(tb, id.slot, (unsigned)id.hl);
    const float wh = lane_weight<N>(mask, (unsigned)id.hl);
    for (int base = 0; base < cnt; base += P) {
        const int rc = min(P, cnt - base);
        setup_round<R, N, BLOCK, BAR, 0, G>(tb, recs + base, rc);
        R are[1], aim[1];
        const bool active = id.slot < rc && recs[base + id.slot].valid;
        if (active) {
            tree_amplitude<R, N, BLOCK, G>(L, id.g, are, aim);
        } else {
            are[0] = aim[0] = R(0);
        }
        combine_groups<R, N, BLOCK, BAR, G>(tb, id, are, aim);
        // a sampled helicity (PointRec::hsel): only the selected lane counts
        const int hsel = active ? recs[base + id.slot].hsel : -1;
        const R v = (are[0] * are[0] + aim[0] * aim[0]) * R(sel_weight<N>(hsel, (unsigned)id.hl, wh));
        const R s = point_reduce<R, N, BLOCK, BAR, G, false>(tb, v);
        if (id.g == 0 && id.hl == 0 && id.slot < rc) recs[base + id.slot].ssum = s;
        group_sync<BAR, BLOCK>();
    }
}

// Amplitude rounds with pair units (four configurations per lane): the same
// contract as amplitude_rounds_lanes.  Each slot's lanes walk their units,
// adding each unit's amplitudes into the slot's accumulators at the absolute
// helicities of their rows; then one warp per point adds the slots in order,
// squares, weights and sums over the helicities in a fixed order.
template <class R, int N, int BLOCK, int BAR, int G>
__device__ __forceinline__ void amplitude_rounds_pairs(unsigned char* table_smem, PointRec<R, N>* recs, int cnt,
                                                       const uint32_t* mask) {
    using RT = RoundTables<R, N, BLOCK, 2, G>;
    using S = TreeShape<N, BLOCK, 2, G>;
    constexpr int P = S::P, NS = 1 << N;
    static_assert(BLOCK / 32 >= P, "one warp per point for the helicity sum");
    const RT tb(table_smem);
    const LaneId<N, BLOCK, 2, G> id(threadIdx.x);
    const int tid = threadIdx.x;
    for (int base = 0; base < cnt; base += P) {
        const int rc = min(P, cnt - base);
        for (int i = tid; i < G * P * NS * 2; i += BLOCK) tb.XCH[i] = R(0);
        setup_round<R, N, BLOCK, BAR, 2, G>(tb, recs + base, rc);   // its first barrier also orders the zeros
        if (id.slot < rc && recs[base + id.slot].valid) {
            R* acc = tb.XCH + ((size_t)id.g * P + id.slot) * NS * 2;
#pragma unroll 1
            for (int u = id.g; u < S::NPRE; u += G) {
                int p, q;
                pair_of_unit<N>(u, p, q);
                const unsigned hfull = spread_pair_bits((unsigned)id.hl, p, q);
                const LaneTables<R, N, BLOCK, 2, G> L = lane_tables(tb, id.slot, hfull);
                R are[4], aim[4];
#pragma unroll
                for (int b = 0; b < 4; ++b) are[b] = aim[b] = R(0);
                pair_unit<R, N, BLOCK, G>(L, p, q, are, aim);
                // units of one slot cover disjoint orderings; its lanes' rows
                // are distinct helicities: no two lanes touch one entry
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const unsigned h = hfull | ((unsigned)(b & 1) << p) | ((unsigned)(b >> 1) << q);
                    acc[2 * h] += are[b];
                    acc[2 * h + 1] += aim[b];
                }
            }
        }
        group_sync<BAR, BLOCK>();
        // one warp per point: slots added in order, |A_h|^2 w_h summed over h
        const int w = tid >> 5, lane = tid & 31;
        if (w < rc) {
            const int hsel = recs[base + w].valid ? recs[base + w].hsel : -1;
            R v = R(0);
            for (int h = lane; h < NS; h += 32) {
                R ar = R(0), ai = R(0);
#pragma unroll 1
                for (int gg = 0; gg < G; ++gg) {
                    const R* a = tb.XCH + (((size_t)gg * P + w) * NS + h) * 2;
                    ar += a[0];
                    ai += a[1];
                }
                v += (ar * ar + ai * ai) * R(sel_weight<N>(hsel, (unsigned)h, lane_weight<N>(mask, (unsigned)h)));
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if (lane == 0) recs[base + w].ssum = v;
        }
        group_sync<BAR, BLOCK>();
    }
}

template <class R, int N, int BLOCK, int BAR = 0, int HB = 0, int G = 1>
__device__ __forceinline__ void amplitude_rounds(unsigned char* table_smem, PointRec<R, N>* recs, int cnt,
                                                 const uint32_t* mask) {
    if constexpr (HB == 2) amplitude_rounds_pairs<R, N, BLOCK, BAR, G>(table_smem, recs, cnt, mask);
    else amplitude_rounds_lanes<R, N, BLOCK, BAR, G>(table_smem, recs, cnt, mask);
}

// Gauge check rounds over recs[0 .. cnt-1]: for each point the largest
// |A_h|^2 over the 2^N photon-helicity configurations (s1 = +) of the
// ordinary tree and of the tree with photon `ward` replaced by k/k^0; stores
// sqrt(max |W_h|^2 / max |A_h|^2) in recs[p].ssum.  |M_h|^2 of the s1 = -
// configurations equal those of s1 = + by parity, so the maxima cover all
// helicities.
template <class R, int N, int BLOCK>
__device__ __forceinline__ void ward_rounds(unsigned char* table_smem, PointRec<R, N>* recs, int cnt, int ward) {
    using RT = RoundTables<R, N, BLOCK>;
    constexpr int P = RT::P;
    const RT tb(table_smem);
    const LaneId<N, BLOCK, 0, 1> id(threadIdx.x);
    const LaneTables<R, N, BLOCK> L = lane_tables(tb, id.slot, (unsigned)id.hl);
    for (int base = 0; base < cnt; base += P) {
        const int rc = min(P, cnt - base);
        R best[2];
#pragma unroll 1
        for (int pass = 0; pass < 2; ++pass) {
            setup_round<R, N, BLOCK>(tb, recs + base, rc, pass ? ward : -1);
            R are[1] = {R(0)}, aim[1] = {R(0)};
            if (id.slot < rc && recs[base + id.slot].valid) tree_amplitude<R, N, BLOCK, 1>(L, 0, are, aim);
            best[pass] = point_reduce<R, N, BLOCK, 0, 1, true>(tb, are[0] * are[0] + aim[0] * aim[0]);
            __syncthreads();
        }
        if (id.hl == 0 && id.slot < rc) {
            const R a = best[0], w = best[1];
            recs[base + id.slot].ssum = a > R(0) ? sqrt(w / a) : (w > R(0) ? R(INFINITY) : R(0));
        }
        __syncthreads();
    }
}

}  // namespace heget
