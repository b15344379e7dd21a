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

// Lane layout of the tree (a compile-time shape):
//   * each lane carries H = 2^HB photon-helicity configurations ("rows"), which
//     differ in the helicities of the top HB photons NB..N-1 (NB = N - HB); one
//     lane's rows share every table load and all index arithmetic, so the
//     per-step overhead is spread over H row updates;
//   * the 2^NB lanes of one point are contiguous ("point lanes"); a group holds
//     the point lanes of all P points of a round, and G groups split the
//     ordered prefixes of depth D0 between them (prefix k goes to group k % G)
//     and add their partial amplitudes before squaring.  A group fills whole
//     warps, so that every warp walks one sequence of subtrees with
//     warp-uniform control flow and its table reads are broadcasts per point;
//   * thread t: group g = t / (P 2^NB), point slot (t / 2^NB) % P, helicity
//     bits hl = t % 2^NB.
// The walk below depth D0 keeps one row set per level in registers; D0 = 3 at
// n = 8 with four rows per lane (the top of the stack is recomputed per
// prefix instead of held, two extra steps per 85), else 2.
template <int N, int BLOCK, int HB, int G>
struct TreeShape {
    static constexpr int H = 1 << HB;
    static constexpr int NB = N - HB;
    static constexpr int NSL = 1 << NB;      // lanes of one point
    static constexpr int GL = BLOCK / G;     // lanes of a group
    static constexpr int P = GL / NSL;       // points per round
    static constexpr int D0 = (N == 8 && HB >= 2) ? 3 : N >= 3 ? 2 : 1;
    static constexpr int NPRE = D0 == 3 ? N * (N - 1) * (N - 2) : D0 == 2 ? N * (N - 1) : N;
    static_assert(HB >= 0 && HB <= 2 && (HB == 0 || NB >= 2), "1, 2 or 4 rows per lane");
    static_assert(BLOCK % G == 0 && GL % NSL == 0 && P >= 1, "a round holds whole points");
    static_assert(G == 1 || GL % 32 == 0, "subtree groups fill whole warps");
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

// Shared-memory tables of one round.  Every lane of a point reads one index
// for its point and one or two lambdas, so entries are laid out
// [index][point][lambda] (plus the two rows of a step matrix next to each
// other): the lanes of a warp hit a few consecutive 16-byte rows.
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
    static constexpr size_t x_elems = G > 1 ? (size_t)BLOCK * S::H * 2 : 0;
    static constexpr size_t p_elems = tree_two_ended<R, N>() ? (size_t)N * (N - 1) * P * 4 : 0;
    static constexpr size_t bytes = (m_elems + 2 * c_elems + p_elems) * sizeof(Row<R>)   // MT, CL, R1, PC
                                  + (size_t)P * N * sizeof(Row<R>)                      // photon data
                                  + (size_t)P * NS * sizeof(Row<R>)                     // set data
                                  + x_elems * sizeof(R)                                 // group exchange
                                  + (size_t)(BLOCK / 32) * sizeof(R) + 16;              // reduction
    Row<R>* MT;   // step matrices M(j, T)^lambda
    Row<R>* CL;   // closures (eps*_j . sigma) u_R
    Row<R>* R1;   // first rows vbar(p2) . M(j, {j})
    Row<R>* PC;   // [pair_slot(a, b)][P][lambda_a 2 + lambda_b]: pair columns (two-ended finish)
    Row<R>* PH;   // [P][N]: (sin th, cos th, cos ph, sin ph)
    Row<R>* SD;   // [P][2^N]: (A, D, Bre, Bim) = ((q0+q3), (q0-q3), q1, q2) / q^2
    R* XCH;       // [BLOCK][H][2]: partial amplitudes of the subtree groups
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

// Photon data PH[p][j] = (sin th, cos th, cos ph, sin ph) and set data
// SD[p][T] = (q0+q3, q0-q3, q1, q2) / t_T, q_T = sum_{i in T} k_i - p2, for
// the points recs[0 .. cnt-1] (P slots).  Everything runs in R: the FP64
// content (denominators) is already in the records.
template <class R, int N, int BLOCK, int P>
__device__ __forceinline__ void setup_photons_and_sets(Row<R>* PH, Row<R>* SD, const PointRec<R, N>* recs, int cnt) {
    constexpr int NS = 1 << N;
    const int tid = threadIdx.x;
    constexpr int n_ph = P * N, n_sd = P * NS;
    for (int it = tid; it < n_ph + n_sd; it += BLOCK) {
        if (it < n_ph) {
            const int p = it / N, j = it - p * N;
            if (p >= cnt) continue;
            const R* k = recs[p].k[j];
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
            PH[p * N + j] = d;
        } else {
            const int r = it - n_ph;
            const int p = r / NS, T = r - p * NS;
            if (p >= cnt || T == 0 || T == NS - 1) continue;
            const PointRec<R, N>& rc = recs[p];
            R q0 = -rc.e2, q1 = R(0), q2 = R(0), q3 = rc.e2;
#pragma unroll
            for (int i = 0; i < N; ++i)
                if (T >> i & 1) {
                    q0 += rc.k[i][0];
                    q1 += rc.k[i][1];
                    q2 += rc.k[i][2];
                    q3 += rc.k[i][3];
                }
            const R it_ = recip<R>(rc.t[T]);   // t_T from FP64, rounded once
            Row<R> d;
            d.ar = (q0 + q3) * it_;
            d.ai = (q0 - q3) * it_;
            d.br = q1 * it_;
            d.bi = q2 * it_;
            SD[p * NS + T] = d;
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
    unsigned hl;  // helicity bits of photons 0 .. NB-1 (lambda = bit set -> +1)
};

template <class R, int N, int BLOCK, int HB, int G>
__device__ __forceinline__ LaneTables<R, N, BLOCK, HB, G> lane_tables(const RoundTables<R, N, BLOCK, HB, G>& tb,
                                                                      int slot, int hl) {
    return LaneTables<R, N, BLOCK, HB, G>{tb.MT + 4 * slot, tb.CL + 2 * slot, tb.R1 + 2 * slot, tb.PC + 4 * slot,
                                          (unsigned)hl};
}

// Rows r[b] . M, photon j below NB: every row of the lane has the same lambda.
template <class R, int H>
__device__ __forceinline__ void step_same(Row<R> (&o)[H], const Row<R> (&r)[H], const Row<R>& m0, const Row<R>& m1) {
#pragma unroll
    for (int b = 0; b < H; ++b) o[b] = row_times(r[b], m0, m1);
}

// Rows r[b] . M^{lambda_b}, photon NB + JB: row b takes lambda = bit JB of b.
template <class R, int H, int JB>
__device__ __forceinline__ void step_split(Row<R> (&o)[H], const Row<R> (&r)[H], const Row<R>& a0, const Row<R>& a1,
                                           const Row<R>& b0, const Row<R>& b1) {
#pragma unroll
    for (int b = 0; b < H; ++b) o[b] = ((b >> JB) & 1) ? row_times(r[b], b0, b1) : row_times(r[b], a0, a1);
}

// Attach photon j to the rows (table entry index idx).
template <class R, int N, int BLOCK, int HB, int G>
__device__ __forceinline__ void attach(const LaneTables<R, N, BLOCK, HB, G>& L, int j, int idx,
                                       const Row<R> (&r)[1 << HB], Row<R> (&o)[1 << HB]) {
    using S = TreeShape<N, BLOCK, HB, G>;
    constexpr int H = S::H, NB = S::NB, P = S::P;
    const Row<R>* e = L.mt + idx * (4 * P);
    if (HB == 0 || j < NB) {
        e += ((L.hl >> j) & 1) * 2;
        step_same<R, H>(o, r, ld_row(e), ld_row(e + 1));
    } else {
        const Row<R> a0 = ld_row(e), a1 = ld_row(e + 1), b0 = ld_row(e + 2), b1 = ld_row(e + 3);
        if constexpr (HB == 1) {
            step_split<R, H, 0>(o, r, a0, a1, b0, b1);
        } else if constexpr (HB == 2) {
            if (j == NB) step_split<R, H, 0>(o, r, a0, a1, b0, b1);
            else step_split<R, H, 1>(o, r, a0, a1, b0, b1);
        }
    }
}

// Closure with the last photon j (iovxx0 against u(p1)).
template <class R, int N, int BLOCK, int HB, int G>
__device__ __forceinline__ void close_rows(const LaneTables<R, N, BLOCK, HB, G>& L, int j, const Row<R> (&r)[1 << HB],
                                           R (&are)[1 << HB], R (&aim)[1 << HB]) {
    using S = TreeShape<N, BLOCK, HB, G>;
    constexpr int H = S::H, NB = S::NB, P = S::P;
    const Row<R>* c = L.cl + j * (2 * P);
    if (HB == 0 || j < NB) {
        const Row<R> c0 = ld_row(c + ((L.hl >> j) & 1));
#pragma unroll
        for (int b = 0; b < H; ++b) close_row(r[b], c0, are[b], aim[b]);
    } else {
        const Row<R> c0 = ld_row(c), c1 = ld_row(c + 1);
        if (HB == 1 || j == NB) {
#pragma unroll
            for (int b = 0; b < H; ++b) close_row(r[b], (b & 1) ? c1 : c0, are[b], aim[b]);
        } else {
#pragma unroll
            for (int b = 0; b < H; ++b) close_row(r[b], ((b >> 1) & 1) ? c1 : c0, are[b], aim[b]);
        }
    }
}

// Pair closures of the rows when photon b (a < b) is the top photon NB + KB
// and a is below NB: row takes lambda_b = bit KB of its index.
template <class R, int H, int KB>
__device__ __forceinline__ void close_pair_split(const Row<R> (&r)[H], const Row<R>& ab0, const Row<R>& ab1,
                                                 const Row<R>& ba0, const Row<R>& ba1, R (&are)[H], R (&aim)[H]) {
#pragma unroll
    for (int row = 0; row < H; ++row) {
        const bool lb = (row >> KB) & 1;
        close_row(r[row], lb ? ab1 : ab0, are[row], aim[row]);
        close_row(r[row], lb ? ba1 : ba0, are[row], aim[row]);
    }
}

// The two orderings left below a node of depth n - 2 by the pair columns:
// acc += r . PC(a -> b) + r . PC(b -> a), a < b, each row with its own
// lambdas.  Which of a, b are top photons is warp-uniform; each case loads
// only the entries its rows use.
template <class R, int N, int BLOCK, int HB, int G>
__device__ __forceinline__ void close_pair(const LaneTables<R, N, BLOCK, HB, G>& L, int a, int b,
                                           const Row<R> (&r)[1 << HB], R (&are)[1 << HB], R (&aim)[1 << HB]) {
    using S = TreeShape<N, BLOCK, HB, G>;
    constexpr int H = S::H, NB = S::NB, P = S::P;
    const Row<R>* ab = L.pc + pair_slot<N>(a, b) * (4 * P);
    const Row<R>* ba = L.pc + pair_slot<N>(b, a) * (4 * P);
    if (HB == 0 || b < NB) {
        const int la = (L.hl >> a) & 1, lb = (L.hl >> b) & 1;
        const Row<R> c1 = ld_row(ab + la * 2 + lb), c2 = ld_row(ba + lb * 2 + la);
#pragma unroll
        for (int row = 0; row < H; ++row) {
            close_row(r[row], c1, are[row], aim[row]);
            close_row(r[row], c2, are[row], aim[row]);
        }
    } else if (a < NB) {
        const int la = (L.hl >> a) & 1;
        const Row<R> ab0 = ld_row(ab + la * 2), ab1 = ld_row(ab + la * 2 + 1);
        const Row<R> ba0 = ld_row(ba + la), ba1 = ld_row(ba + 2 + la);
        if constexpr (HB == 1) {
            close_pair_split<R, H, 0>(r, ab0, ab1, ba0, ba1, are, aim);
        } else if constexpr (HB == 2) {
            if (b == NB) close_pair_split<R, H, 0>(r, ab0, ab1, ba0, ba1, are, aim);
            else close_pair_split<R, H, 1>(r, ab0, ab1, ba0, ba1, are, aim);
        }
    } else if constexpr (HB == 2) {
        // a = NB, b = NB + 1: lambda_a = row bit 0, lambda_b = row bit 1
        Row<R> cab[4], cba[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            cab[e] = ld_row(ab + e);
            cba[e] = ld_row(ba + e);
        }
#pragma unroll
        for (int row = 0; row < H; ++row) {
            const int la = row & 1, lb = row >> 1;
            close_row(r[row], cab[la * 2 + lb], are[row], aim[row]);
            close_row(r[row], cba[lb * 2 + la], are[row], aim[row]);
        }
    }
}

// First rows vbar(p2) . M(j, {j}) for the lane's helicities.
template <class R, int N, int BLOCK, int HB, int G>
__device__ __forceinline__ void first_rows(const LaneTables<R, N, BLOCK, HB, G>& L, int j, Row<R> (&r)[1 << HB]) {
    using S = TreeShape<N, BLOCK, HB, G>;
    constexpr int H = S::H, NB = S::NB, P = S::P;
    const Row<R>* e = L.r1 + j * (2 * P);
    if (HB == 0 || j < NB) {
        const Row<R> a = ld_row(e + ((L.hl >> j) & 1));
#pragma unroll
        for (int b = 0; b < H; ++b) r[b] = a;
    } else {
        const Row<R> a0 = ld_row(e), a1 = ld_row(e + 1);
        if (HB == 1 || j == NB) {
#pragma unroll
            for (int b = 0; b < H; ++b) r[b] = (b & 1) ? a1 : a0;
        } else {
#pragma unroll
            for (int b = 0; b < H; ++b) r[b] = ((b >> 1) & 1) ? a1 : a0;
        }
    }
}

__device__ __forceinline__ int tree_child(int n, unsigned T, int j) {
    return c_tables.child[child_offset(n) + T * n + j];
}

// The bottom three levels of the walk, written out from the per-set index
// entry (Bottom3): below a node with rows r and three photons a < b < c
// left, attach each of them and close the two orderings of the other two by
// the pair columns.  KA, KB, KC: -1 for a photon below NB (its lambda is the
// lane's bit), else the row bit that carries its lambda; fixed per case, so
// every load and row selection is resolved at compile time.
template <class R, int N, int BLOCK, int HB, int G, int K>
__device__ __forceinline__ void bottom_step(const LaneTables<R, N, BLOCK, HB, G>& L, int st, int lam,
                                            const Row<R> (&r)[1 << HB], Row<R> (&o)[1 << HB]) {
    constexpr int P = TreeShape<N, BLOCK, HB, G>::P, H = 1 << HB;
    const Row<R>* e = L.mt + st * (4 * P);
    if constexpr (K < 0) {
        e += lam * 2;
        step_same<R, H>(o, r, ld_row(e), ld_row(e + 1));
    } else {
        step_split<R, H, K>(o, r, ld_row(e), ld_row(e + 1), ld_row(e + 2), ld_row(e + 3));
    }
}

template <class R, int N, int BLOCK, int HB, int G, int K1, int K2>
__device__ __forceinline__ void bottom_pair(const LaneTables<R, N, BLOCK, HB, G>& L, int s12, int s21, int l1, int l2,
                                            const Row<R> (&r)[1 << HB], R (&are)[1 << HB], R (&aim)[1 << HB]) {
    constexpr int P = TreeShape<N, BLOCK, HB, G>::P, H = 1 << HB;
    // PC(y -> z)[ly][lz] and PC(z -> y)[lz][ly]
    const Row<R>* ab = L.pc + s12 * (4 * P);
    const Row<R>* ba = L.pc + s21 * (4 * P);
    Row<R> c1[4], c2[4];   // entries by row-dependent lambdas (index 2 ly' + lz')
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const int vy = v >> 1, vz = v & 1;
        if ((K1 < 0 && vy) || (K2 < 0 && vz)) continue;   // only the entries the rows use
        const int ly = K1 < 0 ? l1 : vy, lz = K2 < 0 ? l2 : vz;
        c1[v] = ld_row(ab + ly * 2 + lz);
        c2[v] = ld_row(ba + lz * 2 + ly);
    }
#pragma unroll
    for (int row = 0; row < H; ++row) {
        const int vy = K1 < 0 ? 0 : (row >> (K1 < 0 ? 0 : K1)) & 1;
        const int vz = K2 < 0 ? 0 : (row >> (K2 < 0 ? 0 : K2)) & 1;
        close_row(r[row], c1[vy * 2 + vz], are[row], aim[row]);
        close_row(r[row], c2[vy * 2 + vz], are[row], aim[row]);
    }
}

template <class R, int N, int BLOCK, int HB, int G, int KA, int KB, int KC>
__device__ __forceinline__ void bottom3_case(const LaneTables<R, N, BLOCK, HB, G>& L, const Bottom3& e, int a, int b,
                                             int c, const Row<R> (&r)[1 << HB], R (&are)[1 << HB],
                                             R (&aim)[1 << HB]) {
    constexpr int H = 1 << HB;
    const int la = KA < 0 ? (int)((L.hl >> a) & 1) : 0;
    const int lb = KB < 0 ? (int)((L.hl >> b) & 1) : 0;
    const int lc = KC < 0 ? (int)((L.hl >> c) & 1) : 0;
    Row<R> r2[H];
    bottom_step<R, N, BLOCK, HB, G, KA>(L, e.st[0], la, r, r2);
    bottom_pair<R, N, BLOCK, HB, G, KB, KC>(L, e.pc[0], e.pc[1], lb, lc, r2, are, aim);
    bottom_step<R, N, BLOCK, HB, G, KB>(L, e.st[1], lb, r, r2);
    bottom_pair<R, N, BLOCK, HB, G, KA, KC>(L, e.pc[2], e.pc[3], la, lc, r2, are, aim);
    bottom_step<R, N, BLOCK, HB, G, KC>(L, e.st[2], lc, r, r2);
    bottom_pair<R, N, BLOCK, HB, G, KA, KB>(L, e.pc[4], e.pc[5], la, lb, r2, are, aim);
}

template <class R, int N, int BLOCK, int HB, int G>
__device__ __forceinline__ void bottom3(const LaneTables<R, N, BLOCK, HB, G>& L, const Row<R> (&r)[1 << HB],
                                        unsigned T, R (&are)[1 << HB], R (&aim)[1 << HB]) {
    constexpr int NB = N - HB;
    constexpr unsigned FULL = (1u << N) - 1;
    const unsigned rem = FULL & ~T, rem2 = rem & (rem - 1);
    const int a = __ffs(rem) - 1, b = __ffs(rem2) - 1, c = __ffs(rem2 & (rem2 - 1)) - 1;
    const Bottom3& e = c_bottom.e[bottom_offset(N) + T];
    // the top photons are the highest: c is one before b is, a never is
    if (HB == 0 || c < NB) {
        bottom3_case<R, N, BLOCK, HB, G, -1, -1, -1>(L, e, a, b, c, r, are, aim);
    } else if constexpr (HB == 1) {
        bottom3_case<R, N, BLOCK, HB, G, -1, -1, 0>(L, e, a, b, c, r, are, aim);
    } else if constexpr (HB == 2) {
        if (b >= NB) bottom3_case<R, N, BLOCK, HB, G, -1, 0, 1>(L, e, a, b, c, r, are, aim);
        else if (c == NB) bottom3_case<R, N, BLOCK, HB, G, -1, -1, 0>(L, e, a, b, c, r, are, aim);
        else bottom3_case<R, N, BLOCK, HB, G, -1, -1, 1>(L, e, a, b, c, r, are, aim);
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

// The orderings of group g for one lane: the subtrees below the ordered
// prefixes k = g, g + G, ... of depth D0 (lexicographic), each prefix's rows
// formed from the first rows by D0 - 1 steps.  Sums, per row, the helicity
// amplitude (up to normalisation) for s1 = +.  g is the same for every lane of
// a warp, so every loop bound and table index below is warp-uniform.
template <class R, int N, int BLOCK, int HB, int G>
__device__ __forceinline__ void tree_amplitude(const LaneTables<R, N, BLOCK, HB, G>& L, int g, R (&are)[1 << HB],
                                               R (&aim)[1 << HB]) {
    using S = TreeShape<N, BLOCK, HB, G>;
    constexpr int H = S::H;
#pragma unroll
    for (int b = 0; b < H; ++b) are[b] = aim[b] = R(0);
#pragma unroll 1
    for (int k = g; k < S::NPRE; k += G) {
        if constexpr (S::D0 == 1) {
            Row<R> r1[H];
            first_rows<R, N, BLOCK, HB, G>(L, k, r1);
            descend<R, N, 1, BLOCK, HB, G>(L, r1, 1u << k, are, aim);
        } else if constexpr (S::D0 == 2) {
            int j1, j2, j3;
            tree_prefix<N, 2>(k, j1, j2, j3);
            Row<R> r1[H], r2[H];
            first_rows<R, N, BLOCK, HB, G>(L, j1, r1);
            attach<R, N, BLOCK, HB, G>(L, j2, tree_child(N, 1u << j1, j2), r1, r2);
            descend<R, N, 2, BLOCK, HB, G>(L, r2, (1u << j1) | (1u << j2), are, aim);
        } else {
            int j1, j2, j3;
            tree_prefix<N, 3>(k, j1, j2, j3);
            Row<R> r1[H], r2[H], r3[H];
            first_rows<R, N, BLOCK, HB, G>(L, j1, r1);
            const unsigned T2 = (1u << j1) | (1u << j2);
            attach<R, N, BLOCK, HB, G>(L, j2, tree_child(N, 1u << j1, j2), r1, r2);
            attach<R, N, BLOCK, HB, G>(L, j3, tree_child(N, T2, j3), r2, r3);
            descend<R, N, 3, BLOCK, HB, G>(L, r3, T2 | (1u << j3), are, aim);
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


// Lane coordinates in a round: subtree group, point slot, helicity bits.
template <int N, int BLOCK, int HB, int G>
struct LaneId {
    using S = TreeShape<N, BLOCK, HB, G>;
    int g, slot, hl;
    __device__ __forceinline__ explicit LaneId(int tid)
        : g(tid / S::GL), slot((tid % S::GL) / S::NSL), hl(tid % S::NSL) {}
};

// The complete amplitudes of the lane's rows: with several subtree groups,
// every group leaves its partial sums in shared memory and group 0 adds them
// in group order (the other groups' amplitudes become 0).  All threads must
// call it.
template <class R, int N, int BLOCK, int BAR, int HB, int G>
__device__ __forceinline__ void combine_groups(const RoundTables<R, N, BLOCK, HB, G>& tb, const LaneId<N, BLOCK, HB, G>& id,
                                               R (&are)[1 << HB], R (&aim)[1 << HB]) {
    if constexpr (G > 1) {
        using S = TreeShape<N, BLOCK, HB, G>;
        constexpr int H = S::H;
        R* x = tb.XCH + (size_t)threadIdx.x * H * 2;
#pragma unroll
        for (int b = 0; b < H; ++b) {
            x[2 * b] = are[b];
            x[2 * b + 1] = aim[b];
        }
        group_sync<BAR, BLOCK>();
        if (id.g == 0) {
#pragma unroll 1
            for (int gg = 1; gg < G; ++gg) {
                const R* y = tb.XCH + (size_t)(threadIdx.x + gg * S::GL) * H * 2;
#pragma unroll
                for (int b = 0; b < H; ++b) {
                    are[b] += y[2 * b];
                    aim[b] += y[2 * b + 1];
                }
            }
        } else {
#pragma unroll
            for (int b = 0; b < H; ++b) are[b] = aim[b] = R(0);
        }
    }
}

// Sum (MAX = false) or maximum (MAX = true) of v over the point lanes of
// group 0 (the other groups hold zeros); the result is valid in the point's
// first lane of group 0.  All threads must call it.
template <class R, int N, int BLOCK, int BAR, int HB, int G, bool MAX>
__device__ __forceinline__ R point_reduce(const RoundTables<R, N, BLOCK, HB, G>& tb, R v) {
    using S = TreeShape<N, BLOCK, HB, G>;
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

// Amplitude rounds over recs[0 .. cnt-1].  For each point the lanes' reduction
// yields S = sum_h w_h |A_h|^2 (scaled units), stored by the point's first
// lane in recs[p].ssum; the FP64 normalisation and the accumulation are left
// to whole warps afterwards (one lane per point), so no FP64 instruction here
// runs with one or two active lanes.  mask: helicity mask (NULL = all).
template <class R, int N, int BLOCK, int BAR = 0, int HB = 0, int G = 1>
__device__ __forceinline__ void amplitude_rounds(unsigned char* table_smem, PointRec<R, N>* recs, int cnt,
                                                 const uint32_t* mask) {
    using RT = RoundTables<R, N, BLOCK, HB, G>;
    using S = TreeShape<N, BLOCK, HB, G>;
    constexpr int P = S::P, H = S::H;
    const RT tb(table_smem);
    const LaneId<N, BLOCK, HB, G> id(threadIdx.x);
    const LaneTables<R, N, BLOCK, HB, G> L = lane_tables(tb, id.slot, id.hl);
    float wh[H];
#pragma unroll
    for (int b = 0; b < H; ++b) wh[b] = lane_weight<N>(mask, (unsigned)id.hl | ((unsigned)b << S::NB));
    for (int base = 0; base < cnt; base += P) {
        const int rc = min(P, cnt - base);
        setup_round<R, N, BLOCK, BAR, HB, G>(tb, recs + base, rc);
        R are[H], aim[H];
        const bool active = id.slot < rc && recs[base + id.slot].valid;
        if (active) {
            tree_amplitude<R, N, BLOCK, HB, G>(L, id.g, are, aim);
        } else {
#pragma unroll
            for (int b = 0; b < H; ++b) are[b] = aim[b] = R(0);
        }
        combine_groups<R, N, BLOCK, BAR, HB, G>(tb, id, are, aim);
        R v = R(0);
#pragma unroll
        for (int b = 0; b < H; ++b) v += (are[b] * are[b] + aim[b] * aim[b]) * R(wh[b]);
        // a sampled helicity (PointRec::hsel): only the selected lane counts
        const int hsel = active ? recs[base + id.slot].hsel : -1;
        if (hsel != -1) {
            v = R(0);
#pragma unroll
            for (int b = 0; b < H; ++b) {
                const unsigned lam = (unsigned)id.hl | ((unsigned)b << S::NB);
                v += (are[b] * are[b] + aim[b] * aim[b]) * R(sel_weight<N>(hsel, lam, wh[b]));
            }
        }
        v = point_reduce<R, N, BLOCK, BAR, HB, G, false>(tb, v);
        if (id.g == 0 && id.hl == 0 && id.slot < rc) recs[base + id.slot].ssum = v;
        group_sync<BAR, BLOCK>();
    }
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
    const LaneTables<R, N, BLOCK> L = lane_tables(tb, id.slot, id.hl);
    for (int base = 0; base < cnt; base += P) {
        const int rc = min(P, cnt - base);
        R best[2];
#pragma unroll 1
        for (int pass = 0; pass < 2; ++pass) {
            setup_round<R, N, BLOCK>(tb, recs + base, rc, pass ? ward : -1);
            R are[1] = {R(0)}, aim[1] = {R(0)};
            if (id.slot < rc && recs[base + id.slot].valid) tree_amplitude<R, N, BLOCK, 0, 1>(L, 0, are, aim);
            best[pass] = point_reduce<R, N, BLOCK, 0, 0, 1, true>(tb, are[0] * are[0] + aim[0] * aim[0]);
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
