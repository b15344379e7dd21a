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
// Lanes: one lane per photon-helicity configuration h in [0, 2^n) with
// s1 = +; every lane of a point walks the same tree (uniform control flow),
// reading the same table entries up to the lambda_j bit (broadcast loads).
// The s1 = - configurations follow from parity, |M_{-h}|^2 = |M_h|^2
// (checked against the oracle), folded into a per-lane weight
// w_h = [mask(+,-,h)] + [mask(-,+,~h)].
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

// Lane layout of the tree (a compile-time shape):
//   * each lane carries H = 2^HB photon-helicity configurations ("rows"), which
//     differ in the helicities of the top HB photons NB..N-1 (NB = N - HB); one
//     lane's rows share every table load and all index arithmetic, so the
//     per-step overhead is spread over H row updates;
//   * a point's 2^NB lanes form a group; G groups per point split the n(n-1)
//     depth-2 prefixes between them (a group must fill whole warps, so that a
//     warp walks one subtree and its table reads stay broadcasts) and add their
//     partial amplitudes before squaring;
//   * P = BLOCK / (2^NB G) points share one round of tables.
// (HB, G) = (0, 1) is one helicity configuration per lane, one group.
template <int N, int BLOCK, int HB, int G>
struct TreeShape {
    static constexpr int H = 1 << HB;
    static constexpr int NB = N - HB;
    static constexpr int NSL = 1 << NB;      // lanes of a group
    static constexpr int LPP = NSL * G;      // lanes of a point
    static constexpr int P = BLOCK / LPP;    // points per round
    static_assert(HB >= 0 && HB <= 2 && HB < N, "1, 2 or 4 rows per lane");
    static_assert(P >= 1 && BLOCK % LPP == 0, "a round holds whole points");
    static_assert(G == 1 || (NSL >= 32 && N >= 3), "subtree groups fill whole warps");
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

// Shared-memory tables of one round.
// Entry layout [index][point][lambda] so that the lanes of a warp, which read
// one index for one or a few points and both lambdas, hit distinct banks.
template <class R, int N, int BLOCK, int HB = 0, int G = 1>
struct RoundTables {
    using S = TreeShape<N, BLOCK, HB, G>;
    static constexpr int P = S::P;
    static constexpr int K = num_pairs(N);
    // step matrices held: with the two-ended finish, those of sets of at
    // most n - 2 photons (the pair index lists them first)
    static constexpr int KW = tree_two_ended<R, N>() ? K - N * (N - 1) : K;
    static constexpr int NS = 1 << N;
    static constexpr size_t m_elems = (size_t)KW * P * 2;
    static constexpr size_t c_elems = (size_t)N * P * 2;
    static constexpr size_t x_elems = G > 1 ? (size_t)BLOCK * S::H * 2 : 0;
    static constexpr size_t p_elems = tree_two_ended<R, N>() ? (size_t)N * (N - 1) * P * 4 : 0;
    static constexpr size_t bytes = (2 * m_elems + 2 * c_elems + p_elems) * sizeof(Row<R>)   // M0, M1, CL, R1, PC
                                  + (size_t)P * N * sizeof(Row<R>)                 // photon data
                                  + (size_t)P * NS * sizeof(Row<R>)                // set data
                                  + x_elems * sizeof(R)                            // group exchange
                                  + (size_t)(BLOCK / 32) * sizeof(R) + 16;         // reduction
    Row<R>* M0;
    Row<R>* M1;
    Row<R>* CL;
    Row<R>* R1;
    Row<R>* PH;   // [P][N]: (sin th, cos th, cos ph, sin ph)
    Row<R>* SD;   // [P][2^N]: (A, D, Bre, Bim) = ((q0+q3), (q0-q3), q1, q2) / q^2
    Row<R>* PC;   // [pair_slot(a, b)][P][lambda_a 2 + lambda_b]: pair columns (two-ended finish)
    R* XCH;       // [BLOCK][H][2]: partial amplitudes of the subtree groups
    R* RED;       // [BLOCK/32]
    __device__ __forceinline__ explicit RoundTables(unsigned char* base) {
        M0 = reinterpret_cast<Row<R>*>(base);
        M1 = M0 + m_elems;
        CL = M1 + m_elems;
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

// acc[b] += r[b] . c, c = (ca, cb) a column 2-spinor
template <class R>
__device__ __forceinline__ void close_row(const Row<R>& r, const Row<R>& c, R& are, R& aim) {
    are += r.ar * c.ar - r.ai * c.ai + r.br * c.br - r.bi * c.bi;
    aim += r.ar * c.ai + r.ai * c.ar + r.br * c.bi + r.bi * c.br;
}

// Fill the round tables for points recs[0 .. cnt-1] (cnt <= P).  Two phases
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
        const Row<R>& m0 = sm.m0;
        const Row<R>& m1 = sm.m1;
        const R e00 = sm.e00, e10r = sm.e10r, e10i = sm.e10i;
        const size_t o = ((size_t)idx * P + p) * 2 + lam_bit;
        st_row(tb.M0 + o, m0);
        st_row(tb.M1 + o, m1);
        if (T == (1 << j)) {
            const size_t oc = ((size_t)j * P + p) * 2 + lam_bit;
            const R n1 = recs[p].n1;
            const R n2 = recs[p].n2;
            st_row(tb.CL + oc, Row<R>{n1 * e00, R(0), n1 * e10r, n1 * e10i});
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

// Per-lane view of the round tables.
template <class R, int N, int BLOCK, int HB = 0, int G = 1>
struct LaneTables {
    using S = TreeShape<N, BLOCK, HB, G>;
    const Row<R>* M0;
    const Row<R>* M1;
    const Row<R>* CL;
    const Row<R>* R1;
    int pp;       // 2 * point slot
    unsigned hl;  // helicity bits of photons 0 .. NB-1 (lambda = bit set -> +1)
    const Row<R>* PC;   // pair columns (two-ended finish), else NULL
};

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
    const int base = idx * P * 2 + L.pp;
    if (HB == 0 || j < NB) {
        const int e = base + ((L.hl >> j) & 1);
        step_same<R, H>(o, r, ld_row(L.M0 + e), ld_row(L.M1 + e));
    } else {
        const Row<R> a0 = ld_row(L.M0 + base), a1 = ld_row(L.M1 + base);
        const Row<R> b0 = ld_row(L.M0 + base + 1), b1 = ld_row(L.M1 + base + 1);
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
    const int base = j * P * 2 + L.pp;
    if (HB == 0 || j < NB) {
        const Row<R> c = ld_row(L.CL + base + ((L.hl >> j) & 1));
#pragma unroll
        for (int b = 0; b < H; ++b) close_row(r[b], c, are[b], aim[b]);
    } else {
        const Row<R> c0 = ld_row(L.CL + base), c1 = ld_row(L.CL + base + 1);
        if (HB == 1 || j == NB) {
#pragma unroll
            for (int b = 0; b < H; ++b) close_row(r[b], (b & 1) ? c1 : c0, are[b], aim[b]);
        } else {
#pragma unroll
            for (int b = 0; b < H; ++b) close_row(r[b], ((b >> 1) & 1) ? c1 : c0, are[b], aim[b]);
        }
    }
}

// The two orderings left below a node of depth n - 2 by the pair columns:
// acc += r . PC(a -> b) + r . PC(b -> a), each row with its own lambdas.
template <class R, int N, int BLOCK, int HB, int G>
__device__ __forceinline__ void close_pair(const LaneTables<R, N, BLOCK, HB, G>& L, int a, int b,
                                           const Row<R> (&r)[1 << HB], R (&are)[1 << HB], R (&aim)[1 << HB]) {
    using S = TreeShape<N, BLOCK, HB, G>;
    constexpr int H = S::H, NB = S::NB, P = S::P;
    const Row<R>* ab = L.PC + ((size_t)pair_slot<N>(a, b) * P) * 4 + 2 * L.pp;
    const Row<R>* ba = L.PC + ((size_t)pair_slot<N>(b, a) * P) * 4 + 2 * L.pp;
#pragma unroll
    for (int row = 0; row < H; ++row) {
        const int la = a < NB ? (int)((L.hl >> a) & 1) : (row >> (a - NB)) & 1;
        const int lb = b < NB ? (int)((L.hl >> b) & 1) : (row >> (b - NB)) & 1;
        close_row(r[row], ld_row(ab + la * 2 + lb), are[row], aim[row]);
        close_row(r[row], ld_row(ba + lb * 2 + la), are[row], aim[row]);
    }
}

// First rows vbar(p2) . M(j, {j}) for the lane's helicities.
template <class R, int N, int BLOCK, int HB, int G>
__device__ __forceinline__ void first_rows(const LaneTables<R, N, BLOCK, HB, G>& L, int j, Row<R> (&r)[1 << HB]) {
    using S = TreeShape<N, BLOCK, HB, G>;
    constexpr int H = S::H, NB = S::NB, P = S::P;
    const int base = j * P * 2 + L.pp;
    if (HB == 0 || j < NB) {
        const Row<R> a = ld_row(L.R1 + base + ((L.hl >> j) & 1));
#pragma unroll
        for (int b = 0; b < H; ++b) r[b] = a;
    } else {
        const Row<R> a0 = ld_row(L.R1 + base), a1 = ld_row(L.R1 + base + 1);
        if (HB == 1 || j == NB) {
#pragma unroll
            for (int b = 0; b < H; ++b) r[b] = (b & 1) ? a1 : a0;
        } else {
#pragma unroll
            for (int b = 0; b < H; ++b) r[b] = ((b >> 1) & 1) ? a1 : a0;
        }
    }
}

// Levels at the bottom of the tree written out without loops: 0, 1 (the
// last two photons as two chains) or 2 (also the loop over the last three),
// per precision and photon count.  FP32 values from a GB300 sweep (n = 5
// +26 %, n = 7 +19 %, n = 8 +23 % over none; n = 4, 6 best without); they
// can be overridden with -DHEGET_F32_UNROLL_<n>=..
#ifndef HEGET_F32_UNROLL_4
#define HEGET_F32_UNROLL_4 0
#endif
#ifndef HEGET_F32_UNROLL_5
#define HEGET_F32_UNROLL_5 2
#endif
#ifndef HEGET_F32_UNROLL_6
#define HEGET_F32_UNROLL_6 0
#endif
#ifndef HEGET_F32_UNROLL_7
#define HEGET_F32_UNROLL_7 1
#endif
#ifndef HEGET_F32_UNROLL_8
#define HEGET_F32_UNROLL_8 1
#endif
template <class R, int N>
__host__ __device__ constexpr int tree_unroll() {
    if (sizeof(R) != sizeof(float)) return 0;
    return N == 4 ? HEGET_F32_UNROLL_4 : N == 5 ? HEGET_F32_UNROLL_5 : N == 6 ? HEGET_F32_UNROLL_6
         : N == 7 ? HEGET_F32_UNROLL_7 : N == 8 ? HEGET_F32_UNROLL_8 : 0;
}

// Depth-first walk of the ordering tree below a node at depth D (D photons
// attached, set T, current rows r), adding the closures to acc.
template <class R, int N, int D, int BLOCK, int HB, int G>
__device__ __forceinline__ void descend(const LaneTables<R, N, BLOCK, HB, G>& L, const Row<R> (&r)[1 << HB],
                                        unsigned T, R (&are)[1 << HB], R (&aim)[1 << HB]) {
    constexpr unsigned FULL = (1u << N) - 1;
    if constexpr (D == N - 1) {
        close_rows<R, N, BLOCK, HB, G>(L, __ffs(FULL & ~T) - 1, r, are, aim);
    } else if constexpr (D == N - 2 && tree_two_ended<R, N>()) {
        const unsigned rem = FULL & ~T;
        close_pair<R, N, BLOCK, HB, G>(L, __ffs(rem) - 1, __ffs(rem & (rem - 1)) - 1, r, are, aim);
    } else if constexpr (D == N - 2 && tree_unroll<R, N>() >= 1) {
        // two photons a < b left: the orderings (a, b) and (b, a) as two
        // independent chains, accumulated in the loop's order
        const unsigned rem = FULL & ~T;
        const int a = __ffs(rem) - 1, b = __ffs(rem & (rem - 1)) - 1;
        Row<R> ra[1 << HB], rb[1 << HB];
        attach<R, N, BLOCK, HB, G>(L, a, c_tables.child[child_offset(N) + T * N + a], r, ra);
        attach<R, N, BLOCK, HB, G>(L, b, c_tables.child[child_offset(N) + T * N + b], r, rb);
        close_rows<R, N, BLOCK, HB, G>(L, b, ra, are, aim);
        close_rows<R, N, BLOCK, HB, G>(L, a, rb, are, aim);
    } else if constexpr (D == N - 3 && tree_unroll<R, N>() >= 2) {
        // three photons left: the loop over them unrolled
        unsigned rem = FULL & ~T;
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            const int j = __ffs(rem) - 1;
            rem &= rem - 1;
            Row<R> r2[1 << HB];
            attach<R, N, BLOCK, HB, G>(L, j, c_tables.child[child_offset(N) + T * N + j], r, r2);
            descend<R, N, D + 1, BLOCK, HB, G>(L, r2, T | (1u << j), are, aim);
        }
    } else {
        unsigned rem = FULL & ~T;
#pragma unroll 1
        while (rem) {
            const int j = __ffs(rem) - 1;
            rem &= rem - 1;
            const int idx = c_tables.child[child_offset(N) + T * N + j];
            Row<R> r2[1 << HB];
            attach<R, N, BLOCK, HB, G>(L, j, idx, r, r2);
            descend<R, N, D + 1, BLOCK, HB, G>(L, r2, T | (1u << j), are, aim);
        }
    }
}

// Subtrees below the depth-2 prefixes k = GI, GI + G, ... of the n(n-1)
// prefixes (j1, j2) in lexicographic order.  GI is a template argument so
// that every loop bound and table index below stays warp-uniform.
template <class R, int N, int BLOCK, int HB, int G, int GI>
__device__ __forceinline__ void tree_group(const LaneTables<R, N, BLOCK, HB, G>& L, R (&are)[1 << HB],
                                           R (&aim)[1 << HB]) {
    constexpr int H = 1 << HB;
#pragma unroll 1
    for (int k = GI; k < N * (N - 1); k += G) {
        const int j1 = k / (N - 1), t = k - j1 * (N - 1), j2 = t + (t >= j1);
        Row<R> r1[H], r2[H];
        first_rows<R, N, BLOCK, HB, G>(L, j1, r1);
        attach<R, N, BLOCK, HB, G>(L, j2, c_tables.child[child_offset(N) + (1u << j1) * N + j2], r1, r2);
        descend<R, N, 2, BLOCK, HB, G>(L, r2, (1u << j1) | (1u << j2), are, aim);
    }
}

// The orderings of group g for one lane: with one group all n! orderings,
// otherwise the group's share of the depth-2 subtrees (a group is a whole
// number of warps, so the switch below never diverges inside a warp).  Sums,
// per row, the helicity amplitude (up to normalisation) for s1 = +.
template <class R, int N, int BLOCK, int HB, int G>
__device__ __forceinline__ void tree_amplitude(const LaneTables<R, N, BLOCK, HB, G>& L, int g, R (&are)[1 << HB],
                                               R (&aim)[1 << HB]) {
    constexpr int H = 1 << HB;
#pragma unroll
    for (int b = 0; b < H; ++b) are[b] = aim[b] = R(0);
    if constexpr (G == 1) {
#pragma unroll 1
        for (int j = 0; j < N; ++j) {
            Row<R> r1[H];
            first_rows<R, N, BLOCK, HB, G>(L, j, r1);
            descend<R, N, 1, BLOCK, HB, G>(L, r1, 1u << j, are, aim);
        }
    } else {
        static_assert(G == 2 || G == 4, "2 or 4 subtree groups");
        switch (g) {
            case 0: tree_group<R, N, BLOCK, HB, G, 0>(L, are, aim); break;
            case 1: tree_group<R, N, BLOCK, HB, G, 1>(L, are, aim); break;
            case 2: if constexpr (G > 2) tree_group<R, N, BLOCK, HB, G, 2>(L, are, aim); break;
            default: if constexpr (G > 3) tree_group<R, N, BLOCK, HB, G, 3>(L, are, aim); break;
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

// Lane coordinates in a round: point slot, subtree group, group-local lane.
template <int N, int BLOCK, int HB, int G>
struct LaneId {
    using S = TreeShape<N, BLOCK, HB, G>;
    int slot, g, hl;
    __device__ __forceinline__ explicit LaneId(int tid)
        : slot(tid / S::LPP), g((tid % S::LPP) / S::NSL), hl(tid % S::NSL) {}
};

// The complete amplitudes of the lane's rows: with several subtree groups,
// every group leaves its partial sums in shared memory and group 0 adds them
// (the other groups' amplitudes become 0).  All threads must call it.
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
#pragma unroll
            for (int gg = 1; gg < G; ++gg) {
                const R* y = tb.XCH + (size_t)(threadIdx.x + gg * S::NSL) * H * 2;
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

// Sum (MAX = false) or maximum (MAX = true) of v over the lanes of each point;
// the result is valid in the point's first lane.  All threads must call it.
template <class R, int N, int BLOCK, int BAR, int HB, int G, bool MAX>
__device__ __forceinline__ R point_reduce(const RoundTables<R, N, BLOCK, HB, G>& tb, R v) {
    using S = TreeShape<N, BLOCK, HB, G>;
    constexpr int W = S::LPP < 32 ? S::LPP : 32;
#pragma unroll
    for (int off = 1; off < W; off <<= 1) {
        const R o = __shfl_xor_sync(0xffffffffu, v, off);
        v = MAX ? fmax(v, o) : v + o;
    }
    if constexpr (S::LPP > 32) {
        const int tid = threadIdx.x;
        if ((tid & 31) == 0) tb.RED[tid >> 5] = v;
        group_sync<BAR, BLOCK>();
        if (tid % S::LPP == 0)
            for (int w = 1; w < S::LPP / 32; ++w) {
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
    const LaneTables<R, N, BLOCK, HB, G> L{tb.M0, tb.M1, tb.CL, tb.R1, 2 * id.slot, (unsigned)id.hl, tb.PC};
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
        if (threadIdx.x % S::LPP == 0 && id.slot < rc) recs[base + id.slot].ssum = v;
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
    const LaneTables<R, N, BLOCK> L{tb.M0, tb.M1, tb.CL, tb.R1, 2 * id.slot, (unsigned)id.hl, tb.PC};
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
        if (threadIdx.x % (1 << N) == 0 && id.slot < rc) {
            const R a = best[0], w = best[1];
            recs[base + id.slot].ssum = a > R(0) ? sqrt(w / a) : (w > R(0) ? R(INFINITY) : R(0));
        }
        __syncthreads();
    }
}

}  // namespace heget
