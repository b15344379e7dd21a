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
// (j, T, lambda_j) only and are precomputed per point in shared memory.
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

// Shared-memory tables of one round: P = BLOCK / 2^N points.
// Entry layout [index][point][lambda] so that the lanes of a warp, which read
// one index for up to 32/2^N points and both lambdas, hit distinct banks.
template <class R, int N, int BLOCK>
struct RoundTables {
    static constexpr int P = BLOCK >> N;
    static constexpr int K = num_pairs(N);
    static constexpr int NS = 1 << N;
    static constexpr size_t m_elems = (size_t)K * P * 2;
    static constexpr size_t c_elems = (size_t)N * P * 2;
    static constexpr size_t bytes = (2 * m_elems + 2 * c_elems) * sizeof(Row<R>)   // M0, M1, CL, R1
                                  + (size_t)P * N * sizeof(Row<R>)                 // photon data
                                  + (size_t)P * NS * sizeof(Row<R>)                // set data
                                  + (size_t)(BLOCK / 32) * sizeof(R) + 16;         // reduction
    Row<R>* M0;
    Row<R>* M1;
    Row<R>* CL;
    Row<R>* R1;
    Row<R>* PH;   // [P][N]: (sin th, cos th, cos ph, sin ph)
    Row<R>* SD;   // [P][2^N]: (A, D, Bre, Bim) = ((q0+q3), (q0-q3), q1, q2) / q^2
    R* RED;       // [BLOCK/32]
    __device__ __forceinline__ explicit RoundTables(unsigned char* base) {
        M0 = reinterpret_cast<Row<R>*>(base);
        M1 = M0 + m_elems;
        CL = M1 + m_elems;
        R1 = CL + c_elems;
        PH = R1 + c_elems;
        SD = PH + (size_t)P * N;
        RED = reinterpret_cast<R*>(SD + (size_t)P * NS);
    }
};

// Fill the round tables for points recs[0 .. cnt-1] (cnt <= P).  Two phases
// separated by barriers; all threads of the block must call it.  Everything
// here runs in R: the FP64 content (invariants) is already in the records.
// ward >= 0 replaces the polarisation of that photon by k/k^0 in every step,
// closure and first row (the gauge check; both lambda entries then agree).
template <class R, int N, int BLOCK, int BAR = 0>
__device__ __forceinline__ void setup_round(const RoundTables<R, N, BLOCK>& tb, const PointRec<R, N>* recs,
                                            int cnt, int ward = -1) {
    using RT = RoundTables<R, N, BLOCK>;
    constexpr int P = RT::P, K = RT::K, NS = RT::NS;
    const int tid = threadIdx.x;
    // (a) photon angles, and propagator data per photon set T:
    //     Qbar_T / t_T with t_T summed from the invariants
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
            tb.PH[p * N + j] = d;
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
            tb.SD[p * NS + T] = d;
        }
    }
    group_sync<BAR, BLOCK>();
    // (b) step matrices M(j, T) = E_j^lambda Qbar_T, closures and first rows
    const R rs2 = R(0.70710678118654752440);
    for (int it = tid; it < P * K * 2; it += BLOCK) {
        const int lam_bit = it & 1;
        const int q = it >> 1;
        const int p = q % P;
        const int idx = q / P;
        if (p >= cnt) continue;
        const uint16_t pr = c_tables.pair[pair_offset(N) + idx];
        const int T = pr & 0xFF, j = pr >> 8;
        const R lam = lam_bit ? R(1) : R(-1);
        const Row<R> ph = tb.PH[p * N + j];
        const Row<R> sd = tb.SD[p * NS + T];
        // E = eps*(k, lambda) . sigma = (1/sqrt2) [[-l s, -(1 - l c) e^{-i phi}],
        //                                         [(1 + l c) e^{i phi}, l s]]
        R e00 = -lam * ph.ar * rs2;
        R e11 = -e00;
        const R am = (R(1) - lam * ph.ai) * rs2, ap = (R(1) + lam * ph.ai) * rs2;
        R e01r = -am * ph.br, e01i = am * ph.bi;   // -(1 - l c) e^{-i phi}
        R e10r = ap * ph.br, e10i = ap * ph.bi;    //  (1 + l c) e^{+i phi}
        if (j == ward) {
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
        Row<R> m0, m1;
        m0.ar = e00 * A + e01r * Br - e01i * Bi;   // M00 = e00 A + e01 B
        m0.ai = e01r * Bi + e01i * Br;
        m0.br = e00 * Br + e01r * D;               // M01 = e00 B* + e01 D
        m0.bi = -e00 * Bi + e01i * D;
        m1.ar = e10r * A + e11 * Br;               // M10 = e10 A + e11 B
        m1.ai = e10i * A + e11 * Bi;
        m1.br = e10r * Br + e10i * Bi + e11 * D;   // M11 = e10 B* + e11 D
        m1.bi = e10i * Br - e10r * Bi;
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
}

// Per-lane view of the round tables.
template <class R, int N, int BLOCK>
struct LaneTables {
    static constexpr int P = BLOCK >> N;
    const Row<R>* M0;
    const Row<R>* M1;
    const Row<R>* CL;
    const Row<R>* R1;
    int pp;       // 2 * point slot
    unsigned h;   // photon helicity bits of this lane
    __device__ __forceinline__ int lam(int j) const { return (h >> j) & 1; }
};

// Depth-first walk of the ordering tree below a node at depth D (D photons
// attached, set T, current row r), adding the closures to acc.
template <class R, int N, int D, int BLOCK>
__device__ __forceinline__ void descend(const LaneTables<R, N, BLOCK>& L, const Row<R>& r, unsigned T,
                                        R& acc_re, R& acc_im) {
    constexpr unsigned FULL = (1u << N) - 1;
    constexpr int P = BLOCK >> N;
    if constexpr (D == N - 1) {
        const int j = __ffs(FULL & ~T) - 1;
        const Row<R> c = ld_row(L.CL + (j * P * 2 + L.pp + L.lam(j)));
        acc_re += r.ar * c.ar - r.ai * c.ai + r.br * c.br - r.bi * c.bi;
        acc_im += r.ar * c.ai + r.ai * c.ar + r.br * c.bi + r.bi * c.br;
    } else {
        unsigned rem = FULL & ~T;
#pragma unroll 1
        while (rem) {
            const int j = __ffs(rem) - 1;
            rem &= rem - 1;
            const int idx = c_tables.child[child_offset(N) + T * N + j];
            const int o = idx * P * 2 + L.pp + L.lam(j);
            const Row<R> r2 = row_times(r, ld_row(L.M0 + o), ld_row(L.M1 + o));
            descend<R, N, D + 1, BLOCK>(L, r2, T | (1u << j), acc_re, acc_im);
        }
    }
}

// The full tree for one lane: sum over all n! orderings of the helicity
// amplitude (up to normalisation) for photon helicities h, s1 = +.
template <class R, int N, int BLOCK>
__device__ __forceinline__ void tree_amplitude(const LaneTables<R, N, BLOCK>& L, R& acc_re, R& acc_im) {
    constexpr int P = BLOCK >> N;
    acc_re = R(0);
    acc_im = R(0);
#pragma unroll 1
    for (int j = 0; j < N; ++j) {
        const Row<R> r1 = ld_row(L.R1 + (j * P * 2 + L.pp + L.lam(j)));
        descend<R, N, 1, BLOCK>(L, r1, 1u << j, acc_re, acc_im);
    }
}

// Parity-folded helicity weight of lane h (see file comment).
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

// Amplitude rounds over recs[0 .. cnt-1].  For each point the lane group's
// reduction yields S = sum_h w_h |A_h|^2 (scaled units), stored by the
// group's first thread in recs[p].ssum; the FP64 normalisation and the
// accumulation are left to whole warps afterwards (one lane per point), so
// no FP64 instruction here runs with one or two active lanes.
template <class R, int N, int BLOCK, int BAR = 0>
__device__ __forceinline__ void amplitude_rounds(unsigned char* table_smem, PointRec<R, N>* recs, int cnt, float wh) {
    using RT = RoundTables<R, N, BLOCK>;
    constexpr int P = RT::P;
    constexpr int NS = 1 << N;
    const RT tb(table_smem);
    const int tid = threadIdx.x;
    const int slot = tid >> N;
    LaneTables<R, N, BLOCK> L{tb.M0, tb.M1, tb.CL, tb.R1, 2 * slot, (unsigned)(tid & (NS - 1))};
    for (int base = 0; base < cnt; base += P) {
        const int rc = min(P, cnt - base);
        setup_round<R, N, BLOCK, BAR>(tb, recs + base, rc);
        R are = R(0), aim = R(0);
        const bool active = slot < rc && recs[base + slot].valid;
        if (active) tree_amplitude<R, N, BLOCK>(L, are, aim);
        R v = (are * are + aim * aim) * R(wh);
        constexpr int G = NS < 32 ? NS : 32;
#pragma unroll
        for (int off = 1; off < G; off <<= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if constexpr (NS <= 32) {
            if ((tid & (NS - 1)) == 0 && slot < rc) recs[base + slot].ssum = v;
        } else {
            if ((tid & 31) == 0) tb.RED[tid >> 5] = v;
            group_sync<BAR, BLOCK>();
            if ((tid & (NS - 1)) == 0 && slot < rc) {
                R s = R(0);
                for (int w = 0; w < NS / 32; ++w) s += tb.RED[(tid >> 5) + w];
                recs[base + slot].ssum = s;
            }
        }
        group_sync<BAR, BLOCK>();
    }
}

// Gauge check rounds over recs[0 .. cnt-1]: for each point the largest
// |A_h|^2 over the 2^N photon-helicity lanes (s1 = +) of the ordinary tree
// and of the tree with photon `ward` replaced by k/k^0; stores
// sqrt(max |W_h|^2 / max |A_h|^2) in recs[p].ssum.  |M_h|^2 of the s1 = -
// configurations equal those of s1 = + by parity, so the maxima cover all
// helicities.
template <class R, int N, int BLOCK>
__device__ __forceinline__ void ward_rounds(unsigned char* table_smem, PointRec<R, N>* recs, int cnt, int ward) {
    using RT = RoundTables<R, N, BLOCK>;
    constexpr int P = RT::P;
    constexpr int NS = 1 << N;
    const RT tb(table_smem);
    const int tid = threadIdx.x;
    const int slot = tid >> N;
    LaneTables<R, N, BLOCK> L{tb.M0, tb.M1, tb.CL, tb.R1, 2 * slot, (unsigned)(tid & (NS - 1))};
    for (int base = 0; base < cnt; base += P) {
        const int rc = min(P, cnt - base);
        R best[2];
#pragma unroll 1
        for (int pass = 0; pass < 2; ++pass) {
            setup_round<R, N, BLOCK>(tb, recs + base, rc, pass ? ward : -1);
            R are = R(0), aim = R(0);
            const bool active = slot < rc && recs[base + slot].valid;
            if (active) tree_amplitude<R, N, BLOCK>(L, are, aim);
            R v = are * are + aim * aim;
            constexpr int G = NS < 32 ? NS : 32;
#pragma unroll
            for (int off = 1; off < G; off <<= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
            if constexpr (NS > 32) {
                if ((tid & 31) == 0) tb.RED[tid >> 5] = v;
                __syncthreads();
                if ((tid & (NS - 1)) == 0)
                    for (int w = 1; w < NS / 32; ++w) v = fmax(v, tb.RED[(tid >> 5) + w]);
                __syncthreads();
            }
            best[pass] = v;
        }
        if ((tid & (NS - 1)) == 0 && slot < rc) {
            const R a = best[0], w = best[1];
            recs[base + slot].ssum = a > R(0) ? sqrt(w / a) : (w > R(0) ? R(INFINITY) : R(0));
        }
        __syncthreads();
    }
}

}  // namespace heget
