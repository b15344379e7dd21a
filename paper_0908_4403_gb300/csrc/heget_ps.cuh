// heget_ps.cuh -- FP64 phase-space generation on the device: sqrt(s-hat)
// samplers, RAMBO flat massless n-body phase space (Sec. 2.1 eq. (4);
// Kleiss, Stirling, Ellis, CPC 40 (1986) 359), the photon cuts of Sec. 2.2
// eqs. (9)-(10), and the per-point record the amplitude kernels consume.
//
// GB300 executes FP64 at about 1/64 of the FP32 rate, so this file keeps
// FP64 for what needs it (RAMBO energies, angles and boosts; the Lorentz
// invariants behind the propagator denominators; cut decisions) and avoids
// FP64 transcendentals where an algebraic identity gives the same decision.
#pragma once

#include "heget_common.cuh"
#include "heget_logtab.h"
#include "heget_sincostab.h"

namespace heget {

// Point record staged in shared memory between event generation (or input
// loading) and the amplitude rounds.  Momenta are divided by sqrt(s-hat) so
// that the FP32 chain works on O(1) numbers; the mass dimension 4 - 2n of
// |M|^2 is restored by `fac`.  The propagator denominators
//   t_T = (sum_{i in T} k_i - p2)^2 / s-hat,   T a proper photon subset,
// come from FP64: FP64 records and FP32 records up to n = 5 hold every t_T,
// computed in FP64 when the record is built (fill_denominators,
// set_denominator) and rounded once to R.  FP32 records from n = 6 hold the
// Lorentz invariants instead, t_T being a sum of them over T or, by momentum
// conservation (k_T - p2 = p1 - k_S, S = all - T), over its complement S,
//   t_T = sum_{i in T} d_i + sum_{i<j in T} s_ij = sum_{i in S} d'_i + sum_{i<j in S} s_ij,
//   d_i = k_i^2 - 2 k_i.p2,  d'_i = k_i^2 - 2 k_i.p1,  s_ij = 2 k_i.k_j,
// each computed in FP64 and kept as an unevaluated sum of two floats
// (hi + lo, about 48 significant bits); the rounds add up those of the
// smaller of T and S in float-float arithmetic (rec_denominator), so the
// FP32 chain again sees t_T with far more than FP32 accuracy, while the FP64
// pipe forms n(n+3)/2 invariants per point instead of 2^n - 2 sums.
template <class R, int N>
__host__ __device__ constexpr bool rec_invariants() {
    return sizeof(R) == sizeof(float) && N >= 6;
}
template <class R, int N, bool INV = rec_invariants<R, N>()>
struct RecDenominators {
    R t[1 << N];      // t_T by subset bitmask T (entries 0 and 2^n - 1 unused)
};
template <class R, int N>
struct RecDenominators<R, N, true> {
    float2 inv[N * (N + 3) / 2];   // (hi, lo): d_i at i, s_ij at N + pair_index(i, j), d'_i after them
};
template <class R, int N>
struct alignas(16) PointRec : RecDenominators<R, N> {
    double fac;       // (4 pi alpha Q^2)^n s-hat^(2-n): scaled sum -> |M|^2
    double wfac;      // scaled sum -> event weight (fb); 0 if masked
    R k[N][4];        // photon momenta / sqrt(s-hat)
    R e1, e2;         // energies of p1, p2 / sqrt(s-hat)  (p1 = e1 (1, 0, 0, 1), p2 = e2 (1, 0, 0, -1))
    R n1, n2;         // sqrt(2 e1), sqrt(2 e2): spinor normalisations
    R ssum;           // result of the tree: sum_h w_h |A_h|^2 in scaled units
    R kap2;           // sum_h w_h B_h^2, B_h >= sum over orderings |A_pi,h| (condition bound)
    int hsel;         // -1: every helicity; >= 0: only this lane (a sampled helicity); -2: none
    int valid;        // 0: amplitude not evaluated (bad input / sampler failure)
    int mask;         // passes the cuts
    int tries;        // outer sampler attempts
    int idx;          // the point's index within its tile or stage (records are compacted)
};

template <int N>
__host__ __device__ constexpr int pair_index(int i, int j) {  // i < j
    return i * N - i * (i + 1) / 2 + (j - i - 1);
}

// Flat massless n-body volume constant: Phi_n(s) = c_n s^(n-2) with
// c_n = (2 pi)^(4-3n) (pi/2)^(n-1) / ((n-1)! (n-2)!).
__host__ __device__ inline double phase_space_const(int n) {
    const double two_pi = 6.283185307179586476925287;
    const double half_pi = 1.570796326794896619231322;
    double f1 = 1, f2 = 1, c = 1;
    for (int i = 2; i <= n - 1; ++i) f1 *= i;
    for (int i = 2; i <= n - 2; ++i) f2 *= i;
    for (int i = 0; i < 3 * n - 4; ++i) c /= two_pi;
    for (int i = 0; i < n - 1; ++i) c *= half_pi;
    return c / (f1 * f2);
}

// FP32 estimate of the uniform u01_from_words(lo, hi) from its top 24 bits:
// |result - u| <= 2^-24.
__device__ __forceinline__ float u01_estimate(uint32_t hi) {
    return (__uint2float_rn(hi >> 8) + 0.5f) * 0x1p-24f;
}

// Toy-PDF momentum fraction: proposal x = u^2 (density ~ x^-1/2), accepted
// if v < (1-x)^3 (both uniforms from one Philox block per try); false when
// the bound of tries is hit.
//
// The acceptance test is the FP64 comparison v < (1 - u^2)^3, with the
// products and the difference rounded separately.  Most tries are settled
// first in FP32 from the same random bits: with |u_f - u|, |v_f - v| <= 2^-24,
// the FP32 value t_f of t = (1-u^2)^3 satisfies |t_f - t| <= 5.1 2^-24 (the
// input error through 3(1-u^2)^2 (2u + u^2 + 1/2) <= 3.1, plus two roundings
// of the cube), so |v_f - t_f| > 2^-20 = 16 2^-24 decides the comparison the
// same way; the FP64 test runs only inside that band (about 2e-6 of the
// tries).
//
// The loop itself is integer and FP32 work (plus the rare FP64 tie-break);
// it returns the accepted try's random words, and the caller converts them to
// x = u^2 in FP64 after the loop, where the lanes of a warp have converged.
__device__ __forceinline__ bool toy_pdf_draw(const PointRng& rng, uint32_t& blk, int max_tries, uint32_t& wx,
                                             uint32_t& wy) {
    for (int t = 0; t < max_tries; ++t) {
        const U4 w = philox4x32_10(U4{rng.ilo, rng.ihi, blk++, kStreamSqrtS}, rng.k0, rng.k1);
        const float uf = u01_estimate(w.y), vf = u01_estimate(w.w);
        const float of = 1.0f - uf * uf;
        const float tf = of * of * of;
        bool accept;
        if (vf < tf - 0x1p-20f) {
            accept = true;
        } else if (vf > tf + 0x1p-20f) {
            accept = false;
        } else {
            const double u = u01_from_words(w.x, w.y), v = u01_from_words(w.z, w.w);
            const double om = __dsub_rn(1.0, __dmul_rn(u, u));
            accept = v < __dmul_rn(__dmul_rn(om, om), om);
        }
        if (accept) {
            wx = w.x;
            wy = w.y;
            return true;
        }
    }
    return false;
}

__device__ __forceinline__ double toy_pdf_x_of(uint32_t wx, uint32_t wy) {
    const double u = u01_from_words(wx, wy);
    return __dmul_rn(u, u);
}

// Scalars of one generated event; its photon momenta (GeV) live in a MomView.
// ey, iey: e^y and e^-y of the partonic frame's rapidity y (1 for the fixed
// and uniform samplers).
struct EventInfo {
    double rs, irs, ey, iey, x1, x2;
    int tries, ok, mask;
};

// Helicity sampling (the paper's events carry one random helicity
// combination, Sec. 3): h = floor(2^(n+2) u) with u draw 0 of the helicity
// stream, bits as everywhere (bit 0 sigma1, bit 1 sigma2, bit 2 + i lambda_i).
// The kernels compute the lanes lambda with sigma1 = +, sigma2 = -; h with
// sigma1 = sigma2 vanishes exactly (-2: no lane), and h with sigma1 = -,
// sigma2 = + equals its parity image, the lane ~lambda.
template <int N>
__device__ __forceinline__ int sampled_lane(const PointRng& rng) {
    const U4 w = rng.words(kStreamHelicity, 0);
    const int h = (int)(u01_from_words(w.x, w.y) * (double)(1 << (N + 2)));
    const int s1 = h & 1, s2 = (h >> 1) & 1, lam = h >> 2;
    return s1 == s2 ? -2 : s1 ? lam : (~lam & ((1 << N) - 1));
}

// The record's lane selection (PointRec::hsel) for point i of stream seed:
// drawn when the record is written, so nothing stays live across RAMBO.
template <int N>
__device__ __forceinline__ int point_hsel(const Physics& ph, uint64_t seed, uint64_t i) {
    return ph.hel_sample ? sampled_lane<N>(PointRng(seed, i)) : -1;
}

// The sampler's random draws for one point, kept apart from the FP64 rest
// of the event: integer and FP32 work (plus a rare FP64 tie-break), which
// another set of threads can run ahead of time.  16 bytes: u01_from_words
// ignores the low 12 bits of its low word, so those of ax carry the outer
// attempts and the success flag.
struct alignas(16) SampleDraw {
    uint32_t ax, ay;   // toy PDF: words of the accepted x1 draw; uniform: the words of sqrt(s-hat)
    uint32_t bx, by;   // toy PDF: words of the accepted x2 draw
    __device__ __forceinline__ int tries() const { return (int)((ax >> 1) & 0x7FFu); }
    __device__ __forceinline__ int ok() const { return (int)(ax & 1u); }
    __device__ __forceinline__ void set(int tries, int ok) { ax = (ax & ~0xFFFu) | ((uint32_t)tries << 1) | (uint32_t)ok; }
};

__device__ __forceinline__ SampleDraw sample_draw(const SamplerArgs& S, const PointRng& rng) {
    SampleDraw d{0u, 0u, 0u, 0u};
    if (S.kind == HEGET_SAMPLER_FIXED) {
        d.set(1, 1);
        return d;
    }
    if (S.kind == HEGET_SAMPLER_UNIFORM) {
        const U4 w = rng.words(kStreamSqrtS, 0);
        d.ax = w.x;
        d.ay = w.y;
        d.set(1, 1);
        return d;
    }
    // The floor test r > floor, r = 2 E sqrt(x1 x2) in FP64, is the test
    // u_a u_b > floor / (2 E) on the uniforms behind x = u^2; their FP32
    // estimates (within 2^-24) settle it outside a band of +-16 2^-24 around
    // the threshold, and the FP64 r decides inside it.  So the loop runs on
    // integer and FP32 work, and r and the fractions are formed once, by
    // sample_finish.
    uint32_t blk = 0;
    int tries = S.max_tries, ok = 0;
    for (int t = 1; t <= S.max_tries; ++t) {
        if (!toy_pdf_draw(rng, blk, S.max_tries, d.ax, d.ay)) break;
        if (!toy_pdf_draw(rng, blk, S.max_tries, d.bx, d.by)) break;
        const float p = u01_estimate(d.ay) * u01_estimate(d.by);
        bool pass = p > S.band_hi;
        if (!pass && p >= S.band_lo) {   // rare
            const double a = toy_pdf_x_of(d.ax, d.ay), b = toy_pdf_x_of(d.bx, d.by);
            pass = 2.0 * S.e_beam * sqrt(a * b) > S.floor;
        }
        if (pass) {
            tries = t;
            ok = 1;
            break;
        }
    }
    d.set(tries, ok);
    return d;
}

// sqrt(s-hat) and its inverse, the momentum fractions, the boost factors
// e^+-y and the outer attempts from the draws.  With sqrt(s-hat) = 2 E
// sqrt(x1 x2), e^y = sqrt(x1 / x2) = 2 E x1 / sqrt(s-hat) and e^-y = 2 E x2 /
// sqrt(s-hat): one division serves all three.  y itself (a logarithm) is
// left to callers that output it.
__device__ __forceinline__ void sample_finish(const SamplerArgs& S, const SampleDraw& d, EventInfo& ev) {
    ev.ok = d.ok();
    ev.tries = d.tries();
    ev.ey = ev.iey = 1.0;
    ev.x1 = ev.x2 = 1.0;
    if (S.kind == HEGET_SAMPLER_FIXED) {
        ev.rs = S.sqrt_s;
        ev.irs = 1.0 / ev.rs;
        return;
    }
    if (S.kind == HEGET_SAMPLER_UNIFORM) {
        ev.rs = S.lo + (S.hi - S.lo) * u01_from_words(d.ax, d.ay);
        ev.irs = 1.0 / ev.rs;
        return;
    }
    if (ev.ok) {
        ev.x1 = toy_pdf_x_of(d.ax, d.ay);
        ev.x2 = toy_pdf_x_of(d.bx, d.by);
        ev.rs = 2.0 * S.e_beam * sqrt(ev.x1 * ev.x2);
    } else {
        ev.rs = S.floor;
    }
    ev.irs = 1.0 / ev.rs;
    const double h = 2.0 * S.e_beam * ev.irs;
    ev.ey = ev.ok ? ev.x1 * h : 1.0;
    ev.iey = ev.ok ? ev.x2 * h : 1.0;
}

// Photon momenta of one point held in shared memory: slot (a, m) at
// p[(slots a + m) * stride], m = 0..3 the components (E, px, py, pz).
// Generated points use slots = kMomSlots with stride = points of the tile
// (point-minor layout: consecutive threads touch consecutive words); input
// rows use slots = 4, stride = 1.
constexpr int kMomSlots = 4;

struct MomView {
    double* p;
    int stride;
    int slots;
    __device__ __forceinline__ double& operator()(int a, int m) const { return p[(slots * a + m) * stride]; }
};

// double -> float, rounded to nearest even, by integer operations on the bit
// pattern: on GB300 the hardware conversion occupies the FP64 pipe, which
// the event generation saturates.  Exact for results in the normal float
// range; results below it become a signed zero (no subnormals), above it
// +-inf, and NaN stays NaN.
__device__ __forceinline__ float f32_rn(double x) {
    // 32-bit words throughout: the round bit is bit 28 of lo, the sticky bits
    // 0..27, the kept bits start at 29; the exponent field of
    // (|x| >> 29) mod 2^32 minus (1023 - 127) << 23 is the float's, and a
    // round-up carry out of the mantissa moves into it
    const unsigned int hi = (unsigned int)__double2hiint(x), lo = (unsigned int)__double2loint(x);
    const unsigned int habs = hi & 0x7FFFFFFFu, sign = hi & 0x80000000u;
    const unsigned int t = __funnelshift_r(lo, habs, 29);          // exponent and top mantissa bits
    const unsigned int inc = (lo >> 28) & ((lo & 0x2FFFFFFFu) != 0u ? 1u : 0u);   // round bit and (sticky or lsb)
    unsigned int f = t - (896u << 23) + inc;
    f = habs < 0x38100000u ? 0u : f;
    f = habs >= 0x47F00000u ? ((habs > 0x7FF00000u || (habs == 0x7FF00000u && lo != 0u)) ? 0x7FC00000u : 0x7F800000u) : f;
    return __uint_as_float(f | sign);
}

// A record field from its FP64 value: f32_rn for FP32 records.
template <class R>
__device__ __forceinline__ R rec_value(double x) {
    if constexpr (sizeof(R) == sizeof(float)) return f32_rn(x);
    else return x;
}

// Natural logarithm of a positive normal double by Tang's table-driven method
// (P. T. P. Tang, ACM TOMS 16 (1990) 378): x = 2^e m with m in [1, 2), F the
// nearest breakpoint 1 + j/256, f = m - F (exact, |f| <= 1/512), r = f / F,
//   ln x = e ln 2 + ln F + ln(1 + r),
// with ln F and ln 2 from double-double tables (heget_logtab.h) and ln(1 + r)
// by its series to r^6 (|r| <= 2^-9: truncation below 2^-56 relative).  F and
// e become doubles through their bit patterns, so the whole costs 15 FP64
// operations instead of a general-purpose logarithm, for the RAMBO energies.
__device__ __forceinline__ double log_table(double x) {
    const int hi = __double2hiint(x), lo = __double2loint(x);
    const int e = ((hi >> 20) & 0x7FF) - 1023;
    const double m = __hiloint2double((hi & 0x000FFFFF) | 0x3FF00000, lo);
    const int j = (((hi >> 11) & 0x1FF) + 1) >> 1;            // nearest breakpoint, 0 .. 256
    const double F = __hiloint2double(0x3FF00000 + (j << 12), 0);   // 1 + j/256
    const double f = m - F;                                          // exact
    const double r = f * __ldg(&kLogTab[j][2]);
    // ln(1 + r) - r = r^2 (-1/2 + r (1/3 + r (-1/4 + r (1/5 - r/6))))
    double q = -1.0 / 6.0;
    q = fma(q, r, 0.2);
    q = fma(q, r, -0.25);
    q = fma(q, r, 1.0 / 3.0);
    q = fma(q, r, -0.5);
    const double p = r * r * q;
    // e as a double: 2^52 + 2^31 + e carries e in its low mantissa bits
    const double ed = __hiloint2double(0x43300000, (int)(0x80000000u + (unsigned)e)) - 0x1.00000800p52;
    const double lhi = fma(ed, kLn2Hi, __ldg(&kLogTab[j][0]));
    const double llo = fma(ed, kLn2Lo, __ldg(&kLogTab[j][1]));
    return lhi + (r + (p + llo));
}

// cos and sin of the RAMBO azimuth phi = 2 pi r for the uniform
// r = u01_from_words(lo, hi) = (2m + 1) 2^-53, m the top 52 bits of (hi, lo),
// by a breakpoint table (heget_sincostab.h): j = round(512 r), a = 2 pi j/512
// and theta = 2 pi (r - j/512), |theta| <= pi/512.  The remainder is exact:
// r - j/512 = D 2^-53 with the integer D = 2m + 1 - j 2^44, |D| <= 2^43.  With
// s = sin theta and c' = cos theta - 1 by their Taylor series (truncated below
// 1e-19),
//   cos phi = cos a + (c' cos a - s sin a),  sin phi = sin a + (c' sin a + s cos a),
// within about 2 ulp; 15 FP64 operations and one table load.
__device__ __forceinline__ void sincos_2pi_words(uint32_t lo, uint32_t hi, double& sp, double& cp) {
    const unsigned long long m = ((((unsigned long long)hi) << 32) | lo) >> 12;
    const unsigned long long j = (m + (1ull << 42)) >> 43;   // 0 .. 512
    const long long D = (long long)(2 * m + 1) - (long long)(j << 44);
    // D as a double without a conversion: 1.5 2^52 + D has D in its mantissa
    const double d = __longlong_as_double(0x4338000000000000ll + D) - 0x1.8p52;
    const double th = d * 0x1.921fb54442d18p-51;   // 2 pi 2^-53
    const double t2 = th * th;
    const double s = fma(th * t2, fma(t2, 1.0 / 120.0, -1.0 / 6.0), th);
    const double cm = t2 * fma(t2, fma(t2, -1.0 / 720.0, 1.0 / 24.0), -0.5);
    const double2 a = __ldg(&kSinCosTab[j & (kSinCosTable - 1)]);
    cp = a.x + fma(a.x, cm, -(a.y * s));
    sp = a.y + fma(a.y, cm, a.x * s);
}

// RAMBO: n massless momenta with total (rs, 0, 0, 0).  Photon i uses draws
// 4i..4i+3 of the RAMBO stream: cos(theta) = 2 r0 - 1, phi = 2 pi r1,
// q0 = -ln(r2 r3); the isotropic q_i are boosted and scaled onto the total.
template <int N>
__device__ __forceinline__ void rambo(const PointRng& rng, double rs, const MomView& v) {
    double Q0 = 0, Q1 = 0, Q2 = 0, Q3 = 0;
#pragma unroll 1
    for (int i = 0; i < N; ++i) {
        const U4 w = rng.words(kStreamRambo, 2 * i);   // r0 = u(w.x, w.y), r1 = u(w.z, w.w)
        double r2, r3;
        rng.pair(kStreamRambo, 2 * i + 1, r2, r3);
        const double c = 2.0 * u01_from_words(w.x, w.y) - 1.0;
        const double s2 = 1.0 - c * c;   // in [2^-51, 1): never 0
        const double s = s2 * rsqrt(s2);
        double sp, cp;
        sincos_2pi_words(w.z, w.w, sp, cp);
        const double q0 = -log_table(r2 * r3);   // r2 r3 in [2^-106, 1): normal
        const double qs = q0 * s;
        const double q1 = qs * cp, q2 = qs * sp, q3 = q0 * c;
        v(i, 0) = q0;
        v(i, 1) = q1;
        v(i, 2) = q2;
        v(i, 3) = q3;
        Q0 += q0;
        Q1 += q1;
        Q2 += q2;
        Q3 += q3;
    }
    // M = sqrt(Q^2), b = -Q/M, gamma = Q0/M, a = 1/(1 + gamma) = M/(M + Q0),
    // x = rs/M; then p_i = x (gamma q0 + b.q, q + b (q0 + a b.q)).
    const double M2 = Q0 * Q0 - Q1 * Q1 - Q2 * Q2 - Q3 * Q3;
    const double iM = rsqrt(M2);
    const double M = M2 * iM;
    const double b1 = -Q1 * iM, b2 = -Q2 * iM, b3 = -Q3 * iM;
    const double a = M / (M + Q0);
    const double x = rs * iM;
    const double xg = x * (Q0 * iM), xb1 = x * b1, xb2 = x * b2, xb3 = x * b3;
#pragma unroll 1
    for (int i = 0; i < N; ++i) {
        const double q0 = v(i, 0), q1 = v(i, 1), q2 = v(i, 2), q3 = v(i, 3);
        const double bq = b1 * q1 + b2 * q2 + b3 * q3;
        const double t = fma(a, bq, q0);
        v(i, 0) = fma(xg, q0, x * bq);
        v(i, 1) = fma(xb1, t, x * q1);
        v(i, 2) = fma(xb2, t, x * q2);
        v(i, 3) = fma(xb3, t, x * q3);
    }
}

// a < b for doubles a, b >= +0 (squares and their products, never -0 or
// NaN): their IEEE bit patterns order like the values, so the comparison
// runs on the integer pipe, not on the FP64 pipe with the arithmetic.
__device__ __forceinline__ bool lt_nonneg(double a, double b) {
    return __double_as_longlong(a) < __double_as_longlong(b);
}

// v < 0 from the bit pattern (false for -0).
__device__ __forceinline__ bool is_negative(double v) {
    const long long b = __double_as_longlong(v);
    return b < 0 && (b << 1) != 0;
}

// v < a * w, decided on squares (w >= 0): no square root; written with
// selects, so the lanes of a warp stay together.
__device__ __forceinline__ bool lt_scaled(double v, double a, double w2) {
    const double v2 = v * v, r2 = a * a * w2;
    const bool neg = is_negative(v);
    return a >= 0 ? (neg || lt_nonneg(v2, r2)) : (neg && lt_nonneg(r2, v2));
}

// Photon cuts, strict (Sec. 2.2): pT > pt_min, |eta + y| < eta_max with
// eta = asinh(pz / pT), and Delta R = sqrt(Delta eta^2 + Delta phi^2) > dr_min
// for every pair (Delta phi in [0, pi]); dr_min <= 0 disables Delta R.
// Evaluated without per-photon transcendentals:
//   eta + y in (-E, E)  <=>  pz / pT in (sinh(-E - y), sinh(E - y)),
//     sinh(E -+ y) = sinh E cosh y -+ cosh E sinh y with e^y = sqrt(x1/x2);
//   sinh(eta_i - eta_j) = (pz_i E_j - pz_j E_i) / (pT_i pT_j)   (|p| = E),
//   cos(phi_i - phi_j)  = (px_i px_j + py_i py_j) / (pT_i pT_j);
// a pair passes at once if |Delta eta| > R or Delta phi > R (compared on
// squares), and only the remaining close pairs evaluate asinh and atan2.
// ey, iey: e^y and e^-y.
template <int N>
__device__ __forceinline__ int pass_cuts(const MomView& p, double ey, double iey, const Physics& ph) {
    // every photon and pair is tested without early exits: the FP64 pipe
    // executes whole warps, so a lane that could stop early saves nothing and
    // the divergence would cost the others
    const double shy = 0.5 * (ey - iey), chy = 0.5 * (ey + iey);
    const double s_hi = ph.sinh_eta * chy - ph.cosh_eta * shy;    // sinh(E - y)
    const double s_lo = -ph.sinh_eta * chy - ph.cosh_eta * shy;   // sinh(-E - y)
    const double pt2min = ph.pt_min * ph.pt_min;
    bool ok = true;
    double pt2[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const double pz = p(i, 3);
        pt2[i] = p(i, 1) * p(i, 1) + p(i, 2) * p(i, 2);
        // pT > pt_min and s_lo pT < pz < s_hi pT
        ok = ok & lt_nonneg(pt2min, pt2[i]) & lt_scaled(pz, s_hi, pt2[i]) & lt_scaled(-pz, -s_lo, pt2[i]);
    }
    if (ph.dr_min > 0) {
        // squares only: |p| = E for massless photons, and the sinh / cos
        // comparisons are decided on squares; pT_i pT_j (a square root) is
        // formed only for the close pairs that need asinh and atan2.  The
        // pairs are screened first (pair_index bits of `close`), then the
        // close ones, which are rare, settled one by one.
        const double sdr2 = ph.sinh_dr * ph.sinh_dr;
        unsigned close = 0;
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
            for (int j = i + 1; j < N; ++j) {
                const double pp2 = pt2[i] * pt2[j];                      // (pT_i pT_j)^2
                const double sh = p(i, 3) * p(j, 0) - p(j, 3) * p(i, 0);   // sinh(d eta) pT_i pT_j
                const double dot = p(i, 1) * p(j, 1) + p(i, 2) * p(j, 2);  // cos(d phi) pT_i pT_j
                const bool far = lt_nonneg(sdr2 * pp2, sh * sh) | lt_scaled(dot, ph.cos_dr, pp2);
                close |= (far ? 0u : 1u) << pair_index<N>(i, j);
            }
        if (!ok) close = 0;
        while (close) {
            int q = __ffs(close) - 1, i = 0;
            close &= close - 1;
            while (q >= N - 1 - i) q -= N - 1 - i++;
            const int j = i + 1 + q;
            const double xi = p(i, 1), yi = p(i, 2), zi = p(i, 3);
            const double xj = p(j, 1), yj = p(j, 2), zj = p(j, 3);
            const double pp2 = (xi * xi + yi * yi) * (xj * xj + yj * yj);
            const double sh = zi * p(j, 0) - zj * p(i, 0);
            const double dot = xi * xj + yi * yj;
            // a close pair: |d eta|, d phi <= R.  With s = |sinh d eta| and
            // t = tan d phi (dot > 0 here when R < pi/2),
            //   s^2 (1 - s^2/6)^2 <= d eta^2 <= s^2,
            //   t^2 (1 - t^2/3)^2 <= d phi^2 <= t^2
            // (asinh and atan lie between their first two Taylor terms and
            // their first), which settles all but the pairs within about 1 %
            // of R; those take asinh and atan2.
            const double cr = xi * yj - yi * xj;
            const double R2 = ph.dr_min * ph.dr_min;
            bool exact = !(dot > 0);
            if (!exact) {
                const double s2 = sh * sh / pp2, t2 = cr * cr / (dot * dot);
                const double a = 1.0 - s2 * (1.0 / 6.0), b = 1.0 - t2 * (1.0 / 3.0);
                const double hi = s2 + t2, lo = s2 * a * a + t2 * b * b;
                if (lo > R2 * (1.0 + 1e-12)) {
                    // Delta R > R: the pair passes
                } else if (hi < R2 * (1.0 - 1e-12)) {
                    ok = false;
                } else {
                    exact = true;
                }
            }
            if (exact) {   // rare
                const double ptt = sqrt(pp2);
                const double deta = asinh(sh / ptt);
                const double dphi = atan2(fabs(cr), dot);
                ok = ok && deta * deta + dphi * dphi > R2;
            }
            if (!ok) close = 0;
        }
    }
    return ok ? 1 : 0;
}

// FP32 prefilter of the cut decisions.  Each test of pass_cuts is decided in
// FP32 when the FP32 value lies clearly on one side of the boundary, and the
// point falls back to the FP64 pass_cuts otherwise, so every decision equals
// the FP64 one.  Error bounds (u = 2^-24): the components convert with
// relative error u; a product or sum of two such terms carries at most a
// few u relative to the magnitudes involved.  Margins are 64 u relative for
// the single-photon tests (no cancellation) and 32 u times the sum of the
// term magnitudes for the pair quantities sinh(d eta) pT pT and
// cos(d phi) pT pT, which cancel.  Only the rare close pairs (which need
// the exact Delta R) and near-boundary tests reach FP64.
struct Tri {   // a decision: certain (true / false) or undecided
    bool ok, sure;
};

// v < a w with w = sqrt(w2) >= 0, from FP32 values v2 = v^2, r2 = a^2 w2
// carrying relative error <= rel, and exact signs of v and a.
__device__ __forceinline__ Tri lt_scaled_f(bool vneg, bool apos, float v2, float r2, float rel) {
    const bool lt = v2 < r2 * (1.0f - rel), gt = v2 > r2 * (1.0f + rel);
    if (apos) return vneg ? Tri{true, true} : Tri{lt, lt || gt};
    return vneg ? Tri{gt, lt || gt} : Tri{false, true};
}

template <int N>
__device__ __forceinline__ int pass_cuts_fast(const MomView& p, double ey, double iey, const Physics& ph) {
    constexpr float kU = 5.9604645e-8f;   // 2^-24
    const double shy = 0.5 * (ey - iey), chy = 0.5 * (ey + iey);
    const double s_hi = ph.sinh_eta * chy - ph.cosh_eta * shy;    // sinh(E - y)
    const double s_lo = -ph.sinh_eta * chy - ph.cosh_eta * shy;   // sinh(-E - y)
    const float shi_f = f32_rn(s_hi), slo_f = f32_rn(s_lo);
    const float shi2 = shi_f * shi_f, slo2 = slo_f * slo_f;
    const float ptmin2 = f32_rn(ph.pt_min * ph.pt_min);
    float x[N], y[N], z[N], e[N], pt2[N];
    bool ok = true, sure = true;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        e[i] = f32_rn(p(i, 0));
        x[i] = f32_rn(p(i, 1));
        y[i] = f32_rn(p(i, 2));
        z[i] = f32_rn(p(i, 3));
        pt2[i] = x[i] * x[i] + y[i] * y[i];
        const bool gt = pt2[i] > ptmin2 * (1.0f + 64.0f * kU), le = pt2[i] < ptmin2 * (1.0f - 64.0f * kU);
        sure = sure && (gt || le);
        ok = ok && gt;
        const float z2 = z[i] * z[i];
        const Tri hi = lt_scaled_f(z[i] < 0.0f, shi_f >= 0.0f, z2, shi2 * pt2[i], 64.0f * kU);
        const Tri lo = lt_scaled_f(z[i] > 0.0f, -slo_f >= 0.0f, z2, slo2 * pt2[i], 64.0f * kU);
        sure = sure && hi.sure && lo.sure;
        ok = ok && hi.ok && lo.ok;
    }
    bool close = false;
    if (ph.dr_min > 0) {
        const float sdr2 = f32_rn(ph.sinh_dr * ph.sinh_dr), cdr = f32_rn(ph.cos_dr);
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
            for (int j = i + 1; j < N; ++j) {
                const float pp2 = pt2[i] * pt2[j];
                const float sh = z[i] * e[j] - z[j] * e[i];
                const float esh = 32.0f * kU * (fabsf(z[i] * e[j]) + fabsf(z[j] * e[i]));
                const float dot = x[i] * x[j] + y[i] * y[j];
                const float edot = 32.0f * kU * (fabsf(x[i] * x[j]) + fabsf(y[i] * y[j]));
                const float ash = fabsf(sh);
                // far in eta: sh^2 > sdr2 pp2, certain if (|sh| - esh)^2 beats it
                const float T = sdr2 * pp2;
                const bool eta_far = ash > esh && (ash - esh) * (ash - esh) > T * (1.0f + 64.0f * kU);
                const bool eta_near = (ash + esh) * (ash + esh) < T * (1.0f - 64.0f * kU);
                // far in phi: dot < cos_dr pT pT
                const float c = cdr * sqrtf(pp2);
                const float ec = 64.0f * kU * fabsf(c);
                const bool phi_far = dot + edot < c - ec;
                const bool phi_near = dot - edot > c + ec;
                const bool far = eta_far || phi_far;
                sure = sure && (far || (eta_near && phi_near));
                close = close || (!far && eta_near && phi_near);
            }
    }
    // undecided tests, and the close pairs (which need the exact Delta R),
    // go to the FP64 decision
    if (!sure || (ok && close)) return pass_cuts<N>(p, ey, iey, ph);
    return ok ? 1 : 0;
}

// Event i of stream `seed` from its sampler draws d: sqrt(s-hat), RAMBO
// momenta into v, cut decision.
template <int N>
__device__ __forceinline__ void generate_from(const PointRng& rng, const SampleDraw& d, const SamplerArgs& S,
                                              const Physics& ph, const MomView& v, EventInfo& ev) {
    sample_finish(S, d, ev);
    rambo<N>(rng, ev.rs, v);
    // the FP32 prefilter keeps 5n floats per photon set live in the producer
    // threads: a gain up to n = 3 (+22 % at n = 2 on GB300), a loss above
    // (at n = 4 1 % slower even with 124 registers a producer thread)
    if constexpr (N <= 3) ev.mask = ev.ok ? pass_cuts_fast<N>(v, ev.ey, ev.iey, ph) : 0;
    else ev.mask = ev.ok ? pass_cuts<N>(v, ev.ey, ev.iey, ph) : 0;
}

template <int N>
__device__ __forceinline__ void generate_event(uint64_t seed, uint64_t i, const SamplerArgs& S, const Physics& ph,
                                               const MomView& v, EventInfo& ev) {
    const PointRng rng(seed, i);
    generate_from<N>(rng, sample_draw(S, rng), S, ph, v, ev);
}

// Flat phase-space weight Phi_n(s) of eq. (4).
template <int N>
__device__ __forceinline__ double phase_space_weight(double s) {
    double sn2 = 1;
    for (int a = 2; a < N; ++a) sn2 *= s;
    return phase_space_const(N) * sn2;
}

// Propagator denominators t_T of the record, in FP64, from photon momenta p
// and p2 = E2 (1, 0, 0, -1), times `is` if SCALE (momenta in GeV, is =
// 1/s-hat; without SCALE the momenta are already divided by sqrt(s-hat)).
// For n <= 5 they are sums of the Lorentz invariants
//   t_T = sum_{i in T} d_i + sum_{i<j in T} s_ij,
//   d_i = k_i^2 - 2 k_i.p2,  s_ij = 2 k_i.k_j,
// built up over the sets in increasing order in registers: with h the
// highest photon of T and U = T - {h},
//   t_T = t_U + e_h(U),  e_h(U) = d_h + sum_{j in U} s_jh = e_h(U - {l}) + s_lh
// (l the lowest photon of U): two additions per set.  Larger n: FP64
// records use set_denominator, FP32 records keep the invariants
// (rec_invariant).
template <class R, int N, bool SCALE>
__device__ __forceinline__ void fill_denominators(const MomView& p, double E2, double is, bool massless,
                                                  PointRec<R, N>& rec) {
    static_assert(N <= 5, "n >= 6 forms its denominators set by set (set_denominator)");
    {
        double d[N], sij[N * (N - 1) / 2 > 0 ? N * (N - 1) / 2 : 1];
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const double e = p(i, 0), x = p(i, 1), y = p(i, 2), z = p(i, 3);
            d[i] = massless ? -(2.0 * E2 * (e + z)) : (e * e - x * x - y * y - z * z) - 2.0 * E2 * (e + z);
#pragma unroll
            for (int j = i + 1; j < N; ++j)
                sij[pair_index<N>(i, j)] = 2.0 * (e * p(j, 0) - x * p(j, 1) - y * p(j, 2) - z * p(j, 3));
        }
        double t[1 << (N - 1)];   // t_U for the sets U below the current highest photon
        double e[1 << (N - 1)];   // e_h(U)
#pragma unroll
        for (int h = 0; h < N; ++h) {
            e[0] = d[h];
#pragma unroll
            for (int U = 1; U < (1 << h); ++U) {
                const int l = __popc((U & -U) - 1);
                e[U] = e[U & (U - 1)] + sij[pair_index<N>(l, h)];
            }
#pragma unroll
            for (int U = 0; U < (1 << h); ++U) {
                const int T = U | (1 << h);
                if (T == (1 << N) - 1) continue;
                const double tt = U ? t[U] + e[U] : e[0];
                rec.t[T] = rec_value<R>(SCALE ? tt * is : tt);
                if (h < N - 1) t[T] = tt;
            }
        }
    }
}

// One denominator of an FP64 record for n >= 6 (one thread per set keeps
// every lane of the FP64 pipe busy): t_T = (sum_{i in T} k_i - p2)^2 by
// components, times `is` if SCALE.  Callers run it over (record, set) pairs
// after the records are built (denominators_parallel).
template <class R, int N, bool SCALE>
__device__ __forceinline__ R set_denominator(const MomView& p, double E2, double is, unsigned T) {
    double q0 = -E2, q1 = 0.0, q2 = 0.0, q3 = E2;
#pragma unroll 1
    for (int i = 0; i < N; ++i)
        if (T >> i & 1) {
            q0 += p(i, 0);
            q1 += p(i, 1);
            q2 += p(i, 2);
            q3 += p(i, 3);
        }
    const double tt = q0 * q0 - q1 * q1 - q2 * q2 - q3 * q3;
    return rec_value<R>(SCALE ? tt * is : tt);
}

// Photon sets as bitmasks: C(n, k), and the rank of S among the sets of its
// size in numeric order (numeric order of bitmasks is colexicographic order,
// so rank(S) = sum over the set bits b_1 < b_2 < ... of C(b_m, m)).
__host__ __device__ constexpr int set_binom(int n, int k) {
    if (k < 0 || k > n) return 0;
    int r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}
// offset of the size-k sets in a list ordered by size, then numerically
__host__ __device__ constexpr int set_level_offset(int n, int k) {
    int o = 0;
    for (int j = 0; j < k; ++j) o += set_binom(n, j);
    return o;
}
template <int N>
__device__ __forceinline__ int set_rank(unsigned S) {
    int r = 0, m = 0;
#pragma unroll
    for (int b = 0; b < N; ++b)
        if (S >> b & 1) r += set_binom(b, ++m);
    return r;
}
// list[offset(|S|) + rank(S)] = S for every S < 2^N (and rank[S] = rank(S)
// if rank != NULL), by threads lid = 0 .. nthr-1.
template <int N>
__device__ __forceinline__ void build_set_list(unsigned char* list, unsigned char* rank, int lid, int nthr) {
    for (int S = lid; S < (1 << N); S += nthr) {
        const int r = set_rank<N>((unsigned)S);
        list[set_level_offset(N, __popc(S)) + r] = (unsigned char)S;
        if (rank) rank[S] = (unsigned char)r;
    }
}

// float -> double by integer operations on the bit pattern (exact; f32_rn
// leaves no subnormals, so only zero needs its own case).
__device__ __forceinline__ double f64_of_f32(float f) {
    const unsigned int u = __float_as_uint(f);
    const unsigned int e = (u >> 23) & 0xFFu;
    const unsigned int hi = e == 0u ? (u & 0x80000000u) : (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7FFFFFu) >> 3);
    return __hiloint2double((int)hi, (int)(e == 0u ? 0u : u << 29));
}

// Invariant q of a record from FP64 momenta p, p1 = E1 (1, 0, 0, 1) and
// p2 = E2 (1, 0, 0, -1): q < N: d_q; N <= q < N + N(N-1)/2: s_ij for
// q = N + pair_index(i, j); after them d'_i; times `is` if SCALE.
template <int N, bool SCALE>
__device__ __forceinline__ double rec_invariant(const MomView& p, double E1, double E2, double is, bool massless,
                                                int q) {
    constexpr int NP = N * (N - 1) / 2;
    double v;
    if (q < N || q >= N + NP) {
        const bool one = q >= N + NP;   // d'_i: against p1
        const int i = one ? q - N - NP : q;
        const double e = p(i, 0), x = p(i, 1), y = p(i, 2), z = p(i, 3);
        const double lin = one ? 2.0 * E1 * (e - z) : 2.0 * E2 * (e + z);
        v = massless ? -lin : (e * e - x * x - y * y - z * z) - lin;
    } else {
        int i = 0, r = q - N;
        while (r >= N - 1 - i) {
            r -= N - 1 - i;
            ++i;
        }
        const int j = i + 1 + r;
        v = 2.0 * (p(i, 0) * p(j, 0) - p(i, 1) * p(j, 1) - p(i, 2) * p(j, 2) - p(i, 3) * p(j, 3));
    }
    return SCALE ? v * is : v;
}

// v as hi + lo: hi = v rounded to float, lo = the rest rounded to float
// (|v - hi - lo| <= 2^-48 |v| roughly).
__device__ __forceinline__ float2 split_ff(double v) {
    const float hi = f32_rn(v);
    return make_float2(hi, f32_rn(v - f64_of_f32(hi)));
}

// t_T of a record that holds invariants: their float-float sum over the
// smaller of T and its complement S (the d_i over T, or the d'_i over S,
// then the s_ij, i < j, by increasing i then j), each term added with an
// error-free two-sum into (S, E); rounded once to float.
template <int N>
__device__ __forceinline__ float rec_denominator(const float2* inv, unsigned T) {
    constexpr int NP = N * (N - 1) / 2;
    const bool comp = __popc(T) > N / 2;
    const unsigned U = comp ? ((1u << N) - 1) & ~T : T;
    const float2* lin = inv + (comp ? N + NP : 0);
    float S = 0.0f, E = 0.0f;
    auto add = [&](const float2 x) {
        const float s = S + x.x;
        const float bb = s - S;
        const float e = (S - (s - bb)) + (x.x - bb);
        S = s;
        E += e + x.y;
    };
    for (unsigned a = U; a; a &= a - 1) add(lin[__ffs(a) - 1]);
    for (unsigned a = U; a; a &= a - 1) {
        const int i = __ffs(a) - 1;
        for (unsigned b = a & (a - 1); b; b &= b - 1) add(inv[N + pair_index<N>(i, __ffs(b) - 1)]);
    }
    return S + E;
}

// Record of a point that passed the cuts, from its photon momenta (GeV) and
// irs = 1/sqrt(s-hat): momenta / sqrt(s-hat), denominators, normalisations,
// the factors to |M|^2 and to the event weight, valid = mask = 1.  The
// momenta are divided by sqrt(s-hat) in place, and the denominators formed
// from the scaled values.  (The caller sets idx and hsel.)
template <class R, int N>
__device__ __forceinline__ void pass_to_rec(const MomView& v, double irs, const Physics& ph, PointRec<R, N>& rec) {
    const double is = irs * irs;
#pragma unroll 1
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const double k = v(a, m) * irs;
            v(a, m) = k;
            rec.k[a][m] = rec_value<R>(k);
        }
    if constexpr (N <= 5) fill_denominators<R, N, false>(v, 0.5, 1.0, true, rec);   // n >= 6: denominators_parallel
    rec.e1 = R(0.5);
    rec.e2 = R(0.5);
    rec.n1 = R(1);
    rec.n2 = R(1);
    double sp = 1;  // s^(2-n)
    for (int a = 2; a < N; ++a) sp *= is;
    rec.fac = ph.cpl * sp;
    rec.wfac = ph.wconst * is;   // w = wfac * (scaled |M|^2 sum)
    rec.valid = 1;
    rec.mask = 1;
}

}  // namespace heget
