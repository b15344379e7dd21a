// heget_ps.cuh -- FP64 phase-space generation on the device: sqrt(s-hat)
// samplers, RAMBO flat massless n-body phase space (Sec. 2.1 eq. (4);
// Kleiss, Stirling, Ellis, CPC 40 (1986) 359), the photon cuts of Sec. 2.2
// eqs. (9)-(10), and the per-point record the amplitude kernels consume.
#pragma once

#include "heget_common.cuh"

namespace heget {

// Point record staged in shared memory between event generation (or input
// loading) and the amplitude rounds.  Momenta are divided by sqrt(s-hat) so
// that the FP32 chain works on O(1) numbers; the mass dimension 4 - 2n of
// |M|^2 is restored by `fac`.
template <int N>
struct alignas(16) PointRec {
    double k[N][4];   // photon momenta / sqrt(s-hat)
    double e1, e2;    // energies of p1 (+z) and p2 (-z) / sqrt(s-hat)
    double fac;       // (4 pi alpha Q^2)^n s-hat^(2-n)
    double wfac;      // event weight per unit |M|^2 sum (fb), 0 if masked
    int valid;        // 0: amplitude not evaluated (bad input / sampler failure)
    int mask;         // passes the cuts
    int tries;        // outer sampler attempts
    int pad;
};

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

// Toy-PDF momentum fraction: proposal x = u^2 (density ~ x^-1/2), accepted
// with probability (1-x)^3; one Philox block per try.  Returns -1 when the
// bound is hit.
__device__ __forceinline__ double toy_pdf_x(const PointRng& rng, uint32_t& blk, int max_tries) {
    for (int t = 0; t < max_tries; ++t) {
        double u, v;
        rng.pair(kStreamSqrtS, blk++, u, v);
        const double x = u * u;
        const double om = 1.0 - x;
        if (v < om * om * om) return x;
    }
    return -1.0;
}

// sqrt(s-hat), boost rapidity y and outer attempts for point i.
__device__ __forceinline__ void sample_sqrt_s(const SamplerArgs& S, const PointRng& rng,
                                              double& rs, double& y, int& tries, int& ok) {
    ok = 1;
    y = 0.0;
    tries = 1;
    if (S.kind == HEGET_SAMPLER_FIXED) {
        rs = S.sqrt_s;
        return;
    }
    if (S.kind == HEGET_SAMPLER_UNIFORM) {
        double u, unused;
        rng.pair(kStreamSqrtS, 0, u, unused);
        rs = S.lo + (S.hi - S.lo) * u;
        return;
    }
    uint32_t blk = 0;
    for (int t = 1; t <= S.max_tries; ++t) {
        const double x1 = toy_pdf_x(rng, blk, S.max_tries);
        const double x2 = x1 < 0 ? -1.0 : toy_pdf_x(rng, blk, S.max_tries);
        if (x1 < 0 || x2 < 0) break;
        const double r = 2.0 * S.e_beam * sqrt(x1 * x2);
        if (r > S.floor) {
            rs = r;
            y = 0.5 * log(x1 / x2);
            tries = t;
            return;
        }
    }
    ok = 0;
    rs = S.floor;
    tries = S.max_tries;
}

// RAMBO: n massless momenta with total (rs, 0, 0, 0).  Photon i uses draws
// 4i..4i+3 of the RAMBO stream: cos(theta) = 2 r0 - 1, phi = 2 pi r1,
// q0 = -ln(r2 r3); the isotropic q_i are boosted and scaled onto the total.
template <int N>
__device__ __forceinline__ void rambo(const PointRng& rng, double rs, double (&p)[N][4]) {
    double Q0 = 0, Q1 = 0, Q2 = 0, Q3 = 0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        double r0, r1, r2, r3;
        rng.pair(kStreamRambo, 2 * i, r0, r1);
        rng.pair(kStreamRambo, 2 * i + 1, r2, r3);
        const double c = 2.0 * r0 - 1.0;
        const double s = sqrt(1.0 - c * c);
        double sp, cp;
        sincospi(2.0 * r1, &sp, &cp);
        const double q0 = -log(r2 * r3);
        p[i][0] = q0;
        p[i][1] = q0 * s * cp;
        p[i][2] = q0 * s * sp;
        p[i][3] = q0 * c;
        Q0 += p[i][0];
        Q1 += p[i][1];
        Q2 += p[i][2];
        Q3 += p[i][3];
    }
    const double M = sqrt(Q0 * Q0 - Q1 * Q1 - Q2 * Q2 - Q3 * Q3);
    const double iM = 1.0 / M;
    const double b1 = -Q1 * iM, b2 = -Q2 * iM, b3 = -Q3 * iM;
    const double g = Q0 * iM;
    const double a = 1.0 / (1.0 + g);
    const double x = rs * iM;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const double bq = b1 * p[i][1] + b2 * p[i][2] + b3 * p[i][3];
        const double q0 = p[i][0];
        p[i][0] = x * (g * q0 + bq);
        p[i][1] = x * (p[i][1] + b1 * q0 + a * bq * b1);
        p[i][2] = x * (p[i][2] + b2 * q0 + a * bq * b2);
        p[i][3] = x * (p[i][3] + b3 * q0 + a * bq * b3);
    }
}

// Photon cuts, strict: pT > pt_min, |eta + y| < eta_max with
// eta = asinh(pz / pT), and Delta R = sqrt(Delta eta^2 + Delta phi^2) > dr_min
// for every pair (Delta phi folded into [0, pi]); dr_min <= 0 disables it.
template <int N>
__device__ __forceinline__ int pass_cuts(const double (&p)[N][4], double y, const Physics& ph) {
    double eta[N], phi[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const double pt = sqrt(p[i][1] * p[i][1] + p[i][2] * p[i][2]);
        if (!(pt > ph.pt_min)) return 0;
        eta[i] = asinh(p[i][3] / pt) + y;
        if (!(fabs(eta[i]) < ph.eta_max)) return 0;
        phi[i] = atan2(p[i][2], p[i][1]);
    }
    if (ph.dr_min > 0) {
        const double pi = 3.141592653589793238462643;
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
            for (int j = i + 1; j < N; ++j) {
                double dphi = fabs(phi[i] - phi[j]);
                if (dphi > pi) dphi = 2.0 * pi - dphi;
                const double deta = eta[i] - eta[j];
                if (!(sqrt(deta * deta + dphi * dphi) > ph.dr_min)) return 0;
            }
    }
    return 1;
}

// (4 pi alpha Q^2)^n
__device__ __forceinline__ double coupling_pow(const Physics& ph, int n) {
    const double g2 = 4.0 * 3.141592653589793238462643 * ph.alpha * ph.q * ph.q;
    double r = 1;
    for (int i = 0; i < n; ++i) r *= g2;
    return r;
}

// One generated event in GeV.
template <int N>
struct Event {
    double p[N][4];
    double rs, y;
    int tries, ok, mask;
};

template <int N>
__device__ __forceinline__ void generate_event(uint64_t seed, uint64_t i, const SamplerArgs& S,
                                               const Physics& ph, Event<N>& ev) {
    const PointRng rng(seed, i);
    sample_sqrt_s(S, rng, ev.rs, ev.y, ev.tries, ev.ok);
    rambo<N>(rng, ev.rs, ev.p);
    ev.mask = ev.ok ? pass_cuts<N>(ev.p, ev.y, ph) : 0;
}

// Flat phase-space weight Phi_n(s) of eq. (4).
template <int N>
__device__ __forceinline__ double phase_space_weight(double s) {
    double sn2 = 1;
    for (int a = 2; a < N; ++a) sn2 *= s;
    return phase_space_const(N) * sn2;
}

// Event -> point record.  Event weight per unit sum_h |M_h|^2 (Sec. 2.1
// eq. (2)): (1/2s)(1/4)(1/9) 3 (1/n!) Phi_n(s), GeV^-2 -> fb.
template <int N>
__device__ __forceinline__ void event_to_rec(const Event<N>& ev, const Physics& ph, PointRec<N>& rec) {
    const double s = ev.rs * ev.rs;
    const double irs = 1.0 / ev.rs;
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int m = 0; m < 4; ++m) rec.k[a][m] = ev.p[a][m] * irs;
    rec.e1 = 0.5;
    rec.e2 = 0.5;
    double sp = 1;  // s^(2-n)
    for (int a = 2; a < N; ++a) sp /= s;
    rec.fac = coupling_pow(ph, N) * sp;
    double nfact = 1;
    for (int a = 2; a <= N; ++a) nfact *= a;
    rec.wfac = ev.mask ? (1.0 / (2.0 * s)) * (1.0 / 12.0) / nfact * phase_space_weight<N>(s) * 0.3893793721e12
                       : 0.0;
    rec.valid = ev.ok;
    rec.mask = ev.mask;
    rec.tries = ev.tries;
    rec.pad = 0;
}

// GeV momenta of an event in the API layout [n+2][4]: p1, p2, k1..kn.
template <int N>
__device__ __forceinline__ void store_event_momenta(const Event<N>& ev, double* __restrict__ dst) {
    double2* o = reinterpret_cast<double2*>(dst);
    const double h = 0.5 * ev.rs;
    o[0] = make_double2(h, 0.0);
    o[1] = make_double2(0.0, h);
    o[2] = make_double2(h, 0.0);
    o[3] = make_double2(0.0, -h);
#pragma unroll
    for (int a = 0; a < N; ++a) {
        o[4 + 2 * a] = make_double2(ev.p[a][0], ev.p[a][1]);
        o[5 + 2 * a] = make_double2(ev.p[a][2], ev.p[a][3]);
    }
}

}  // namespace heget
