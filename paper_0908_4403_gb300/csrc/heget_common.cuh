// heget_common.cuh -- shared device types for the GB300 HEGET hot path:
// Philox4x32-10, the prefix-tree index tables, small complex helpers and
// double-double (TwoSum) accumulation.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "heget.h"

namespace heget {

constexpr int kMaxN = 8;
constexpr int kMinN = 2;

// ---------------------------------------------------------------------------
// Prefix-tree index tables.
//
// The ordering tree attaches photons to the ubar end one at a time.  A node is
// an ordered prefix; the off-shell current after attaching photon j to a
// prefix with photon set S depends on (j, T = S u {j}) only through the step
// matrix M(j, T) = eps*_j.sigma  (q_T.sigmabar)/q_T^2 with q_T = sum_{i in T}
// k_i - p2.  Steps exist for 1 <= |T| <= n-1; each (T, j in T) pair gets a
// compact index, ordered by |T|, then T, then j (so the n(n-1) pairs with
// |T| = n-1 come last, and a table that needs only the smaller sets stops
// before them):
//   pair[idx]        = T | (j << 8)
//   child[S * n + j] = idx of (S | 1<<j, j)   for j not in S, |S| <= n-2.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int num_pairs(int n) { return n * (1 << (n - 1)) - n; }
__host__ __device__ constexpr int pair_offset(int n) {
    int o = 0;
    for (int m = kMinN; m < n; ++m) o += num_pairs(m);
    return o;
}
__host__ __device__ constexpr int child_offset(int n) {
    int o = 0;
    for (int m = kMinN; m < n; ++m) o += (1 << m) * m;
    return o;
}
constexpr int kPairTotal = pair_offset(kMaxN + 1);
constexpr int kChildTotal = child_offset(kMaxN + 1);

struct TreeTables {
    uint16_t pair[kPairTotal];
    uint16_t child[kChildTotal];
};

__host__ __device__ constexpr TreeTables make_tree_tables() {
    TreeTables t{};
    for (int n = kMinN; n <= kMaxN; ++n) {
        int po = pair_offset(n), co = child_offset(n);
        for (int i = 0; i < (1 << n) * n; ++i) t.child[co + i] = 0xFFFF;
        int idx = 0;
        for (int size = 1; size < n; ++size)
            for (int T = 1; T < (1 << n) - 1; ++T) {
                int pop = 0;
                for (int b = 0; b < n; ++b) pop += (T >> b) & 1;
                if (pop != size) continue;
                for (int j = 0; j < n; ++j)
                    if (T >> j & 1) {
                        t.pair[po + idx] = (uint16_t)(T | (j << 8));
                        t.child[co + (T & ~(1 << j)) * n + j] = (uint16_t)idx;
                        ++idx;
                    }
            }
    }
    return t;
}

// one copy per translation unit, built at compile time
static __constant__ const TreeTables c_tables = make_tree_tables();

// The last three levels of the walk below a node whose set T leaves three
// photons a < b < c: the step indices of attaching a, b and c to T, and the
// ordered pair slots a (n - 1) + b - [b > a] of the pairs left after each
// attach, (b, c), (c, b), (a, c), (c, a), (a, b), (b, a).  Indexed by T for
// n = 5..8 (entries of other sets unused); 32 bytes, so that a warp reads an
// entry in two 16-byte constant loads.
struct alignas(16) Bottom3 {
    uint16_t st[3];
    uint16_t pc[6];
    uint16_t pad[7];
};
__host__ __device__ constexpr int bottom_offset(int n) {
    int o = 0;
    for (int m = 5; m < n; ++m) o += 1 << m;
    return o;
}
constexpr int kBottomTotal = bottom_offset(kMaxN + 1);

struct BottomTables {
    Bottom3 e[kBottomTotal];
};

__host__ __device__ constexpr BottomTables make_bottom_tables() {
    BottomTables b{};
    const TreeTables t = make_tree_tables();
    for (int n = 5; n <= kMaxN; ++n) {
        const int co = child_offset(n);
        for (int T = 0; T < (1 << n); ++T) {
            int pop = 0;
            for (int i = 0; i < n; ++i) pop += (T >> i) & 1;
            if (pop != n - 3) continue;
            int r[3] = {0, 0, 0}, k = 0;
            for (int i = 0; i < n; ++i)
                if (!((T >> i) & 1)) r[k++] = i;
            Bottom3& e = b.e[bottom_offset(n) + T];
            for (int x = 0; x < 3; ++x) e.st[x] = t.child[co + T * n + r[x]];
            const int pairs[3][2] = {{r[1], r[2]}, {r[0], r[2]}, {r[0], r[1]}};
            for (int x = 0; x < 3; ++x) {
                const int y = pairs[x][0], z = pairs[x][1];
                e.pc[2 * x] = (uint16_t)(y * (n - 1) + z - (z > y));
                e.pc[2 * x + 1] = (uint16_t)(z * (n - 1) + y - (y > z));
            }
        }
    }
    return b;
}
static __constant__ const BottomTables c_bottom = make_bottom_tables();

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from the
// published round function: two 32x32->64 multiplies per round, Weyl key
// schedule, 10 rounds.
// ---------------------------------------------------------------------------
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Uniform in (0,1) from two Philox words: m = ((hi << 32) | lo) >> 12 (52
// bits), u = (m + 1/2) 2^-52.  1 + m 2^-52 is built from bits and
// (1 - 2^-53) subtracted exactly (Sterbenz), so u is exact.
__device__ __forceinline__ double u01_from_words(uint32_t lo, uint32_t hi) {
    const uint64_t m = ((((uint64_t)hi) << 32) | lo) >> 12;
    return __longlong_as_double((long long)(0x3FF0000000000000ull | m)) -
           0x1.fffffffffffffp-1;
}

// Random stream of one phase-space point: counter (i lo, i hi, draw/2, tag),
// key = seed.  One Philox call yields draws 2b and 2b+1.
constexpr uint32_t kStreamSqrtS = 0u;
constexpr uint32_t kStreamRambo = 1u;
constexpr uint32_t kStreamHelicity = 2u;   // helicity sampling: draw 0

struct PointRng {
    uint32_t k0, k1, ilo, ihi;
    __device__ __forceinline__ PointRng(uint64_t seed, uint64_t i)
        : k0((uint32_t)seed), k1((uint32_t)(seed >> 32)), ilo((uint32_t)i),
          ihi((uint32_t)(i >> 32)) {}
    // the random words of block b of stream `tag`: draw 2b from (x, y), 2b+1 from (z, w)
    __device__ __forceinline__ U4 words(uint32_t tag, uint32_t b) const {
        return philox4x32_10(U4{ilo, ihi, b, tag}, k0, k1);
    }
    // both draws of block b of stream `tag`
    __device__ __forceinline__ void pair(uint32_t tag, uint32_t b, double& u0,
                                         double& u1) const {
        const U4 w = words(tag, b);
        u0 = u01_from_words(w.x, w.y);
        u1 = u01_from_words(w.z, w.w);
    }
};

// ---------------------------------------------------------------------------
// Double-double accumulation (TwoSum of Knuth / Moller; pair addition with
// two TwoSums and renormalisation, Joldes-Muller-Popescu 2017 "AccurateDWPlusDW").
// ---------------------------------------------------------------------------
struct DD { double hi, lo; };

__host__ __device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
    s = a + b;
    const double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__host__ __device__ __forceinline__ DD dd_add_d(DD a, double b) {
    double s, e;
    two_sum(a.hi, b, s, e);
    e += a.lo;
    double h, l;
    two_sum(s, e, h, l);
    return DD{h, l};
}

__host__ __device__ __forceinline__ DD dd_add(DD a, DD b) {
    double s, e, t, f;
    two_sum(a.hi, b.hi, s, e);
    two_sum(a.lo, b.lo, t, f);
    e += t;
    double h, l;
    two_sum(s, e, h, l);
    l += f;
    double h2, l2;
    two_sum(h, l, h2, l2);
    return DD{h2, l2};
}

// Per-block Monte Carlo partial: sums of w and w^2, counters.
struct Partial {
    DD sw, sw2;
    long long npass, ntotal, ntries, nesc;
};

__host__ __device__ __forceinline__ Partial partial_add(const Partial& a, const Partial& b) {
    Partial r;
    r.sw = dd_add(a.sw, b.sw);
    r.sw2 = dd_add(a.sw2, b.sw2);
    r.npass = a.npass + b.npass;
    r.ntotal = a.ntotal + b.ntotal;
    r.ntries = a.ntries + b.ntries;
    r.nesc = a.nesc + b.nesc;
    return r;
}

// ---------------------------------------------------------------------------
// Kernel arguments
// ---------------------------------------------------------------------------
// Physics constants of one launch (derived on the host from heget_params and n).
struct Physics {
    double alpha, q, pt_min, eta_max, dr_min;
    double cpl;                 // (4 pi alpha q^2)^n
    double wconst;              // cpl c_n / (24 n!) GeV^-2 -> fb (weight = wconst S / s)
    double sinh_eta, cosh_eta;  // sinh, cosh of eta_max
    double sinh_dr, cos_dr;     // sinh, cos of dr_min
    double esc_tau;             // FP32 -> FP64 escalation: relative error bound that triggers it (0 = off)
    int alg;                    // ordering sum: 0 prefix tree, 1 subset recursion
    int hel_sample;             // 1: one sampled helicity per point (Sec. 3), weighted 2^(n+2)
};

struct SamplerArgs {
    int kind;
    int max_tries;
    double sqrt_s, lo, hi, e_beam, floor;
    // toy PDF: the floor test sqrt(s-hat) > floor in terms of the uniforms,
    // u_a u_b > floor / (2 e_beam), settled in FP32 outside [band_lo, band_hi]
    float band_lo, band_hi;
};

// Launch shape of the amplitude kernels (chosen per (n, precision)).
struct AmpShape {
    int block;     // threads per block (multiple of 2^n and of 32)
    int tile;      // points per block tile (multiple of block / 2^n)
    int grid;      // blocks (grid-stride over tiles)
};

}  // namespace heget
