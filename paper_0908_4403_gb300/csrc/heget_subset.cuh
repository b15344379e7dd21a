// heget_subset.cuh -- algorithm ids and the FP32 condition bound of the
// ordering sum (for FP32 -> FP64 escalation).  The subset algorithm's
// amplitudes are in heget_meet.cuh.
#pragma once

#include "heget_meet.cuh"

namespace heget {

constexpr int kAlgTree = 0;
constexpr int kAlgSubset = 1;
constexpr int kAlgAny = -1;   // kernel template argument: Physics::alg decides at run time

// Largest C(n,k) 2^k over the levels k = 1 .. n-1 (bound rows per buffer).
__host__ __device__ constexpr int kappa_level_rows(int n) {
    int m = 0;
    for (int k = 1; k <= n - 1; ++k) {
        const int v = set_binom(n, k) << k;
        m = v > m ? v : m;
    }
    return m;
}

// Largest C(n,k) k 2 over the levels k = 2 .. n-1 (step-matrix norms per level).
__host__ __device__ constexpr int kappa_level_mats(int n) {
    int m = 2;
    for (int k = 2; k <= n - 1; ++k) {
        const int v = set_binom(n, k) * k * 2;
        m = v > m ? v : m;
    }
    return m;
}

// Points per round of the bound for a block of BLOCK threads.
__host__ __device__ constexpr int kappa_points(int n, int block) {
    const int p = n <= 2 ? block / 8 : n <= 4 ? block / 16 : n == 5 ? block / 32 : n == 6 ? block / 64
                                                                                 : n == 7 ? block / 128 : block / 256;
    return p > 0 ? p : 1;
}

template <class R, int N, int BLOCK>
struct KappaTables {
    static constexpr int P = kappa_points(N, BLOCK);
    static constexpr int NS = 1 << N;
    static constexpr int JR = kappa_level_rows(N);
    static constexpr int MR = kappa_level_mats(N);
    static constexpr size_t bytes = ((size_t)P * N + (size_t)P * NS) * sizeof(Row<R>)                  // PH, SD
                                    + (2 * (size_t)P * JR + (size_t)P * MR + (size_t)P * N * 2 +
                                       (size_t)P * NS) * sizeof(R)                                       // bounds
                                    + 2 * (size_t)NS + 16;                                               // rank, list
    Row<R>* PH;            // [P][N]
    Row<R>* SD;            // [P][2^N]
    R* JN[2];              // [P][JR]: norm bounds of the currents, level k in JN[k & 1]
    R* NM;                 // [P][MR]: norms of the level's step matrices
    R* CLN;                // [P][N][2]: norms of the closure columns
    R* B2;                 // [P][2^N]: weighted squared bounds
    unsigned char* RANK;   // [2^N]: rank of S among the sets of its size
    unsigned char* LIST;   // [2^N]: sets by size, then rank
    __device__ __forceinline__ explicit KappaTables(unsigned char* base) {
        PH = reinterpret_cast<Row<R>*>(base);
        SD = PH + (size_t)P * N;
        JN[0] = reinterpret_cast<R*>(SD + (size_t)P * NS);
        JN[1] = JN[0] + (size_t)P * JR;
        NM = JN[1] + (size_t)P * JR;
        CLN = NM + (size_t)P * MR;
        B2 = CLN + (size_t)P * N * 2;
        RANK = reinterpret_cast<unsigned char*>(B2 + (size_t)P * NS);
        LIST = RANK + NS;
    }
};

// |r| = |Re r0| + |Im r0| + |Re r1| + |Im r1| (the norm of the condition bound)
template <class R>
__device__ __forceinline__ R row_norm1(const Row<R>& r) {
    return fabs(r.ar) + fabs(r.ai) + fabs(r.br) + fabs(r.bi);
}

// lambda_S with the bit at position pos removed (the helicities of S \ i)
__device__ __forceinline__ int drop_bit(int lam, int pos) {
    return (lam & ((1 << pos) - 1)) | ((lam >> (pos + 1)) << pos);
}

// ---------------------------------------------------------------------------
// Condition bound of the ordering sum, for FP32 -> FP64 escalation.
//
// For each helicity h the sum A_h = sum_pi A_pi,h cancels when the orderings
// nearly cancel; its FP32 rounding error is about u32 times
// sum_pi |A_pi,h| (times a small factor), not u32 |A_h|.  The pass below
// bounds sum_pi |A_pi,h| from above without enumerating orderings: with the
// row norm |r| = |Re r0| + |Im r0| + |Re r1| + |Im r1| and, for a step
// matrix M with rows m0, m1, |M| = max(|m0|, |m1|), one step obeys
// |r . M| <= |r| |M|, so the currents' norms propagate over subsets like the
// currents themselves:
//   Jn(S) = sum_{i in S} Jn(S \ i) |M(i, S)|,   B = sum_i Jn(all \ i) |c_i|,
// with |c| = max(|c0|, |c1|) for a closure column.  Then
//   |sum_h w_h |A_h|^2 (FP32) - exact| <~ 2 u32 sqrt(sum w B^2) sqrt(sum w |A|^2),
// and a point whose relative error bound u32 sqrt(kap2 / ssum) exceeds the
// context's threshold is recomputed in FP64.  The bound runs on the same
// records as either algorithm; it stores kap2 = sum_h w_h B_h^2.
// ---------------------------------------------------------------------------
template <class R, int N, int BLOCK, int BAR, int K>
__device__ __forceinline__ void kappa_level(const KappaTables<R, N, BLOCK>& tb, int cnt) {
    using ST = KappaTables<R, N, BLOCK>;
    constexpr int P = ST::P, NS = ST::NS, JR = ST::JR, MR = ST::MR;
    constexpr int CK = set_binom(N, K);
    constexpr int LOFF = set_level_offset(N, K);
    const R* Jp = tb.JN[(K - 1) & 1];
    R* Jc = tb.JN[K & 1];
    const int tid = threadIdx.x;
    for (int it = tid; it < P * CK * K * 2; it += BLOCK) {
        const int lam = it & 1;
        int q = it >> 1;
        const int pos = q % K;
        q /= K;
        const int rS = q % CK, p = q / CK;
        if (p >= cnt) continue;
        const unsigned S = tb.LIST[LOFF + rS];
        unsigned s = S;
        for (int u = 0; u < pos; ++u) s &= s - 1;
        const int i = __ffs(s) - 1;
        const StepMat<R> sm = step_matrix<R>(tb.PH[p * N + i], tb.SD[p * NS + S], lam, false);
        tb.NM[(size_t)p * MR + (size_t)(rS * K + pos) * 2 + lam] = fmax(row_norm1(sm.m0), row_norm1(sm.m1));
    }
    group_sync<BAR, BLOCK>();
    for (int it = tid; it < (P * CK) << K; it += BLOCK) {
        const int lamS = it & ((1 << K) - 1);
        const int q = it >> K;
        const int rS = q % CK, p = q / CK;
        if (p >= cnt) continue;
        const unsigned S = tb.LIST[LOFF + rS];
        R acc = R(0);
        unsigned s = S;
#pragma unroll
        for (int pos = 0; pos < K; ++pos) {
            const int i = __ffs(s) - 1;
            s &= s - 1;
            acc += Jp[(size_t)p * JR + ((int)tb.RANK[S ^ (1u << i)] << (K - 1)) + drop_bit(lamS, pos)] *
                   tb.NM[(size_t)p * MR + (size_t)(rS * K + pos) * 2 + ((lamS >> pos) & 1)];
        }
        Jc[(size_t)p * JR + ((size_t)rS << K) + lamS] = acc;
    }
    group_sync<BAR, BLOCK>();
    if constexpr (K + 1 <= N - 1) kappa_level<R, N, BLOCK, BAR, K + 1>(tb, cnt);
}

// recs[p].kap2 for recs[0 .. cnt-1] (all valid), after either algorithm's
// amplitude rounds on the same shared memory.  A separate call, so that its
// registers do not add to the rounds'.  All threads must call it.
template <class R, int N, int BLOCK, int BAR = 0>
__device__ __noinline__ void kappa_rounds(unsigned char* table_smem, PointRec<R, N>* recs, int cnt,
                                          const uint32_t* mask) {
    using ST = KappaTables<R, N, BLOCK>;
    constexpr int P = ST::P, NS = ST::NS, JR = ST::JR;
    constexpr unsigned FULL = NS - 1;
    const ST tb(table_smem);
    const int tid = threadIdx.x;
    build_set_list<N>(tb.LIST, tb.RANK, tid, BLOCK);
    group_sync<BAR, BLOCK>();
    for (int base = 0; base < cnt; base += P) {
        const int rc = min(P, cnt - base);
        const PointRec<R, N>* rb = recs + base;
        setup_photons_and_sets<R, N, BLOCK, P>(tb.PH, tb.SD, rb, rc, tb.LIST);
        group_sync<BAR, BLOCK>();
        for (int it = tid; it < P * N * 2; it += BLOCK) {
            const int lam = it & 1;
            const int q = it >> 1;
            const int i = q % N, p = q / N;
            if (p >= rc) continue;
            const StepMat<R> sm = step_matrix<R>(tb.PH[p * N + i], tb.SD[p * NS + (1 << i)], lam, false);
            tb.JN[1][(size_t)p * JR + i * 2 + lam] = rb[p].n2 * row_norm1(sm.m1);
            tb.CLN[(p * N + i) * 2 + lam] = rb[p].n1 * fmax(fabs(sm.e00), fabs(sm.e10r) + fabs(sm.e10i));
        }
        group_sync<BAR, BLOCK>();
        if constexpr (N >= 3) kappa_level<R, N, BLOCK, BAR, 2>(tb, rc);
        const R* Jl = tb.JN[(N - 1) & 1];
        for (int it = tid; it < P * NS; it += BLOCK) {
            const int lam = it & (NS - 1), p = it >> N;
            if (p >= rc) continue;
            R b = R(0);
#pragma unroll
            for (int i = 0; i < N; ++i)
                b += Jl[(size_t)p * JR + ((int)tb.RANK[FULL ^ (1u << i)] << (N - 1)) + drop_bit(lam, i)] *
                     tb.CLN[(p * N + i) * 2 + ((lam >> i) & 1)];
            tb.B2[p * NS + lam] = b * b * R(sel_weight<N>(rb[p].hsel, (unsigned)lam, lane_weight<N>(mask, (unsigned)lam)));
        }
        group_sync<BAR, BLOCK>();
        for (int p = tid >> 5; p < rc; p += BLOCK / 32) {
            R v = R(0);
            for (int l = tid & 31; l < NS; l += 32) v += tb.B2[p * NS + l];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if ((tid & 31) == 0) recs[base + p].kap2 = v;
        }
        group_sync<BAR, BLOCK>();
    }
}

}  // namespace heget
