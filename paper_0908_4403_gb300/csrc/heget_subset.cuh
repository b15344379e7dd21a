// heget_subset.cuh -- the ordering sum as a recursion over photon subsets.
//
// The chain step of the prefix tree, r <- r . M(j, T) with
// M(j, T) = (eps*_j . sigma)(q_T . sigmabar)/q_T^2, depends on the prefix
// only through the SET T of photons attached so far (q_T is a sum over T).
// Summing all orderings of a set before extending it is therefore exact
// (distributivity, the Berends-Giele form of the same sum):
//     J(S) = sum_{i in S} J(S \ i) . M(i, S),       J({i}) = vbar(p2) . M(i, {i}),
//     A    = sum_i J(all \ i) . (eps*_i . sigma) u_R(p1),
// which is sum_k C(n,k) k steps per helicity configuration instead of the
// tree's sum_l n!/(n-l)! (1,016 vs 69,272 at n = 8).  J(S) depends only on the
// helicities of the photons in S, so each (S, lambda_S) is computed once for
// all helicity configurations that share it: sum_k C(n,k) k 2^k steps per
// point.  The result is the same sum of products as the tree and the paper's
// permutation loop (Sec. 2.1 eqs. (6)-(8), Appendix A.2), rounded in a
// different order.
//
// Work per round of P points, level by level (|S| = k = 2 .. n-1), with
// barriers between the phases:
//   (M) M(i, S)^lambda for every |S| = k, i in S, lambda (table MK),
//   (J) J(S, lambda_S) for every |S| = k and helicity assignment of S,
// then A(lambda) for all 2^n photon helicities, w_lambda |A|^2, and a fixed-
// order sum per point.  Levels k-1 and k live in two ping-pong buffers;
// subsets of one size are indexed by their rank in numeric order.
#pragma once

#include "heget_amp.cuh"

namespace heget {

constexpr int kAlgTree = 0;
constexpr int kAlgSubset = 1;
constexpr int kAlgAny = -1;   // kernel template argument: Physics::alg decides at run time

__host__ __device__ constexpr int binom(int n, int k) {
    if (k < 0 || k > n) return 0;
    int r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

// Largest C(n,k) 2^k over the stored levels k = 1 .. n-1 (rows per buffer).
__host__ __device__ constexpr int subset_level_rows(int n) {
    int m = 0;
    for (int k = 1; k <= n - 1; ++k) {
        const int v = binom(n, k) << k;
        m = v > m ? v : m;
    }
    return m;
}

// Largest C(n,k) k 2 over the levels k = 2 .. n-1 (step matrices per level).
__host__ __device__ constexpr int subset_level_mats(int n) {
    int m = 2;
    for (int k = 2; k <= n - 1; ++k) {
        const int v = binom(n, k) * k * 2;
        m = v > m ? v : m;
    }
    return m;
}

// Points per round for a block of BLOCK threads.
__host__ __device__ constexpr int subset_points(int n, int block) {
    return n <= 2 ? block / 8 : n <= 4 ? block / 16 : n == 5 ? block / 32 : n == 6 ? block / 64
                                                                                : n == 7 ? block / 128 : block / 256;
}

// Offset of the size-k subsets in the rank-ordered subset list.
__host__ __device__ constexpr int subset_list_offset(int n, int k) {
    int o = 0;
    for (int j = 0; j < k; ++j) o += binom(n, j);
    return o;
}

template <class R, int N, int BLOCK>
struct SubsetTables {
    static constexpr int P = subset_points(N, BLOCK) > 0 ? subset_points(N, BLOCK) : 1;
    static constexpr int NS = 1 << N;
    static constexpr int JR = subset_level_rows(N);
    static constexpr int MR = subset_level_mats(N);
    // bytes_core: what the recursion needs; bytes: with the condition-bound
    // arrays (FP32 escalation), which come last
    static constexpr size_t bytes_core = ((size_t)P * N + (size_t)P * NS + (size_t)P * N * 2   // PH, SD, CL
                                          + 2 * (size_t)P * JR                                   // J ping-pong
                                          + 2 * (size_t)P * MR) * sizeof(Row<R>)                 // M0K, M1K
                                         + (size_t)P * NS * sizeof(R)                            // weighted |A|^2
                                         + 2 * (size_t)NS + 16;                                  // rank, subset list
    static constexpr size_t bytes = bytes_core + (2 * (size_t)P * JR + (size_t)P * MR + (size_t)P * N * 2 +
                                                  (size_t)P * NS) * sizeof(R);                  // condition bound
    Row<R>* PH;    // [P][N]
    Row<R>* SD;    // [P][2^N]
    Row<R>* CL;    // [P][N][2]: closure columns (eps*_i . sigma) u_R, lambda minor
    Row<R>* J[2];  // [P][JR]: level k in J[k & 1], entry rank(S) 2^k + lambda_S
    Row<R>* M0K;   // [P][MR]: level's step matrices, entry (rank(S) k + pos) 2 + lambda
    Row<R>* M1K;
    R* A2;                 // [P][2^N]
    unsigned char* RANK;   // [2^N]: rank of S among the subsets of its size
    unsigned char* LIST;   // [2^N]: subsets by size, then rank
    R* JN[2];              // [P][JR]: norm bounds of the currents (condition bound)
    R* NM;                 // [P][MR]: norms of the level's step matrices
    R* CLN;                // [P][N][2]: norms of the closure columns
    R* B2;                 // [P][2^N]: weighted squared bounds
    __device__ __forceinline__ explicit SubsetTables(unsigned char* base) {
        PH = reinterpret_cast<Row<R>*>(base);
        SD = PH + (size_t)P * N;
        CL = SD + (size_t)P * NS;
        J[0] = CL + (size_t)P * N * 2;
        J[1] = J[0] + (size_t)P * JR;
        M0K = J[1] + (size_t)P * JR;
        M1K = M0K + (size_t)P * MR;
        A2 = reinterpret_cast<R*>(M1K + (size_t)P * MR);
        RANK = reinterpret_cast<unsigned char*>(A2 + (size_t)P * NS);
        LIST = RANK + NS;
        JN[0] = reinterpret_cast<R*>(base + bytes_core);
        JN[1] = JN[0] + (size_t)P * JR;
        NM = JN[1] + (size_t)P * JR;
        CLN = NM + (size_t)P * MR;
        B2 = CLN + (size_t)P * N * 2;
    }
};

// acc += r . M (rows m0, m1), all fused multiply-adds
template <class R>
__device__ __forceinline__ void row_times_acc(Row<R>& acc, const Row<R>& r, const Row<R>& m0, const Row<R>& m1) {
    acc.ar += r.ar * m0.ar - r.ai * m0.ai + r.br * m1.ar - r.bi * m1.ai;
    acc.ai += r.ar * m0.ai + r.ai * m0.ar + r.br * m1.ai + r.bi * m1.ar;
    acc.br += r.ar * m0.br - r.ai * m0.bi + r.br * m1.br - r.bi * m1.bi;
    acc.bi += r.ar * m0.bi + r.ai * m0.br + r.br * m1.bi + r.bi * m1.br;
}

// |r| = |Re r0| + |Im r0| + |Re r1| + |Im r1| (the norm of the condition bound)
template <class R>
__device__ __forceinline__ R row_norm1(const Row<R>& r) {
    return fabs(r.ar) + fabs(r.ai) + fabs(r.br) + fabs(r.bi);
}

// lambda_S with the bit at position pos removed (the helicities of S \ i)
__device__ __forceinline__ int drop_bit(int lam, int pos) {
    return (lam & ((1 << pos) - 1)) | ((lam >> (pos + 1)) << pos);
}

// One level k: step matrices, then currents.  All threads must call it.
template <class R, int N, int BLOCK, int BAR, int K>
__device__ __forceinline__ void subset_level(const SubsetTables<R, N, BLOCK>& tb, const PointRec<R, N>* rb, int cnt,
                                             bool kappa) {
    using ST = SubsetTables<R, N, BLOCK>;
    constexpr int P = ST::P, NS = ST::NS, JR = ST::JR, MR = ST::MR;
    constexpr int CK = binom(N, K);
    constexpr int LOFF = subset_list_offset(N, K);
    const int tid = threadIdx.x;
    // (M) M(i, S)^lambda for |S| = K
    for (int it = tid; it < P * CK * K * 2; it += BLOCK) {
        const int lam = it & 1;
        int q = it >> 1;
        const int pos = q % K;
        q /= K;
        const int rS = q % CK, p = q / CK;
        if (p >= cnt || !rb[p].valid) continue;
        const unsigned S = tb.LIST[LOFF + rS];
        unsigned s = S;
        for (int u = 0; u < pos; ++u) s &= s - 1;
        const int i = __ffs(s) - 1;
        const StepMat<R> sm = step_matrix<R>(tb.PH[p * N + i], tb.SD[p * NS + S], lam, false);
        const size_t o = (size_t)p * MR + (size_t)(rS * K + pos) * 2 + lam;
        st_row(tb.M0K + o, sm.m0);
        st_row(tb.M1K + o, sm.m1);
        if (kappa) tb.NM[o] = fmax(row_norm1(sm.m0), row_norm1(sm.m1));
    }
    group_sync<BAR, BLOCK>();
    // (J) J(S, lambda_S) = sum_{pos} J(S \ i_pos, lambda without bit pos) . M(i_pos, S)^{lambda bit pos}
    const Row<R>* Jp = tb.J[(K - 1) & 1];
    Row<R>* Jc = tb.J[K & 1];
    for (int it = tid; it < (P * CK) << K; it += BLOCK) {
        const int lamS = it & ((1 << K) - 1);
        const int q = it >> K;
        const int rS = q % CK, p = q / CK;
        if (p >= cnt || !rb[p].valid) continue;
        const unsigned S = tb.LIST[LOFF + rS];
        const Row<R>* jp = Jp + (size_t)p * JR;
        const size_t mo = (size_t)p * MR + (size_t)rS * K * 2;
        Row<R> acc{R(0), R(0), R(0), R(0)};
        R nacc = R(0);
        const R* jn = tb.JN[(K - 1) & 1] + (size_t)p * JR;
        unsigned s = S;
#pragma unroll
        for (int pos = 0; pos < K; ++pos) {
            const int i = __ffs(s) - 1;
            s &= s - 1;
            const int li = (lamS >> pos) & 1;
            const int src = ((int)tb.RANK[S ^ (1u << i)] << (K - 1)) + drop_bit(lamS, pos);
            const Row<R> r = ld_row(jp + src);
            const size_t e = mo + pos * 2 + li;
            row_times_acc(acc, r, ld_row(tb.M0K + e), ld_row(tb.M1K + e));
            if (kappa) nacc += jn[src] * tb.NM[e];
        }
        st_row(Jc + (size_t)p * JR + ((size_t)rS << K) + lamS, acc);
        if (kappa) tb.JN[K & 1][(size_t)p * JR + ((size_t)rS << K) + lamS] = nacc;
    }
    group_sync<BAR, BLOCK>();
    if constexpr (K + 1 <= N - 1) subset_level<R, N, BLOCK, BAR, K + 1>(tb, rb, cnt, kappa);
}

// Amplitude rounds over recs[0 .. cnt-1] by the subset recursion; the same
// contract as amplitude_rounds (recs[p].ssum = sum_h w_h |A_h|^2 in the
// scaled units of the records).  All threads must call it.
template <class R, int N, int BLOCK, int BAR = 0>
__device__ __forceinline__ void amplitude_rounds_subset(unsigned char* table_smem, PointRec<R, N>* recs, int cnt,
                                                        const uint32_t* mask, bool kappa = false) {
    using ST = SubsetTables<R, N, BLOCK>;
    constexpr int P = ST::P, NS = ST::NS, JR = ST::JR;
    constexpr unsigned FULL = NS - 1;
    const ST tb(table_smem);
    const int tid = threadIdx.x;
    // subset ranks and the rank-ordered list (numeric order within a size)
    for (int S = tid; S < NS; S += BLOCK) {
        const int k = __popc(S);
        int r = 0;
        for (int u = 0; u < S; ++u) r += __popc(u) == k;
        tb.RANK[S] = (unsigned char)r;
        int off = 0;
        for (int j = 0; j < k; ++j) off += binom(N, j);
        tb.LIST[off + r] = (unsigned char)S;
    }
    group_sync<BAR, BLOCK>();
    for (int base = 0; base < cnt; base += P) {
        const int rc = min(P, cnt - base);
        const PointRec<R, N>* rb = recs + base;
        setup_photons_and_sets<R, N, BLOCK, P>(tb.PH, tb.SD, rb, rc);
        group_sync<BAR, BLOCK>();
        // level 1: J({i}, lambda) = n2 (row 1 of M(i, {i})); closure columns
        for (int it = tid; it < P * N * 2; it += BLOCK) {
            const int lam = it & 1;
            const int q = it >> 1;
            const int i = q % N, p = q / N;
            if (p >= rc || !rb[p].valid) continue;
            const StepMat<R> sm = step_matrix<R>(tb.PH[p * N + i], tb.SD[p * NS + (1 << i)], lam, false);
            const R n1 = rb[p].n1, n2 = rb[p].n2;
            st_row(tb.J[1] + (size_t)p * JR + i * 2 + lam,
                   Row<R>{n2 * sm.m1.ar, n2 * sm.m1.ai, n2 * sm.m1.br, n2 * sm.m1.bi});
            st_row(tb.CL + (size_t)(p * N + i) * 2 + lam, Row<R>{n1 * sm.e00, R(0), n1 * sm.e10r, n1 * sm.e10i});
            if (kappa) {
                tb.JN[1][(size_t)p * JR + i * 2 + lam] = n2 * row_norm1(sm.m1);
                tb.CLN[(p * N + i) * 2 + lam] = n1 * fmax(fabs(sm.e00), fabs(sm.e10r) + fabs(sm.e10i));
            }
        }
        group_sync<BAR, BLOCK>();
        if constexpr (N >= 3) subset_level<R, N, BLOCK, BAR, 2>(tb, rb, rc, kappa);
        // closures: A(lambda) = sum_i J(all \ i, lambda without bit i) . CL(i)^{lambda_i}
        const Row<R>* Jl = tb.J[(N - 1) & 1];
        for (int it = tid; it < P * NS; it += BLOCK) {
            const int lam = it & (NS - 1), p = it >> N;
            if (p >= rc || !rb[p].valid) continue;
            R are = R(0), aim = R(0), b = R(0);
            const R* jn = tb.JN[(N - 1) & 1] + (size_t)p * JR;
#pragma unroll
            for (int i = 0; i < N; ++i) {
                const int src = ((int)tb.RANK[FULL ^ (1u << i)] << (N - 1)) + drop_bit(lam, i);
                const int c = (p * N + i) * 2 + ((lam >> i) & 1);
                close_row(ld_row(Jl + (size_t)p * JR + src), ld_row(tb.CL + (size_t)c), are, aim);
                if (kappa) b += jn[src] * tb.CLN[c];
            }
            const R wl = R(sel_weight<N>(rb[p].hsel, (unsigned)lam, lane_weight<N>(mask, (unsigned)lam)));
            tb.A2[p * NS + lam] = (are * are + aim * aim) * wl;
            if (kappa) tb.B2[p * NS + lam] = b * b * wl;
        }
        group_sync<BAR, BLOCK>();
        // fixed-order sum per point: one warp per point
        for (int p = tid >> 5; p < rc; p += BLOCK / 32) {
            R v = R(0), k2 = R(0);
            for (int l = tid & 31; l < NS; l += 32) {
                v += tb.A2[p * NS + l];
                if (kappa) k2 += tb.B2[p * NS + l];
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                v += __shfl_xor_sync(0xffffffffu, v, off);
                k2 += __shfl_xor_sync(0xffffffffu, k2, off);
            }
            if ((tid & 31) == 0) {
                recs[base + p].ssum = rb[p].valid ? v : R(0);
                if (kappa) recs[base + p].kap2 = k2;
            }
        }
        group_sync<BAR, BLOCK>();
    }
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
__device__ __forceinline__ void kappa_level(const SubsetTables<R, N, BLOCK>& tb, int cnt) {
    using ST = SubsetTables<R, N, BLOCK>;
    constexpr int P = ST::P, NS = ST::NS, JR = ST::JR, MR = ST::MR;
    constexpr int CK = binom(N, K);
    constexpr int LOFF = subset_list_offset(N, K);
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

// recs[p].kap2 for recs[0 .. cnt-1] (all valid), for the prefix tree (the
// subset recursion computes it alongside its currents).  A separate call, so
// that its registers do not add to the tree's.  All threads must call it.
template <class R, int N, int BLOCK, int BAR = 0>
__device__ __noinline__ void kappa_rounds(unsigned char* table_smem, PointRec<R, N>* recs, int cnt,
                                          const uint32_t* mask) {
    using ST = SubsetTables<R, N, BLOCK>;
    constexpr int P = ST::P, NS = ST::NS, JR = ST::JR;
    constexpr unsigned FULL = NS - 1;
    const ST tb(table_smem);
    const int tid = threadIdx.x;
    for (int S = tid; S < NS; S += BLOCK) {
        const int k = __popc(S);
        int r = 0;
        for (int u = 0; u < S; ++u) r += __popc(u) == k;
        tb.RANK[S] = (unsigned char)r;
        int off = 0;
        for (int j = 0; j < k; ++j) off += binom(N, j);
        tb.LIST[off + r] = (unsigned char)S;
    }
    group_sync<BAR, BLOCK>();
    for (int base = 0; base < cnt; base += P) {
        const int rc = min(P, cnt - base);
        const PointRec<R, N>* rb = recs + base;
        setup_photons_and_sets<R, N, BLOCK, P>(tb.PH, tb.SD, rb, rc);
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
