// heget_kernels.cuh -- the hot-path kernels:
//   amp2_kernel   : momenta [N][n+2][4] -> sum_h |M_h|^2          (heget_amp2)
//   xsec_kernel   : RNG -> sqrt(s-hat) -> RAMBO -> cuts -> |M|^2 -> weight ->
//                   double-double block partials, all in one pass  (heget_xsec)
// plus the launch-shape bookkeeping shared with the host code.
#pragma once

#include "heget_subset.cuh"

namespace heget {

__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

constexpr int kBatchThreads = 256;   // threads of the mixed-n batch kernel


// Tree shape per precision, photon count and threads of the rounds: 2^HB
// helicity configurations per lane and G groups (see TreeShape).  FP64 keeps
// one configuration per lane: its DFMA pipe, not instruction issue, is the
// limit.  FP32 from n = 6 runs pair units with four configurations per lane,
// which spreads each step's table loads and index work over four row
// updates, with one slot per warp (two points of 16 lanes at n = 6, one point
// of 32 lanes at n = 7) or per two warps (n = 8, 64 lanes); the blocks of the
// fused tile kernels share the units out evenly (15 over 5 slots at n = 6,
// 21 over 7 at n = 7, 28 over 4 at n = 8).
template <int HB_, int G_>
struct ShapeOf {
    static constexpr int HB = HB_, G = G_;
};
template <class R, int N, int BLOCK>
__host__ __device__ constexpr int tree_hb() {
    return sizeof(R) == sizeof(float) && N >= 6 ? 2 : 0;
}
template <class R, int N, int BLOCK>
__host__ __device__ constexpr int tree_groups() {
    return tree_hb<R, N, BLOCK>() == 0 ? 1 : N == 8 ? BLOCK / 64 : BLOCK / 32;
}
template <class R, int N, int BLOCK>
struct DefaultShape : ShapeOf<tree_hb<R, N, BLOCK>(), tree_groups<R, N, BLOCK>()> {};
// (HB, G) given, or the default of the block (HB < 0)
template <class R, int N, int BLOCK, int HB, int G>
struct ShapeSel : ShapeOf<HB < 0 ? tree_hb<R, N, BLOCK>() : HB, HB < 0 ? tree_groups<R, N, BLOCK>() : G> {};

// Tile-kernel shapes of the fused cross section that the autotuner searches
// (the analogue of the paper's register x block-size scan, Sec. 6.1): shape
// 0 is the default (the warp-specialised kernel where it applies, else the
// tile kernel of xsec_block threads with DefaultShape); the FP32 tree from
// n = 6 adds tile kernels of other block sizes, pair-unit slots and rows per
// lane (threads, HB, G), HB = 0 being one configuration per lane.
struct TileShape {
    int block, hb, g;
};
template <class R, int N, int ALG>
__host__ __device__ constexpr int num_tile_shapes() {
    return sizeof(R) == sizeof(float) && ALG == kAlgTree && N >= 6 ? 4 : 1;
}
// shape k = 1..3 of the FP32 tree at n = 6..8 (k = 0: the default)
__host__ __device__ constexpr TileShape tree_tile_shape(int n, int k) {
    return n == 6 ? (k == 1 ? TileShape{96, 2, 3} : k == 2 ? TileShape{320, 2, 5} : TileShape{256, 0, 1})
         : n == 7 ? (k == 1 ? TileShape{96, 2, 3} : k == 2 ? TileShape{128, 0, 1} : TileShape{256, 0, 1})
                  : (k == 1 ? TileShape{128, 2, 2} : k == 2 ? TileShape{448, 2, 7} : TileShape{256, 0, 1});
}
template <class R, int N, int ALG>
__host__ __device__ constexpr TileShape tile_shape(int k) {
    return tree_tile_shape(N, k);
}

// Shared-memory table layouts: the tree's (kAlgTree), the subset
// recursion's without (kAlgSubset) or with (kTabSubsetKappa) the arrays of
// the FP32 condition bound, or room for any of them (kAlgAny).
constexpr int kTabSubsetKappa = 2;
constexpr int kTabTreeKappa = 3;   // the tree's tables or the condition bound's

// Round-table bytes of layout TAB: the tree's default shape (at least those
// of one configuration per lane, which the gauge check uses, where the block
// holds whole points of that shape), the subset
// recursion's, or the larger of the two.
template <class R, int N, int BLOCK>
__host__ __device__ constexpr size_t ward_table_bytes() {
    if constexpr (BLOCK % (1 << N) == 0) return RoundTables<R, N, BLOCK>::bytes;
    else return 0;
}
template <class R, int N, int BLOCK, int TAB = kAlgAny, int HB = -1, int G = -1>
__host__ __device__ constexpr size_t table_bytes() {
    using SH = ShapeSel<R, N, BLOCK, HB, G>;
    constexpr size_t a = RoundTables<R, N, BLOCK, SH::HB, SH::G>::bytes, b = ward_table_bytes<R, N, BLOCK>();
    constexpr size_t c = MeetTables<R, N, BLOCK>::bytes, kb = KappaTables<R, N, BLOCK>::bytes;
    constexpr size_t ab = a > b ? a : b, ck = c > kb ? c : kb;
    return align16(TAB == kAlgTree ? ab : TAB == kAlgSubset ? c : TAB == kTabSubsetKappa ? ck
                 : TAB == kTabTreeKappa ? (ab > kb ? ab : kb) : (ab > ck ? ab : ck));
}

// The table layout of a kernel of algorithm ALG: the condition-bound pass
// (FP32 escalation) needs the subset tables' bound arrays, and the tree's
// (kappa_rounds) runs on the subset layout, so a tree kernel with it
// reserves both.
template <int ALG, bool KAPPA>
__host__ __device__ constexpr int table_alg() {
    return !KAPPA ? ALG : ALG == kAlgTree ? kTabTreeKappa : ALG == kAlgSubset ? kTabSubsetKappa : ALG;
}

// The amplitude rounds of the ordering-sum algorithm: the prefix tree of the
// paper's method or the subset recursion, fixed per kernel by ALG, or (ALG =
// kAlgAny) chosen by `alg`, uniform per launch.
// kappa: also the condition bound recs[p].kap2 (FP32 escalation).
template <class R, int N, int BLOCK, int BAR = 0, int ALG = kAlgAny, int HB = -1, int G = -1>
__device__ __forceinline__ void amp_rounds(unsigned char* smem, PointRec<R, N>* recs, int cnt, const uint32_t* mask,
                                           int alg, bool kappa = false) {
    if constexpr (ALG == kAlgSubset) {
        amplitude_rounds_meet<R, N, BLOCK, BAR>(smem, recs, cnt, mask);
        if (kappa) kappa_rounds<R, N, BLOCK, BAR>(smem, recs, cnt, mask);
    } else if constexpr (ALG == kAlgTree) {
        using SH = ShapeSel<R, N, BLOCK, HB, G>;
        amplitude_rounds<R, N, BLOCK, BAR, SH::HB, SH::G>(smem, recs, cnt, mask);
        if (kappa) kappa_rounds<R, N, BLOCK, BAR>(smem, recs, cnt, mask);
    } else if (alg == kAlgSubset) {
        amp_rounds<R, N, BLOCK, BAR, kAlgSubset>(smem, recs, cnt, mask, alg, kappa);
    } else {
        amp_rounds<R, N, BLOCK, BAR, kAlgTree, HB, G>(smem, recs, cnt, mask, alg, kappa);
    }
}

// Shared memory: [region][records].  The region holds the round tables during
// the amplitude rounds and, before them, the tile's FP64 momenta (input rows
// for amp2, generated photons for xsec); the two uses never overlap in time.
__host__ __device__ constexpr int amp2_row(int N) { return (N + 2) * 4 + 1; }   // odd stride: conflict-free rows

template <class R, int N, int BLOCK, int ALG = kAlgAny>
__host__ __device__ constexpr size_t amp2_region_bytes(int tile) {
    const size_t st = align16((size_t)tile * amp2_row(N) * sizeof(double));
    return table_bytes<R, N, BLOCK, ALG>() > st ? table_bytes<R, N, BLOCK, ALG>() : st;
}
template <class R, int N, int BLOCK, int ALG = kAlgAny, int HB = -1, int G = -1>
__host__ __device__ constexpr size_t xsec_region_bytes(int tile) {
    const size_t st = align16((size_t)tile * N * kMomSlots * sizeof(double));
    constexpr size_t tb = table_bytes<R, N, BLOCK, ALG, HB, G>();
    return tb > st ? tb : st;
}
template <class R, int N, int BLOCK, int ALG = kAlgAny>
__host__ __device__ constexpr size_t amp2_smem_bytes(int tile) {
    return amp2_region_bytes<R, N, BLOCK, ALG>(tile) + align16((size_t)tile * sizeof(PointRec<R, N>));
}
// The fused tile's running sums wait in shared memory (one Partial per
// thread, after the records) while the FP32 amplitude rounds from n = 6 hold
// every register they can get.
template <class R, int N>
__host__ __device__ constexpr bool xsec_parks_sums() {
    return sizeof(R) == sizeof(float) && N >= 6;
}
template <class R, int N, int BLOCK, int ALG = kAlgAny, int HB = -1, int G = -1>
__host__ __device__ constexpr size_t xsec_smem_bytes(int tile) {
    return xsec_region_bytes<R, N, BLOCK, ALG, HB, G>(tile) + align16((size_t)tile * sizeof(PointRec<R, N>)) +
           (xsec_parks_sums<R, N>() ? (size_t)BLOCK * sizeof(Partial) : 0);
}

// FP32 -> FP64 escalation lists of a fused launch: block b appends the
// points it flags (absolute point index, FP32 weight) in a fixed order to
// idx/w[b cap ...] and stores their number in cnt[b]; idx == NULL disables
// the bound and the lists (FP64 launches, batches).
struct EscArgs {
    long long* idx;
    double* w;
    int* cnt;
    int cap;
    int pad;
};

// A record escalates when its relative error bound u32 sqrt(kap2 / ssum)
// exceeds tau: kap2 > (tau / u32)^2 ssum.
__device__ __forceinline__ float esc_threshold(double tau) {
    const double q = tau * 16777216.0;   // tau / u32, u32 = 2^-24
    return (float)(q * q);
}

// Record of one input row (smem, API layout [n+2][4]); p1 must be massless
// along +z and p2 along -z, every entry finite.
template <class R, int N>
__device__ __forceinline__ void input_to_rec(const double* __restrict__ row, const Physics& ph, PointRec<R, N>& rec,
                                             int* __restrict__ flag) {
    bool ok = true;
#pragma unroll 1
    for (int a = 0; a < (N + 2) * 4; ++a) ok = ok && isfinite(row[a]);
    const double E1 = row[0], E2 = row[4];
    const double tol = 1e-12;
    ok = ok && E1 > 0 && E2 > 0;
    ok = ok && fabs(row[1]) <= tol * E1 && fabs(row[2]) <= tol * E1 && fabs(row[3] - E1) <= tol * E1;
    ok = ok && fabs(row[5]) <= tol * E2 && fabs(row[6]) <= tol * E2 && fabs(row[7] + E2) <= tol * E2;
    const double s = ok ? 2.0 * (E1 * E2 - row[3] * row[7]) : 1.0;
    const double is = 1.0 / s;
    const double irs = sqrt(is);
    const MomView v{const_cast<double*>(row) + 8, 1, 4};
#pragma unroll 1
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int m = 0; m < 4; ++m) rec.k[a][m] = R(v(a, m) * irs);
    rec.hsel = -1;
    if constexpr (N <= 5) fill_denominators<R, N, true>(v, E2, is, false, rec);   // n >= 6: denominators_parallel
    rec.e1 = R(E1 * irs);
    rec.e2 = R(E2 * irs);
    rec.n1 = R(sqrt(2.0 * E1 * irs));
    rec.n2 = R(sqrt(2.0 * E2 * irs));
    double sp = 1;
    for (int a = 2; a < N; ++a) sp *= is;
    rec.fac = ph.cpl * sp;
    rec.wfac = 0;
    rec.valid = ok;
    rec.mask = 1;
    rec.tries = 1;
    if (!ok) atomicOr(flag, 1);
}

// Denominators of the records recs[0 .. cnt-1] at n >= 6 by the calling
// threads (local id lid of nthr), one item per thread so that the FP64 pipe
// runs whole warps: FP32 records get their n(n+1)/2 invariants (item =
// (record, invariant)), FP64 records their 2^n - 2 denominators (item =
// (record, set)).  view(c, E1, E2, is) gives record c's photon momenta, the
// energies of p1 and p2 and the scale 1/s-hat (SCALE: momenta in GeV; MASSLESS: photons on
// shell, k^2 = 0).  Nothing at n <= 5 (the records hold their denominators
// already).
template <class R, int N, bool SCALE, bool MASSLESS, class View>
__device__ __forceinline__ void denominators_parallel(PointRec<R, N>* recs, int cnt, int lid, int nthr,
                                                      const View& view) {
    if constexpr (rec_invariants<R, N>()) {
        constexpr int NI = N * (N + 3) / 2;
        for (int it = lid; it < cnt * NI; it += nthr) {
            const int c = it / NI, q = it - c * NI;
            double E1, E2, is;
            const MomView v = view(c, E1, E2, is);
            recs[c].inv[q] = split_ff(rec_invariant<N, SCALE>(v, E1, E2, is, MASSLESS, q));
        }
    } else if constexpr (N >= 6) {
        constexpr int NSET = (1 << N) - 2;
        for (int it = lid; it < cnt * NSET; it += nthr) {
            const int c = it / NSET;
            const unsigned T = 1u + (unsigned)(it - c * NSET);
            double E1, E2, is;
            const MomView v = view(c, E1, E2, is);
            recs[c].t[T] = set_denominator<R, N, SCALE>(v, E2, is, T);
        }
    }
}

// Staged input row c (stride srow) as a view for denominators_parallel: the
// photons, the energies of p1 and p2 and 1/s-hat as input_to_rec forms them (a row it
// refuses is never evaluated).
__device__ __forceinline__ MomView row_view(double* stage, int srow, int c, double& E1, double& E2, double& is) {
    double* row = stage + (size_t)c * srow;
    E1 = row[0];
    E2 = row[4];
    const double s = 2.0 * (row[0] * row[4] - row[3] * row[7]);
    is = s > 0 ? 1.0 / s : 1.0;
    return MomView{row + 8, 1, 4};
}

// Resident blocks per SM an amp2 kernel is compiled for: the FP32 subset
// recursion from n = 6 keeps three blocks of its 60 KB tables (at most 85
// registers a thread); elsewhere the compiler's choice.
template <class R, int N, int ALG>
__host__ __device__ constexpr int amp2_min_blocks() {
    return sizeof(R) == sizeof(float) && ALG == kAlgSubset && N >= 6 ? 3 : 1;
}

template <class R, int N, int BLOCK, bool ESC, int ALG>
__global__ void __launch_bounds__(BLOCK, amp2_min_blocks<R, N, ALG>())
amp2_kernel(const double* __restrict__ mom, long long npts, const uint32_t* __restrict__ mask,
            double* __restrict__ out, int tile, Physics ph, int* __restrict__ flag, int* __restrict__ esc_list,
            int* __restrict__ esc_count) {
    extern __shared__ __align__(16) unsigned char smem[];
    double* stage = reinterpret_cast<double*>(smem);
    constexpr bool esc = ESC && sizeof(R) == sizeof(float);
    PointRec<R, N>* recs =
        reinterpret_cast<PointRec<R, N>*>(smem + amp2_region_bytes<R, N, BLOCK, table_alg<ALG, esc>()>(tile));
    constexpr int ROW = (N + 2) * 4, SROW = amp2_row(N);
    for (long long t0 = (long long)blockIdx.x * tile; t0 < npts; t0 += (long long)gridDim.x * tile) {
        const int cnt = (int)min((long long)tile, npts - t0);
        // coalesced copy of the tile's rows into shared memory
        const double* src = mom + (size_t)t0 * ROW;
        for (int e = threadIdx.x; e < cnt * ROW; e += BLOCK) {
            const int t = e / ROW;
            stage[t * SROW + (e - t * ROW)] = __ldg(src + e);
        }
        __syncthreads();
        for (int t = threadIdx.x; t < cnt; t += BLOCK) input_to_rec<R, N>(stage + t * SROW, ph, recs[t], flag);
        if constexpr (N >= 6) {
            denominators_parallel<R, N, true, false>(recs, cnt, threadIdx.x, BLOCK, [&](int c, double& E1, double& E2, double& is) {
                return row_view(stage, SROW, c, E1, E2, is);
            });
        }
        __syncthreads();
        amp_rounds<R, N, BLOCK, 0, ALG>(smem, recs, cnt, mask, ph.alg, esc);
        const float thr = esc ? esc_threshold(ph.esc_tau) : 0.0f;
        // one thread per point: FP64 normalisation and a coalesced store; points
        // whose FP32 error bound exceeds the threshold are listed for FP64
        for (int t = threadIdx.x; t < cnt; t += BLOCK) {
            out[t0 + t] = recs[t].valid ? (double)recs[t].ssum * recs[t].fac
                                        : __longlong_as_double(0x7ff8000000000000ll);
            if (esc && recs[t].valid && recs[t].kap2 > thr * recs[t].ssum) esc_list[atomicAdd(esc_count, 1)] = (int)(t0 + t);
        }
    }
}

// Gauge check: ratio[i] = max_h |M_h(eps_w -> k_w/k_w^0)| / max_h |M_h| for
// the input rows (same staging and records as amp2_kernel).
template <class R, int N, int BLOCK>
__global__ void __launch_bounds__(BLOCK)
ward_kernel(const double* __restrict__ mom, long long npts, int ward, double* __restrict__ out, int tile,
            Physics ph, int* __restrict__ flag) {
    extern __shared__ __align__(16) unsigned char smem[];
    double* stage = reinterpret_cast<double*>(smem);
    PointRec<R, N>* recs = reinterpret_cast<PointRec<R, N>*>(smem + amp2_region_bytes<R, N, BLOCK, kAlgTree>(tile));
    constexpr int ROW = (N + 2) * 4, SROW = amp2_row(N);
    for (long long t0 = (long long)blockIdx.x * tile; t0 < npts; t0 += (long long)gridDim.x * tile) {
        const int cnt = (int)min((long long)tile, npts - t0);
        const double* src = mom + (size_t)t0 * ROW;
        for (int e = threadIdx.x; e < cnt * ROW; e += BLOCK) {
            const int t = e / ROW;
            stage[t * SROW + (e - t * ROW)] = __ldg(src + e);
        }
        __syncthreads();
        for (int t = threadIdx.x; t < cnt; t += BLOCK) input_to_rec<R, N>(stage + t * SROW, ph, recs[t], flag);
        if constexpr (N >= 6) {
            denominators_parallel<R, N, true, false>(recs, cnt, threadIdx.x, BLOCK, [&](int c, double& E1, double& E2, double& is) {
                return row_view(stage, SROW, c, E1, E2, is);
            });
        }
        __syncthreads();
        ward_rounds<R, N, BLOCK>(smem, recs, cnt, ward);
        for (int t = threadIdx.x; t < cnt; t += BLOCK)
            out[t0 + t] = recs[t].valid ? (double)recs[t].ssum : __longlong_as_double(0x7ff8000000000000ll);
    }
}

// Deterministic block reduction of per-thread partials (shuffle tree, then
// warp leaders in order).  Uses `scratch` (BLOCK/32 Partials of shared
// memory); result valid in thread 0.
template <int BLOCK>
__device__ __forceinline__ Partial block_reduce_partial(Partial a, Partial* scratch) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        Partial b;
        b.sw.hi = __shfl_down_sync(0xffffffffu, a.sw.hi, off);
        b.sw.lo = __shfl_down_sync(0xffffffffu, a.sw.lo, off);
        b.sw2.hi = __shfl_down_sync(0xffffffffu, a.sw2.hi, off);
        b.sw2.lo = __shfl_down_sync(0xffffffffu, a.sw2.lo, off);
        b.npass = __shfl_down_sync(0xffffffffu, a.npass, off);
        b.ntotal = __shfl_down_sync(0xffffffffu, a.ntotal, off);
        b.ntries = __shfl_down_sync(0xffffffffu, a.ntries, off);
        b.nesc = __shfl_down_sync(0xffffffffu, a.nesc, off);
        a = partial_add(a, b);
    }
    if ((threadIdx.x & 31) == 0) scratch[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int w = 1; w < BLOCK / 32; ++w) a = partial_add(a, scratch[w]);
    return a;
}

__device__ __forceinline__ Partial zero_partial() {
    Partial p;
    p.sw = DD{0, 0};
    p.sw2 = DD{0, 0};
    p.npass = p.ntotal = p.ntries = p.nesc = 0;
    return p;
}

// Ordered compaction: the position of this thread's flagged item among the
// flagged items of the calling threads (in thread order), and their total.
// All THREADS threads (whole warps, local ids 0 .. THREADS-1) must call it;
// they synchronise on __syncthreads (bar = 0) or on named barrier `bar`.
// cnts: THREADS/32 ints of shared memory.
template <int THREADS>
__device__ __forceinline__ int compact_pos(bool flag, int local, int* cnts, int bar, int& total) {
    const unsigned b = __ballot_sync(0xffffffffu, flag);
    const int warp = local >> 5, lane = local & 31;
    if (lane == 0) cnts[warp] = __popc(b);
    if (bar == 0) __syncthreads();
    else asm volatile("bar.sync %0, %1;" ::"r"(bar), "n"(THREADS) : "memory");
    int before = 0;
    total = 0;
#pragma unroll
    for (int w = 0; w < THREADS / 32; ++w) {
        const int c = cnts[w];
        before += w < warp ? c : 0;
        total += c;
    }
    if (bar == 0) __syncthreads();
    else asm volatile("bar.sync %0, %1;" ::"r"(bar), "n"(THREADS) : "memory");
    return before + __popc(b & ((1u << lane) - 1u));
}

// One tile of the fused path: points first .. first+cnt-1 (cnt <= tile) of
// stream `seed` are generated (one thread per point).  Only points that pass
// the cuts get a record, compacted in point order (a point that fails has
// weight 0 and needs no amplitude); their amplitudes are computed in rounds
// and their weights folded into acc.  w_out (may be NULL) receives the
// tile's weights (0 for points that fail the cuts).
template <class R, int N, int BLOCK, bool ESC = false, int ALG = kAlgAny, int HB = -1, int G = -1>
__device__ __forceinline__ void xsec_tile(unsigned char* smem, int tile, uint64_t seed, long long first, int cnt,
                                          const SamplerArgs& S, const Physics& ph, Partial& acc,
                                          double* __restrict__ w_out, const EscArgs& esc, int& esc_n) {
    __shared__ int s_cnt[BLOCK / 32];
    double* stage = reinterpret_cast<double*>(smem);
    constexpr bool kEsc = ESC && sizeof(R) == sizeof(float);
    PointRec<R, N>* recs =
        reinterpret_cast<PointRec<R, N>*>(smem + xsec_region_bytes<R, N, BLOCK, table_alg<ALG, kEsc>(), HB, G>(tile));
    int npass = 0;
    for (int t0 = 0; t0 < cnt; t0 += BLOCK) {
        const int t = t0 + (int)threadIdx.x;
        const MomView v{stage + t, tile, kMomSlots};
        EventInfo ev;
        bool pass = false;
        if (t < cnt) {
            generate_event<N>(seed, (uint64_t)(first + t), S, ph, v, ev);
            pass = ev.ok && ev.mask;
            acc.npass += ev.mask;
            acc.ntotal += 1;
            acc.ntries += ev.tries;
            if (w_out && !pass) w_out[t] = 0.0;
        }
        int tot;
        const int pos = compact_pos<BLOCK>(pass, threadIdx.x, s_cnt, 0, tot);
        if (pass) {
            recs[npass + pos].idx = t;
            recs[npass + pos].hsel = point_hsel<N>(ph, seed, (uint64_t)(first + t));
            recs[npass + pos].fac = ev.irs;   // 1/sqrt(s-hat) until the record is built
        }
        npass += tot;
    }
    __syncthreads();
    // records built one per thread in compacted order: every lane busy
    for (int c = threadIdx.x; c < npass; c += BLOCK) {
        PointRec<R, N>& rec = recs[c];
        pass_to_rec<R, N>(MomView{stage + rec.idx, tile, kMomSlots}, rec.fac, ph, rec);
    }
    if constexpr (N >= 6) {
        __syncthreads();   // the staged momenta are scaled in place by pass_to_rec
        denominators_parallel<R, N, false, true>(recs, npass, threadIdx.x, BLOCK, [&](int c, double& E1, double& E2, double& is) {
            E1 = E2 = 0.5;
            is = 1.0;
            return MomView{stage + recs[c].idx, tile, kMomSlots};
        });
    }
    __syncthreads();
    if constexpr (xsec_parks_sums<R, N>()) {
        Partial* park = reinterpret_cast<Partial*>(reinterpret_cast<unsigned char*>(recs) +
                                                   align16((size_t)tile * sizeof(PointRec<R, N>)));
        park[threadIdx.x] = acc;
        amp_rounds<R, N, BLOCK, 0, ALG, HB, G>(smem, recs, npass, nullptr, ph.alg, kEsc);
        acc = park[threadIdx.x];
    } else {
        amp_rounds<R, N, BLOCK, 0, ALG, HB, G>(smem, recs, npass, nullptr, ph.alg, kEsc);
    }
    // one thread per record: weight and double-double accumulation; records
    // whose FP32 error bound exceeds the threshold join the escalation list
    if constexpr (!kEsc) {
        for (int c = threadIdx.x; c < npass; c += BLOCK) {
            const double w = (double)recs[c].ssum * recs[c].wfac;
            acc.sw = dd_add_d(acc.sw, w);
            acc.sw2 = dd_add_d(acc.sw2, w * w);
            if (w_out) w_out[recs[c].idx] = w;
        }
        return;
    }
    const float thr = esc_threshold(ph.esc_tau);
    for (int c0 = 0; c0 < npass; c0 += BLOCK) {
        const int c = c0 + (int)threadIdx.x;
        bool flag = false;
        double w = 0.0;
        if (c < npass) {
            w = (double)recs[c].ssum * recs[c].wfac;
            acc.sw = dd_add_d(acc.sw, w);
            acc.sw2 = dd_add_d(acc.sw2, w * w);
            if (w_out) w_out[recs[c].idx] = w;
            flag = recs[c].kap2 > thr * recs[c].ssum;
        }
        {
            int tot;
            const int pos = compact_pos<BLOCK>(flag, threadIdx.x, s_cnt, 0, tot);
            if (flag && esc_n + pos < esc.cap) {
                const size_t e = (size_t)blockIdx.x * esc.cap + esc_n + pos;
                esc.idx[e] = first + recs[c].idx;
                esc.w[e] = w;
            }
            esc_n += tot;
        }
    }
}

// Resident blocks per SM a tile kernel is compiled for (its register
// budget; a sub-partition holds at most 16384 registers of its warps): for
// the FP32 tree from n = 6 as many blocks as 128 registers per thread allow
// (three 160-thread blocks at n = 6, two blocks of 224 or 256 above); n = 2
// three blocks (at most 68 KB); elsewhere two blocks (up to 128 registers).
template <class R, int N, int BLOCK, bool ESC, int ALG>
__host__ __device__ constexpr int tile_min_blocks() {
    return (sizeof(R) == sizeof(float) && ALG == kAlgTree && !ESC && N >= 6)
               ? (65536 / (BLOCK * 128) > 1 ? 65536 / (BLOCK * 128) : 1)
               : N == 2 ? 3 : 2;
}
// Threads of a fused tile kernel's block: for the FP32 tree, as many warps as
// share out the depth-2 prefixes evenly with one subtree group per warp
// (30 / 5 at n = 6, 42 / 7 at n = 7), 256 elsewhere.
template <class R, int N, int ALG>
__host__ __device__ constexpr int xsec_block() {
    return sizeof(R) == sizeof(float) && ALG == kAlgTree ? (N == 6 ? 160 : N == 7 ? 224 : 256) : 256;
}

template <class R, int N, int BLOCK, bool ESC, int ALG, int HB = -1, int G = -1>
__global__ void __launch_bounds__(BLOCK, tile_min_blocks<R, N, BLOCK, ESC, ALG>())
xsec_kernel(uint64_t seed, long long i0, long long npts, SamplerArgs S, Physics ph, int tile,
            Partial* __restrict__ partials, double* __restrict__ w_out, EscArgs esc) {
    extern __shared__ __align__(16) unsigned char smem[];
    Partial acc = zero_partial();
    int esc_n = 0;
    for (long long t0 = (long long)blockIdx.x * tile; t0 < npts; t0 += (long long)gridDim.x * tile) {
        const int cnt = (int)min((long long)tile, npts - t0);
        xsec_tile<R, N, BLOCK, ESC, ALG, HB, G>(smem, tile, seed, i0 + t0, cnt, S, ph, acc, w_out ? w_out + t0 : nullptr, esc,
                                         esc_n);
    }
    if (ESC && threadIdx.x == 0) esc.cnt[blockIdx.x] = min(esc_n, esc.cap);
    // the round tables are free now: reuse them as reduction scratch
    const Partial r = block_reduce_partial<BLOCK>(acc, reinterpret_cast<Partial*>(smem));
    if (threadIdx.x == 0) partials[blockIdx.x] = r;
}

// FP64 recomputation of the points an FP32 launch flagged (same grid): block
// b regenerates the events of its list in order, evaluates them in FP64 (with
// the subset recursion: the same |M|^2 as the tree, far cheaper at large n) and
// leaves the corrections sum (w64 - w32), sum (w64^2 - w32^2) and the count
// in out[b]; w_out (relative to i0) receives the FP64 weights.  Combined
// after the FP32 partials in fixed order, they make the flagged points count
// with their FP64 weights.
template <int N, int BLOCK>
__global__ void __launch_bounds__(BLOCK)
xsec_escalate_kernel(uint64_t seed, long long i0, SamplerArgs S, Physics ph, int tile, EscArgs esc,
                     Partial* __restrict__ out, double* __restrict__ w_out) {
    extern __shared__ __align__(16) unsigned char smem[];
    double* stage = reinterpret_cast<double*>(smem);
    PointRec<double, N>* recs =
        reinterpret_cast<PointRec<double, N>*>(smem + xsec_region_bytes<double, N, BLOCK, kAlgSubset>(tile));
    const int nb = esc.cnt[blockIdx.x];
    const size_t base = (size_t)blockIdx.x * esc.cap;
    Partial acc = zero_partial();
    for (int c0 = 0; c0 < nb; c0 += tile) {
        const int cnt = min(tile, nb - c0);
        for (int t = threadIdx.x; t < cnt; t += BLOCK) {
            const MomView v{stage + t, tile, kMomSlots};
            EventInfo ev;
            generate_event<N>(seed, (uint64_t)esc.idx[base + c0 + t], S, ph, v, ev);
            pass_to_rec<double, N>(v, ev.irs, ph, recs[t]);
            recs[t].idx = t;
            recs[t].hsel = point_hsel<N>(ph, seed, (uint64_t)esc.idx[base + c0 + t]);
        }
        if constexpr (N >= 6) {
            __syncthreads();
            denominators_parallel<double, N, false, true>(recs, cnt, threadIdx.x, BLOCK, [&](int c, double& E1, double& E2, double& is) {
                E1 = E2 = 0.5;
                is = 1.0;
                return MomView{stage + c, tile, kMomSlots};
            });
        }
        __syncthreads();
        amp_rounds<double, N, BLOCK, 0, kAlgSubset>(smem, recs, cnt, nullptr, kAlgSubset);
        for (int t = threadIdx.x; t < cnt; t += BLOCK) {
            const double w64 = recs[t].ssum * recs[t].wfac, w32 = esc.w[base + c0 + t];
            acc.sw = dd_add_d(acc.sw, w64 - w32);
            acc.sw2 = dd_add_d(acc.sw2, w64 * w64 - w32 * w32);
            if (w_out) w_out[esc.idx[base + c0 + t] - i0] = w64;
        }
        __syncthreads();
    }
    Partial r = block_reduce_partial<BLOCK>(acc, reinterpret_cast<Partial*>(smem));
    if (threadIdx.x == 0) {
        r.nesc = nb;
        out[blockIdx.x] = r;
    }
}

// FP64 |M|^2 (subset recursion) of the rows listed by an FP32 heget_amp2
// launch (their number in *count): out[list[k]] is overwritten.
template <int N, int BLOCK>
__global__ void __launch_bounds__(BLOCK)
amp2_list_kernel(const double* __restrict__ mom, const int* __restrict__ list, const int* __restrict__ count,
                 const uint32_t* __restrict__ mask, double* __restrict__ out, int tile, Physics ph,
                 int* __restrict__ flag) {
    extern __shared__ __align__(16) unsigned char smem[];
    double* stage = reinterpret_cast<double*>(smem);
    PointRec<double, N>* recs =
        reinterpret_cast<PointRec<double, N>*>(smem + amp2_region_bytes<double, N, BLOCK, kAlgSubset>(tile));
    constexpr int ROW = (N + 2) * 4, SROW = amp2_row(N);
    const long long npts = *count;
    for (long long t0 = (long long)blockIdx.x * tile; t0 < npts; t0 += (long long)gridDim.x * tile) {
        const int cnt = (int)min((long long)tile, npts - t0);
        for (int e = threadIdx.x; e < cnt * ROW; e += BLOCK) {
            const int t = e / ROW;
            stage[t * SROW + (e - t * ROW)] = __ldg(mom + (size_t)list[t0 + t] * ROW + (e - t * ROW));
        }
        __syncthreads();
        for (int t = threadIdx.x; t < cnt; t += BLOCK) input_to_rec<double, N>(stage + t * SROW, ph, recs[t], flag);
        if constexpr (N >= 6) {
            denominators_parallel<double, N, true, false>(recs, cnt, threadIdx.x, BLOCK, [&](int c, double& E1, double& E2, double& is) {
                return row_view(stage, SROW, c, E1, E2, is);
            });
        }
        __syncthreads();
        amp_rounds<double, N, BLOCK, 0, kAlgSubset>(smem, recs, cnt, mask, kAlgSubset);
        for (int t = threadIdx.x; t < cnt; t += BLOCK) out[list[t0 + t]] = (double)recs[t].ssum * recs[t].fac;
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Mixed-n batch: one launch over a work list of tiles drawn from several
// requests (any n in 2..8, any N).  Each block takes work items in a
// grid-stride loop; the item's n selects the code path (uniform per block),
// and every item leaves one partial, in its request's partial array at the
// tile's index.  A request's tiles do not depend on the rest of the batch,
// and its partials are combined in tile order, so a request gives the same
// result, bit for bit, alone or in any mix.
// ---------------------------------------------------------------------------
struct BatchReq {
    uint64_t seed;
    long long i0;
    SamplerArgs S;
    Physics ph;
    double* w_out;
    heget_xsec_result* result;
    Partial* parts;   // this request's tile partials, tile k at parts[k]
    int n, tile, ntiles, pad;
};

struct WorkItem {
    int req;          // index into the request table
    int n;            // photons of that request
    int count;        // points in this tile
    int pad;
    long long start;  // first point of the tile, relative to the request
};

// One instantiation per ordering-sum algorithm (ALG = kAlgTree or kAlgSubset,
// the context's, uniform over a batch), so that neither algorithm's code
// shapes the other's registers and instruction footprint.
template <class R, int ALG>
__global__ void __launch_bounds__(kBatchThreads)
xsec_batch_kernel(const WorkItem* __restrict__ items, int nitems, const BatchReq* __restrict__ reqs) {
    extern __shared__ __align__(16) unsigned char smem[];
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const WorkItem w = items[it];
        const BatchReq& rq = reqs[w.req];
        Partial acc = zero_partial();
        int esc_n = 0;
        const EscArgs kNoEsc{nullptr, nullptr, nullptr, 0, 0};
        double* wo = rq.w_out ? rq.w_out + w.start : nullptr;
        const long long first = rq.i0 + w.start;
        switch (w.n) {
#define HEGET_BATCH_CASE(NN)                                                                                   \
    case NN:                                                                                                   \
        xsec_tile<R, NN, kBatchThreads, false, ALG>(smem, rq.tile, rq.seed, first, w.count, rq.S, rq.ph, acc, wo, \
                                                     kNoEsc, esc_n);                                           \
        break;
            HEGET_BATCH_CASE(2)
            HEGET_BATCH_CASE(3)
            HEGET_BATCH_CASE(4)
            HEGET_BATCH_CASE(5)
            HEGET_BATCH_CASE(6)
            HEGET_BATCH_CASE(7)
            HEGET_BATCH_CASE(8)
#undef HEGET_BATCH_CASE
            default:
                break;
        }
        const Partial r = block_reduce_partial<kBatchThreads>(acc, reinterpret_cast<Partial*>(smem));
        if (threadIdx.x == 0) rq.parts[w.start / rq.tile] = r;
        __syncthreads();   // the scratch is the next item's staging area
    }
}

// ---------------------------------------------------------------------------
// Warp-specialised fused kernel (FP32 chain).
//
// GB300 runs FP64 at ~1/64 of the FP32 rate and with long latency, so the FP64
// event generation (RAMBO, cuts, denominators) costs more than the FP32
// amplitudes at small n (and at every n with the subset recursion), and at
// n = 6 still about half of them, and needs many events in flight while the
// amplitudes run.  Each block therefore splits into roles that run
// concurrently:
//   consumers (ws_consumers(n, alg, esc) threads, the first warps): the amplitude
//               rounds, and the sampler draws of the stage two ahead;
//   producers (ws_stage(n, alg) threads, the last warps): one event per
//               thread per stage from its draws: the FP64 rest (sqrt(s-hat),
//               RAMBO, cuts, records).
// The sampler (the toy PDF's rejection loops) is integer and FP32 work whose
// iteration counts differ from lane to lane; run on the producers it would
// idle the FP64 pipe, on the consumers it fills their waits.
// Producers fill a double-buffered ring of ws_stage(n) point records in shared
// memory; the two roles hand stages over through named barriers
//   FULL[s]  (bar.arrive by producers, bar.sync by consumers) and
//   EMPTY[s] (bar.arrive by consumers, bar.sync by producers);
// the draws of stage k + 2 go into slot s = k & 1 of a second double buffer
// before the consumers' EMPTY[s] arrival (those of stages 0 and 1 before the
// roles split),
// while the consumers' own rounds synchronise on barrier kBarRounds.  Every
// thread of both roles runs the same number of stages, so each barrier
// instance collects exactly ws_consumers + ws_stage arrivals.  A block walks tiles
// blockIdx.x, blockIdx.x + gridDim.x, ...; the grid is sized to the resident
// blocks so that each block pipelines many stages.
// ---------------------------------------------------------------------------
constexpr int kBarRounds = 1, kBarFull = 2, kBarEmpty = 4;   // named barrier ids (2,3 / 4,5)
constexpr int kBarProducers = 6;                              // producers' stage compaction

// Consumer threads: 256; 128 for the tree up to n = 4 without the FP32
// error bound, whose amplitudes are a small share of the block's work (with
// 256, the consumer warps took issue slots from the FP64 producers: GB300
// n = 4, 4.98e8 against 4.77e8 evaluated points/s; 96 or 64 starve the
// amplitudes, and so does the bound of the escalating kernel, which keeps
// 256; the subset recursion up to n = 4 and the tree at n = 5 ran 4-16 %
// slower with 128); 160 for the FP32 tree at n = 6 (five pair-unit slots of two points
// share out the 15 units evenly); 384 for the subset recursion from n = 7
// (three groups of four warps, one block per SM).
__host__ __device__ constexpr int ws_consumers(int n, int alg, bool esc) {
    return n <= 4 && alg == 0 && !esc ? 128 : n == 6 && alg == 0 ? 160 : n >= 7 && alg == 1 ? 384 : 256;
}
// Points per stage (= producer threads, a multiple of 32): as many as the
// shared memory of the ring, the producers' staging and the round tables
// allows at two resident blocks per SM; 64 at n = 5, 6, whose FP64
// generation then spans two warps (one warp leaves the FP64 pipe waiting on
// its own latencies).  The subset recursion from n = 7 takes 96 with its 384
// consumers at one block per SM: there the FP64 generation of about four
// events per evaluated point outweighs the recursion, and three producer
// warps keep three sub-partitions' FP64 units busy (GB300, n = 8: 8.5e7
// points/s, from 6.2e7 with 32 producers and two blocks per SM).
__host__ __device__ constexpr int ws_stage(int n, int alg) {
    return n <= 4 ? 128 : n <= 6 ? 64 : alg == 1 ? 96 : 32;
}

__device__ __forceinline__ void named_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void named_arrive(int id, int count) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Shared-memory layout of the warp-specialised kernel of algorithm ALG with
// table layout TAB: round tables, the double-buffered ring of records, the
// producers' staging.
// Threads of a warp-specialised block (one value for the kernel's launch
// bounds, its barriers and its launch); a table layout with the FP32 error
// bound marks the escalating kernel.
__host__ __device__ constexpr bool tab_has_bound(int tab) { return tab == kTabTreeKappa || tab == kTabSubsetKappa; }
template <int N, int ALG, bool ESC>
__host__ __device__ constexpr int ws_threads() {
    return ws_consumers(N, ALG, ESC) + ws_stage(N, ALG);
}
template <class R, int N, int ALG, int TAB>
__host__ __device__ constexpr size_t ws_recs_offset() {
    return table_bytes<R, N, ws_consumers(N, ALG, tab_has_bound(TAB)), TAB>();
}
template <class R, int N, int ALG, int TAB>
__host__ __device__ constexpr size_t ws_stage_offset() {
    return ws_recs_offset<R, N, ALG, TAB>() + 2 * align16((size_t)ws_stage(N, ALG) * sizeof(PointRec<R, N>));
}
template <class R, int N, int ALG, int TAB = ALG>
__host__ __device__ constexpr size_t ws_smem_bytes() {
    return ws_stage_offset<R, N, ALG, TAB>() + align16((size_t)ws_stage(N, ALG) * N * kMomSlots * sizeof(double));
}
template <class R, int N, int ALG, int TAB>
__host__ __device__ constexpr int ws_min_blocks() {
    return ws_smem_bytes<R, N, ALG, TAB>() <= 113 * 1024 ? 2 : 1;
}

template <class R, int N, bool ESC, int ALG>
__global__ void __launch_bounds__(ws_threads<N, ALG, ESC>(), ws_min_blocks<R, N, ALG, table_alg<ALG, ESC>()>())
xsec_ws_kernel(uint64_t seed, long long i0, long long npts, SamplerArgs S, Physics ph,
               Partial* __restrict__ partials, double* __restrict__ w_out, EscArgs esc) {
    constexpr int kWsConsumers = ws_consumers(N, ALG, ESC);
    constexpr int kWsStage = ws_stage(N, ALG);
    constexpr int kWsThreads = ws_threads<N, ALG, ESC>();
    static_assert(kWsThreads == kWsConsumers + kWsStage, "block shape");
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int TAB = table_alg<ALG, ESC>();
    PointRec<R, N>* ring = reinterpret_cast<PointRec<R, N>*>(smem + ws_recs_offset<R, N, ALG, TAB>());
    constexpr size_t ring_stride = align16((size_t)kWsStage * sizeof(PointRec<R, N>)) / sizeof(PointRec<R, N>);
    double* stage = reinterpret_cast<double*>(smem + ws_stage_offset<R, N, ALG, TAB>());
    __shared__ int s_cnt[kWsStage / 32];
    __shared__ int stage_n[2];   // records (cut-passing points) of the stage in each ring slot
    __shared__ SampleDraw s_draw[2][kWsStage];   // sampler draws of the stage in each slot
    const int tid = threadIdx.x;
    const long long tiles = (npts + kWsStage - 1) / kWsStage;
    const int count = tiles > blockIdx.x ? (int)((tiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;
    Partial acc = zero_partial();
    auto stage_t0 = [&](int k) { return ((long long)blockIdx.x + (long long)k * gridDim.x) * kWsStage; };
    // draws of stage k into slot s by `nthr` threads (local ids `lid`)
    auto draw_stage = [&](int k, int s, int lid, int nthr) {
        const long long t0 = stage_t0(k);
        for (int p = lid; p < kWsStage; p += nthr)
            if (t0 + p < npts) s_draw[s][p] = sample_draw(S, PointRng(seed, (uint64_t)(i0 + t0 + p)));
    };
    for (int k = 0; k < 2 && k < count; ++k) draw_stage(k, k, tid, kWsThreads);
    __syncthreads();
    // the producer owning slot g of stage k folds that point's weight into its
    // accumulator once the consumers have released the stage
    int esc_n = 0;
    const float thr = ESC ? esc_threshold(ph.esc_tau) : 0.0f;
    // (called by every producer for the same stages, in order)
    auto harvest = [&](int k, int g) {
        bool flag = false;
        double w = 0.0;
        const PointRec<R, N>& rec = ring[(k & 1) * ring_stride + g];
        if (g < stage_n[k & 1]) {
            w = (double)rec.ssum * rec.wfac;
            acc.sw = dd_add_d(acc.sw, w);
            acc.sw2 = dd_add_d(acc.sw2, w * w);
            if (w_out) w_out[stage_t0(k) + rec.idx] = w;
            flag = ESC && rec.kap2 > thr * rec.ssum;
        }
        if constexpr (ESC) {
            int tot;
            const int pos = compact_pos<kWsStage>(flag, g, s_cnt, kBarProducers, tot);
            if (flag && esc_n + pos < esc.cap) {
                const size_t e = (size_t)blockIdx.x * esc.cap + esc_n + pos;
                esc.idx[e] = i0 + stage_t0(k) + rec.idx;
                esc.w[e] = w;
            }
            esc_n += tot;
        }
    };
    if (tid >= kWsConsumers) {
        // producers
        const int g = tid - kWsConsumers;
        const MomView v{stage + g, kWsStage, kMomSlots};
        for (int k = 0; k < count; ++k) {
            const int s = k & 1;
            if (k >= 2) {
                named_sync(kBarEmpty + s, kWsThreads);
                harvest(k - 2, g);
            }
            const long long t0 = stage_t0(k);
            const int cnt = (int)min((long long)kWsStage, npts - t0);
            EventInfo ev;
            bool pass = false;
            if (g < cnt) {
                generate_from<N>(PointRng(seed, (uint64_t)(i0 + t0 + g)), s_draw[s][g], S, ph, v, ev);
                pass = ev.ok && ev.mask;
                acc.npass += ev.mask;
                acc.ntotal += 1;
                acc.ntries += ev.tries;
                if (w_out && !pass) w_out[t0 + g] = 0.0;
            }
            // records only for points that pass the cuts, compacted in point order
            int tot;
            const int pos = compact_pos<kWsStage>(pass, g, s_cnt, kBarProducers, tot);
            PointRec<R, N>* rs_ring = ring + s * ring_stride;
            if (pass) {
                rs_ring[pos].idx = g;
                rs_ring[pos].hsel = point_hsel<N>(ph, seed, (uint64_t)(i0 + t0 + g));
                rs_ring[pos].fac = ev.irs;   // 1/sqrt(s-hat) until the record is built
            }
            named_sync(kBarProducers, kWsStage);
            // records built one per producer in compacted order: every lane busy
            if (g < tot)
                pass_to_rec<R, N>(MomView{stage + rs_ring[g].idx, kWsStage, kMomSlots}, rs_ring[g].fac, ph,
                                  rs_ring[g]);
            if constexpr (N >= 6) {
                named_sync(kBarProducers, kWsStage);   // scaled momenta in place
                denominators_parallel<R, N, false, true>(rs_ring, tot, g, kWsStage, [&](int c, double& E1, double& E2, double& is) {
                    E1 = E2 = 0.5;
                    is = 1.0;
                    return MomView{stage + rs_ring[c].idx, kWsStage, kMomSlots};
                });
            }
            // every producer has read the staged momenta it needed before any
            // of them generates the next stage into its column
            named_sync(kBarProducers, kWsStage);
            if (g == 0) stage_n[s] = tot;
            __threadfence_block();
            named_arrive(kBarFull + s, kWsThreads);
        }
    } else {
        // consumers
        for (int k = 0; k < count; ++k) {
            const int s = k & 1;
            named_sync(kBarFull + s, kWsThreads);
            const int cnt = stage_n[s];
            amp_rounds<R, N, kWsConsumers, kBarRounds, ALG>(smem, ring + s * ring_stride, cnt, nullptr, ph.alg, ESC);
            if (k + 2 < count) {
                draw_stage(k + 2, s, tid, kWsConsumers);   // the producers read slot s after EMPTY[s]
                __threadfence_block();
                named_arrive(kBarEmpty + s, kWsThreads);
            }
        }
    }
    __syncthreads();
    // the last (up to) two stages were never reclaimed: harvest them now
    if (tid >= kWsConsumers) {
        for (int k = count - 2 < 0 ? 0 : count - 2; k < count; ++k) harvest(k, tid - kWsConsumers);
        if (ESC && tid == kWsConsumers) esc.cnt[blockIdx.x] = min(esc_n, esc.cap);
    }
    __syncthreads();
    const Partial r = block_reduce_partial<kWsThreads>(acc, reinterpret_cast<Partial*>(smem));
    if (threadIdx.x == 0) partials[blockIdx.x] = r;
}

// ---------------------------------------------------------------------------
// Host-side launch descriptors.
// ---------------------------------------------------------------------------
struct AmpLaunch {
    int block, tile, grid;
    size_t smem;
    bool ws;        // warp-specialised xsec kernel (FP32)
    int shape = 0;  // tile-kernel shape of the fused cross section (tile_shape; 0 = default)
};

// The warp-specialised kernel runs FP32 cross sections where the FP64 event
// generation is a large share of the work: n <= 5 with the tree, every n with
// the subset recursion.  The tree from n = 6 runs faster on the tile kernel
// with 64-point tiles (GB300: 6.3e7 against 5.6e7 points/s at n = 6; its
// generation spans two warps, and more blocks share an SM).
constexpr bool use_ws(int n, int precision, bool xsec, int alg) {
    return xsec && precision == HEGET_FP32 && (n <= 5 || alg == kAlgSubset);
}

// Per-algorithm launchers over n = 2..8 (ALG = kAlgTree or kAlgSubset),
// defined in heget_launch.cuh and instantiated once per precision and
// algorithm by the kernel translation units.  Return cudaError_t as int.
template <class R, int ALG>
int launch_amp2_alg(int n, const double* mom, long long npts, const uint32_t* mask, double* out, const Physics& ph,
                    int* flag, int* esc_list, int* esc_count, const AmpLaunch& L, cudaStream_t st);
template <class R, int ALG>
int launch_xsec_alg(int n, uint64_t seed, long long i0, long long npts, const SamplerArgs& S, const Physics& ph,
                    Partial* partials, double* w_out, const EscArgs& esc, const AmpLaunch& L, cudaStream_t st);
template <class R, int ALG>
int occupancy_alg(int n, int tile, int* bpsm, size_t* smem, int shape = 0);
template <int ALG>
int occupancy_ws_alg(int n, int* bpsm, size_t* smem);

// The same, dispatched on ph.alg (heget_api.cu).
int launch_amp2_f32(int n, const double* mom, long long npts, const uint32_t* mask, double* out,
                    const Physics& ph, int* flag, int* esc_list, int* esc_count, const AmpLaunch& L, cudaStream_t st);
int launch_amp2_f64(int n, const double* mom, long long npts, const uint32_t* mask, double* out,
                    const Physics& ph, int* flag, int* esc_list, int* esc_count, const AmpLaunch& L, cudaStream_t st);
int launch_xsec_f32(int n, uint64_t seed, long long i0, long long npts, const SamplerArgs& S,
                    const Physics& ph, Partial* partials, double* w_out, const EscArgs& esc, const AmpLaunch& L,
                    cudaStream_t st);
int launch_xsec_f64(int n, uint64_t seed, long long i0, long long npts, const SamplerArgs& S,
                    const Physics& ph, Partial* partials, double* w_out, const EscArgs& esc, const AmpLaunch& L,
                    cudaStream_t st);
// FP64 recomputations of escalated points (subset recursion).
int launch_amp2_list_f64(int n, const double* mom, const int* list, const int* count, const uint32_t* mask,
                         double* out, const Physics& ph, int* flag, int tile, int grid, cudaStream_t st);
int launch_escalate_f64(int n, uint64_t seed, long long i0, const SamplerArgs& S, const Physics& ph, int tile,
                        const EscArgs& esc, Partial* out, double* w_out, int grid, cudaStream_t st);
// Gauge check (prefix tree).
int launch_ward_f32(int n, const double* mom, long long npts, int ward, double* out, const Physics& ph, int* flag,
                    const AmpLaunch& L, cudaStream_t st);
int launch_ward_f64(int n, const double* mom, long long npts, int ward, double* out, const Physics& ph, int* flag,
                    const AmpLaunch& L, cudaStream_t st);
// Mixed-n batch launch (one launch per precision); smem sized for the tiles.
// alg: the ordering-sum algorithm of every item (kAlgTree or kAlgSubset).
int launch_batch_f32(const WorkItem* items, int nitems, const BatchReq* reqs, size_t smem, int grid, int alg,
                     cudaStream_t st, bool set_attr = true);
int launch_batch_f64(const WorkItem* items, int nitems, const BatchReq* reqs, size_t smem, int grid, int alg,
                     cudaStream_t st, bool set_attr = true);
int prepare_batch_f32(size_t smem, int alg);
int prepare_batch_f64(size_t smem, int alg);
// Shared memory of a batch tile of n photons at `precision` with algorithm alg.
size_t batch_tile_smem(int n, int precision, int alg, int tile);
// Points per batch tile when the context sets none: the fused tile kernel's
// default for the tree; for the subset recursion tiles that fill two blocks
// per SM (its per-point cost is far below the tree's at large n).
int batch_default_tile(int n, int precision, int alg);
// One block per request: its tile partials, in order, into its result.
int launch_batch_finalize(const BatchReq* reqs, int nreqs, cudaStream_t st);

// Default launch shape and the maximum resident blocks per SM.
int default_tile(int n, bool xsec);
int default_amp_launch(int n, int precision, long long npts, int num_sms, AmpLaunch* L, bool xsec, int tile,
                       int alg = kAlgTree, int shape = 0);
// Tile-kernel shapes available for the fused cross section (num_tile_shapes).
int xsec_shape_count(int n, int precision, int alg);

}  // namespace heget
