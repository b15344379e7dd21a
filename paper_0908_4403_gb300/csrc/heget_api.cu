// heget_api.cu -- the C ABI of include/heget.h: context, argument checks,
// launch shapes, the phase-space kernel and the fixed-order reductions.
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "heget_kernels.cuh"
#include "heget_internal.h"

namespace heget {

// Launchers dispatched on the ordering-sum algorithm of the launch; each
// algorithm's kernels are separate instantiations (heget_tree_*.cu,
// heget_subset_*.cu), so neither shapes the other's registers.
int launch_amp2_f32(int n, const double* mom, long long npts, const uint32_t* mask, double* out,
                    const Physics& ph, int* flag, int* esc_list, int* esc_count, const AmpLaunch& L, cudaStream_t st) {
    return ph.alg == kAlgSubset
               ? launch_amp2_alg<float, kAlgSubset>(n, mom, npts, mask, out, ph, flag, esc_list, esc_count, L, st)
               : launch_amp2_alg<float, kAlgTree>(n, mom, npts, mask, out, ph, flag, esc_list, esc_count, L, st);
}
int launch_amp2_f64(int n, const double* mom, long long npts, const uint32_t* mask, double* out,
                    const Physics& ph, int* flag, int* esc_list, int* esc_count, const AmpLaunch& L, cudaStream_t st) {
    return ph.alg == kAlgSubset
               ? launch_amp2_alg<double, kAlgSubset>(n, mom, npts, mask, out, ph, flag, esc_list, esc_count, L, st)
               : launch_amp2_alg<double, kAlgTree>(n, mom, npts, mask, out, ph, flag, esc_list, esc_count, L, st);
}
int launch_xsec_f32(int n, uint64_t seed, long long i0, long long npts, const SamplerArgs& S, const Physics& ph,
                    Partial* partials, double* w_out, const EscArgs& esc, const AmpLaunch& L, cudaStream_t st) {
    return ph.alg == kAlgSubset
               ? launch_xsec_alg<float, kAlgSubset>(n, seed, i0, npts, S, ph, partials, w_out, esc, L, st)
               : launch_xsec_alg<float, kAlgTree>(n, seed, i0, npts, S, ph, partials, w_out, esc, L, st);
}
int launch_xsec_f64(int n, uint64_t seed, long long i0, long long npts, const SamplerArgs& S, const Physics& ph,
                    Partial* partials, double* w_out, const EscArgs& esc, const AmpLaunch& L, cudaStream_t st) {
    return ph.alg == kAlgSubset
               ? launch_xsec_alg<double, kAlgSubset>(n, seed, i0, npts, S, ph, partials, w_out, esc, L, st)
               : launch_xsec_alg<double, kAlgTree>(n, seed, i0, npts, S, ph, partials, w_out, esc, L, st);
}

static thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    // The status reports this error; take it out of the runtime's per-thread
    // record so that it does not surface again in the caller's next error
    // check (a sticky error stays sticky regardless).
    cudaGetLastError();
    return fail(HEGET_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// ---------------------------------------------------------------------------
// phase-space kernel: one thread per point
// ---------------------------------------------------------------------------
// Momenta are generated into shared memory (point-minor) and written out
// cooperatively, so the [N][n+2][4] stores are coalesced.
constexpr int kPsBlock = 64;

template <int N>
__global__ void __launch_bounds__(kPsBlock)
phase_space_kernel(uint64_t seed, long long i0, long long npts, SamplerArgs S, Physics ph, double* __restrict__ mom,
                   double* __restrict__ w, double* __restrict__ rs_out, double* __restrict__ y_out,
                   uint8_t* __restrict__ mask_out, int32_t* __restrict__ tries_out) {
    __shared__ double stage[N * kMomSlots * kPsBlock];
    __shared__ double rs_s[kPsBlock];
    constexpr int ROW = (N + 2) * 4;
    for (long long j0 = (long long)blockIdx.x * kPsBlock; j0 < npts; j0 += (long long)gridDim.x * kPsBlock) {
        const int cnt = (int)min((long long)kPsBlock, npts - j0);
        const int t = threadIdx.x;
        if (t < cnt) {
            const long long j = j0 + t;
            const MomView v{stage + t, kPsBlock, kMomSlots};
            EventInfo ev;
            generate_event<N>(seed, (uint64_t)(i0 + j), S, ph, v, ev);
            rs_s[t] = ev.rs;
            if (w) w[j] = ev.ok ? phase_space_weight<N>(ev.rs * ev.rs) : 0.0;
            if (rs_out) rs_out[j] = ev.rs;
            if (y_out) y_out[j] = (S.kind == HEGET_SAMPLER_TOY_PDF && ev.ok) ? 0.5 * log(ev.x1 / ev.x2) : 0.0;
            if (mask_out) mask_out[j] = (uint8_t)ev.mask;
            if (tries_out) tries_out[j] = ev.tries;
        }
        __syncthreads();
        if (mom) {
            double* dst = mom + (size_t)j0 * ROW;
            for (int e = threadIdx.x; e < cnt * ROW; e += kPsBlock) {
                const int p = e / ROW, c = e - p * ROW, a = c >> 2, m = c & 3;
                double val;
                if (a >= 2) {
                    val = stage[(kMomSlots * (a - 2) + m) * kPsBlock + p];
                } else {   // p1 = (rs/2)(1,0,0,1), p2 = (rs/2)(1,0,0,-1)
                    const double h = 0.5 * rs_s[p];
                    val = m == 0 ? h : (m == 3 ? (a == 0 ? h : -h) : 0.0);
                }
                dst[e] = val;
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) log_table_kernel(const double* __restrict__ x, double* __restrict__ y,
                                                        long long n) {
    for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < n; i += (long long)gridDim.x * 256)
        y[i] = log_table(x[i]);
}

__global__ void __launch_bounds__(256) sincos_kernel(const uint32_t* __restrict__ words, double* __restrict__ cs,
                                                     long long n) {
    for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < n; i += (long long)gridDim.x * 256)
        sincos_2pi_words(words[2 * i], words[2 * i + 1], cs[2 * i + 1], cs[2 * i]);
}

__global__ void __launch_bounds__(256) f32_round_kernel(const double* __restrict__ x, float* __restrict__ y,
                                                        long long n) {
    for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < n; i += (long long)gridDim.x * 256)
        y[i] = f32_rn(x[i]);
}

// ---------------------------------------------------------------------------
// fixed-order reductions
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) sum_kernel(const double* __restrict__ x, long long n,
                                                  Partial* __restrict__ partials) {
    __shared__ Partial scratch[8];
    Partial a = zero_partial();
    for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
        const double v = x[i];
        a.sw = dd_add_d(a.sw, v);
        a.sw2 = dd_add_d(a.sw2, v * v);
        a.ntotal += 1;
    }
    const Partial r = block_reduce_partial<256>(a, scratch);
    if (threadIdx.x == 0) partials[blockIdx.x] = r;
}

// Combines nparts block partials in index order (called by one whole block).
// mode 0: write the heget_xsec_result (toy-PDF scale when kind == TOY_PDF);
// mode 1: write (sum, sum of squares) to sums.
__device__ __forceinline__ void finalize_block(const Partial* __restrict__ partials, int nparts, int kind, int mode,
                                               heget_xsec_result* __restrict__ res, double* __restrict__ sums,
                                               Partial* scratch) {
    Partial a = zero_partial();
    for (int b = threadIdx.x; b < nparts; b += 256) a = partial_add(a, partials[b]);
    const Partial r = block_reduce_partial<256>(a, scratch);
    if (threadIdx.x != 0) return;
    const double sw = r.sw.hi + r.sw.lo, sw2 = r.sw2.hi + r.sw2.lo;
    if (mode == 1) {
        sums[0] = sw;
        sums[1] = sw2;
        return;
    }
    const double N = (double)r.ntotal;
    const double mean = N > 0 ? sw / N : 0.0;
    const double var = N > 1 ? fmax(0.0, (sw2 - sw * mean) / (N - 1.0)) : 0.0;
    const double accept = r.ntries > 0 ? N / (double)r.ntries : 1.0;
    const double scale = (kind == HEGET_SAMPLER_TOY_PDF) ? 2.0 * accept : 1.0;
    heget_xsec_result o;
    o.sigma_fb = scale * mean;
    o.err_fb = N > 0 ? scale * sqrt(var / N) : 0.0;
    o.sum_w = sw;
    o.sum_w2 = sw2;
    o.accept = accept;
    o.reserved = 0;
    o.n_pass = r.npass;
    o.n_total = r.ntotal;
    o.n_tries = r.ntries;
    o.n_escalated = r.nesc;
    *res = o;
}

__global__ void __launch_bounds__(256) finalize_kernel(const Partial* __restrict__ partials, int nparts, int kind,
                                                       int mode, heget_xsec_result* __restrict__ res,
                                                       double* __restrict__ sums) {
    __shared__ Partial scratch[8];
    finalize_block(partials, nparts, kind, mode, res, sums, scratch);
}

// One block per batch request: its tile partials, in order, into its result.
__global__ void __launch_bounds__(256) finalize_batch_kernel(const BatchReq* __restrict__ reqs) {
    __shared__ Partial scratch[8];
    const BatchReq& r = reqs[blockIdx.x];
    finalize_block(r.parts, r.ntiles, r.S.kind, 0, r.result, nullptr, scratch);
}

int launch_batch_finalize(const BatchReq* reqs, int nreqs, cudaStream_t st) {
    if (nreqs <= 0) return 0;
    finalize_batch_kernel<<<nreqs, 256, 0, st>>>(reqs);
    return (int)cudaGetLastError();
}

// FMA-throughput probe: kPeakChains independent chains per thread, so the
// FMA pipe, not the FMA latency, limits the rate.
constexpr int kPeakChains = 8;

template <class T>
__global__ void __launch_bounds__(256) fma_peak_kernel(int iters, double* __restrict__ sink) {
    T x[kPeakChains];
    const T a = T(0.999999), b = T(1e-7);
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) x[c] = T(threadIdx.x + c);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kPeakChains; ++c) x[c] = fma(x[c], a, b);
    T s = 0;
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) s += x[c];
    sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = (double)s;
}

// ---------------------------------------------------------------------------
// launch shapes
// ---------------------------------------------------------------------------
int default_tile(int n, bool xsec) {
    // Points per block tile.  amp2: four rounds of block/2^n points (keeps the
    // staged rows and records small); xsec: 128 points (half the threads
    // generate, three blocks fit an SM) up to n = 4, 64 at n = 5, 6 (the
    // generation spans two warps), then smaller tiles so that large-n grids
    // still cover every SM many times (a GB300 sweep of tiles and shapes).
    static const int amp2_tile[9] = {0, 0, 256, 128, 64, 32, 16, 8, 4};
    static const int xsec_tile[9] = {0, 0, 128, 128, 128, 64, 64, 32, 8};
    return xsec ? xsec_tile[n] : amp2_tile[n];
}

// heget_amp2 tiles of the subset recursion: larger than the tree's, so that
// more threads build the tile's records (FP64) at once and the recursion's
// per-call index tables and barriers are shared by more points (a GB300 sweep:
// FP32 +30 % at n = 6..8, +69 % at n = 5; FP64 a few per cent).
int subset_amp2_tile(int n, int precision) {
    static const int t32[9] = {0, 0, 256, 128, 128, 128, 64, 32, 32};
    static const int t64[9] = {0, 0, 256, 128, 64, 32, 32, 8, 8};
    return precision == HEGET_FP64 ? t64[n] : t32[n];
}

int xsec_shape_count(int n, int precision, int alg) {
    return precision == HEGET_FP32 && alg == kAlgTree && n >= 6 ? 4 : 1;
}

int default_amp_launch(int n, int precision, long long npts, int num_sms, AmpLaunch* L, bool xsec, int tile,
                       int alg, int shape) {
    L->shape = xsec && shape > 0 && shape < xsec_shape_count(n, precision, alg) ? shape : 0;
    // an explicit tile or shape selects the tile kernel
    L->ws = use_ws(n, precision, xsec, alg) && tile <= 0 && L->shape == 0;
    int bpsm = 1;
    size_t smem = 0;
    if (L->ws) {
        // warp-specialised: fixed stage size, one resident wave of blocks that
        // each pipeline many stages
        L->block = ws_consumers(n, alg, false) + ws_stage(n, alg);   // (the escalating kernel: more consumers)
        L->tile = ws_stage(n, alg);
        const int e = alg == kAlgSubset ? occupancy_ws_alg<kAlgSubset>(n, &bpsm, &smem)
                                        : occupancy_ws_alg<kAlgTree>(n, &bpsm, &smem);
        if (e) return e;
        if (bpsm < 1) bpsm = 1;
        L->smem = smem;
        const long long tiles = (npts + L->tile - 1) / L->tile;
        const long long wave = (long long)num_sms * bpsm;
        L->grid = (int)(tiles < wave ? (tiles < 1 ? 1 : tiles) : wave);
        return 0;
    }
    // xsec_block(): the FP32 tree's tile kernel at n = 6, 7 runs 160 / 224 threads
    L->block = xsec && precision == HEGET_FP32 && alg != kAlgSubset && (n == 6 || n == 7) ? (n == 6 ? 160 : 224)
                                                                                        : kBlockThreads;
    if (L->shape > 0) L->block = tree_tile_shape(n, L->shape).block;
    L->tile = tile > 0 ? tile : !xsec && alg == kAlgSubset ? subset_amp2_tile(n, precision) : default_tile(n, xsec);
    const bool sub = alg == kAlgSubset;
    const int e = precision == HEGET_FP32
                      ? (sub ? occupancy_alg<float, kAlgSubset>(n, L->tile, &bpsm, &smem)
                             : occupancy_alg<float, kAlgTree>(n, L->tile, &bpsm, &smem, L->shape))
                      : (sub ? occupancy_alg<double, kAlgSubset>(n, L->tile, &bpsm, &smem)
                             : occupancy_alg<double, kAlgTree>(n, L->tile, &bpsm, &smem));
    if (e) return e;
    if (bpsm < 1) bpsm = 1;
    L->smem = smem;
    const long long tiles = (npts + L->tile - 1) / L->tile;
    long long grid = tiles;
    const long long cap = (long long)kMaxGrid;
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    L->grid = (int)grid;
    return 0;
}

}  // namespace heget

using namespace heget;

namespace heget {

// Launch constants for n photons: couplings (4 pi alpha Q^2)^n, the event
// weight constant (1/2)(1/2^2)(1/3^2) 3 (1/n!) c_n (4 pi alpha Q^2)^n in fb
// (Sec. 2.1 eq. (2); Phi_n = c_n s^(n-2)), and the cut constants.
Physics physics_of(const heget_params& p, int n) {
    Physics ph{};
    ph.alpha = p.alpha;
    ph.q = p.q_charge;
    ph.pt_min = p.pt_min;
    ph.eta_max = p.eta_max;
    ph.dr_min = p.dr_min;
    const double g2 = 4.0 * M_PI * p.alpha * p.q_charge * p.q_charge;
    double cpl = 1, nfact = 1;
    for (int i = 0; i < n; ++i) cpl *= g2;
    for (int i = 2; i <= n; ++i) nfact *= i;
    ph.cpl = cpl;
    ph.wconst = cpl * phase_space_const(n) / (24.0 * nfact) * 0.3893793721e12;
    ph.sinh_eta = std::sinh(p.eta_max);
    ph.cosh_eta = std::cosh(p.eta_max);
    ph.sinh_dr = p.dr_min > 0 ? std::sinh(p.dr_min) : 0.0;
    ph.cos_dr = p.dr_min > 0 ? std::cos(p.dr_min) : 1.0;
    return ph;
}

Physics physics_of(const heget_ctx* c, int n) {
    Physics ph = physics_of(c->params, n);
    ph.alg = c->alg;
    ph.esc_tau = c->esc_tau;
    ph.hel_sample = c->hel_sample;
    return ph;
}

int check_sampler(const heget_sampler* s) {
    if (!s) return fail(HEGET_EINVAL, "sampler is NULL");
    switch (s->kind) {
        case HEGET_SAMPLER_FIXED:
            if (!(s->sqrt_s > 0) || !std::isfinite(s->sqrt_s)) return fail(HEGET_EINVAL, "sqrt_s must be > 0");
            return HEGET_OK;
        case HEGET_SAMPLER_UNIFORM:
            if (!(s->lo > 0) || !(s->hi >= s->lo) || !std::isfinite(s->hi))
                return fail(HEGET_EINVAL, "uniform sampler needs 0 < lo <= hi");
            return HEGET_OK;
        case HEGET_SAMPLER_TOY_PDF:
            if (!(s->e_beam > 0) || !(s->floor >= 0) || !(s->floor < 2 * s->e_beam))
                return fail(HEGET_EINVAL, "toy-PDF sampler needs e_beam > 0 and 0 <= floor < 2 e_beam");
            if (s->max_tries < 1 || s->max_tries > 64) return fail(HEGET_EINVAL, "max_tries must be in [1, 64]");
            return HEGET_OK;
        default:
            return fail(HEGET_EINVAL, "unknown sampler kind %d", s->kind);
    }
}

SamplerArgs sampler_args(const heget_sampler* s) {
    SamplerArgs a;
    a.kind = s->kind;
    a.max_tries = s->max_tries;
    a.sqrt_s = s->sqrt_s;
    a.lo = s->lo;
    a.hi = s->hi;
    a.e_beam = s->e_beam;
    a.floor = s->floor;
    // the FP32 product of the two uniforms' 24-bit estimates is within
    // 3 2^-24 of u_a u_b; 16 2^-24 on either side of the threshold is left to FP64
    const double c = s->kind == HEGET_SAMPLER_TOY_PDF ? s->floor / (2.0 * s->e_beam) : 0.0;
    a.band_lo = (float)(c - 16.0 * 0x1p-24);
    a.band_hi = (float)(c + 16.0 * 0x1p-24);
    return a;
}

int check_common(const heget_ctx* ctx, int n, long long N) {
    if (!ctx) return fail(HEGET_EINVAL, "context is NULL");
    if (n < kMinN || n > kMaxN) return fail(HEGET_EINVAL, "n = %d outside [2, 8]", n);
    if (N < 0) return fail(HEGET_EINVAL, "N = %lld < 0", N);
    return HEGET_OK;
}

int check_precision(int p) {
    if (p != HEGET_FP32 && p != HEGET_FP64) return fail(HEGET_EINVAL, "precision must be 32 or 64, got %d", p);
    return HEGET_OK;
}

int check_range(long long i0, long long N) {
    if (i0 < 0) return fail(HEGET_EINVAL, "i0 = %lld < 0", i0);
    if (N > 0 && i0 > LLONG_MAX - N) return fail(HEGET_EINVAL, "point indices i0 + N overflow int64");
    return HEGET_OK;
}

int check_params(const heget_params* p) {
    if (!(p->alpha > 0) || !std::isfinite(p->alpha) || !std::isfinite(p->q_charge) || p->q_charge == 0)
        return fail(HEGET_EINVAL, "alpha must be finite and > 0, q_charge finite and nonzero");
    if (!(p->pt_min >= 0) || !std::isfinite(p->pt_min) || !(p->eta_max > 0) || !std::isfinite(p->eta_max) ||
        std::isnan(p->dr_min))
        return fail(HEGET_EINVAL, "cuts need finite pt_min >= 0 and eta_max > 0, and dr_min not NaN");
    return HEGET_OK;
}
}  // namespace heget

namespace {
// Point tiles of one precision in one heget_xsec_batch call (a 96 MiB work
// list; 16.7 M points at n = 8, 537 M at n <= 4).
constexpr long long kMaxBatchTiles = 1ll << 22;

template <class R, int ALG>
size_t batch_tile_smem_t(int n, int tile) {
    switch (n) {
        case 2: return xsec_smem_bytes<R, 2, kBatchThreads, ALG>(tile);
        case 3: return xsec_smem_bytes<R, 3, kBatchThreads, ALG>(tile);
        case 4: return xsec_smem_bytes<R, 4, kBatchThreads, ALG>(tile);
        case 5: return xsec_smem_bytes<R, 5, kBatchThreads, ALG>(tile);
        case 6: return xsec_smem_bytes<R, 6, kBatchThreads, ALG>(tile);
        case 7: return xsec_smem_bytes<R, 7, kBatchThreads, ALG>(tile);
        default: return xsec_smem_bytes<R, 8, kBatchThreads, ALG>(tile);
    }
}

}  // namespace

namespace heget {
size_t batch_tile_smem(int n, int precision, int alg, int tile) {
    if (precision == HEGET_FP32)
        return alg == kAlgSubset ? batch_tile_smem_t<float, kAlgSubset>(n, tile) : batch_tile_smem_t<float, kAlgTree>(n, tile);
    return alg == kAlgSubset ? batch_tile_smem_t<double, kAlgSubset>(n, tile) : batch_tile_smem_t<double, kAlgTree>(n, tile);
}

int batch_default_tile(int n, int precision, int alg) {
    // subset recursion: the largest tile whose block (records, staging and
    // the recursion's tables) still lets two blocks share an SM, up to 128
    static const int sub32[9] = {0, 0, 128, 128, 128, 64, 64, 64, 64};
    static const int sub64[9] = {0, 0, 128, 128, 64, 16, 8, 8, 8};
    if (alg != kAlgSubset) return default_tile(n, true);
    return precision == HEGET_FP64 ? sub64[n] : sub32[n];
}
}  // namespace heget

namespace heget {
// Grows a workspace buffer to at least `need` bytes (device or pinned host).
int grow(void** p, size_t* cap, size_t need, bool pinned) {
    if (*cap >= need) return HEGET_OK;
    size_t c = *cap ? *cap : 4096;
    while (c < need) c *= 2;
    void* q = nullptr;
    cudaError_t e = pinned ? cudaMallocHost(&q, c) : cudaMalloc(&q, c);
    if (e != cudaSuccess) return fail(HEGET_ENOMEM, "workspace growth to %zu bytes failed: %s", c, cudaGetErrorString(e));
    if (*p) pinned ? cudaFreeHost(*p) : cudaFree(*p);
    *p = q;
    *cap = c;
    return HEGET_OK;
}
}  // namespace heget

namespace heget {
// Entries per block of the escalation lists: every point a block can own.
int escalation_cap(const AmpLaunch& L, long long N) {
    const long long tiles = (N + L.tile - 1) / L.tile;
    return (int)(((tiles + L.grid - 1) / L.grid) * L.tile);
}

int reserve_escalation(heget_ctx* ctx, const AmpLaunch& L, long long N) {
    const size_t entries = (size_t)L.grid * (size_t)escalation_cap(L, N);
    int r = grow((void**)&ctx->esc_idx, &ctx->esc_idx_cap, entries * sizeof(long long), false);
    if (!r) r = grow((void**)&ctx->esc_w, &ctx->esc_w_cap, entries * sizeof(double), false);
    if (!r) r = grow((void**)&ctx->esc_cnt, &ctx->esc_cnt_cap, (size_t)L.grid * sizeof(int), false);
    return r;
}
}  // namespace heget

extern "C" {

const char* heget_last_error(void) { return g_err.c_str(); }
const char* heget_version(void) { return "heget-gb300 0.1 (sm_103a)"; }

int heget_create(int device, heget_ctx** out) {
    if (!out) return fail(HEGET_EINVAL, "out is NULL");
    *out = nullptr;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= count) return fail(HEGET_EINVAL, "device %d not present (%d devices)", device, count);
    DeviceGuard g(device);
    heget_ctx* c = new heget_ctx();
    c->device = device;
    c->params = heget_params{1.0 / 137.035999, 2.0 / 3.0, 20.0, 2.5, 0.4};
    e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    // block partials of a launch, followed by those of its escalation launch
    if (e == cudaSuccess) e = cudaMalloc(&c->partials, 2 * sizeof(Partial) * (size_t)kMaxGrid);
    if (e == cudaSuccess) e = cudaMalloc(&c->amp_esc_count, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->amp_esc_count, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&c->flag, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->flag, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&c->res_dev, sizeof(heget_xsec_result));
    if (e == cudaSuccess) e = cudaMallocHost(&c->res_host, sizeof(heget_xsec_result));
    if (e != cudaSuccess) {
        heget_destroy(c);
        return cuda_fail(e, "heget_create");
    }
    *out = c;
    return HEGET_OK;
}

void heget_destroy(heget_ctx* c) {
    if (!c) return;
    DeviceGuard g(c->device);
    c->batch_graphs.release();
    if (c->batch_copied) cudaEventSynchronize(c->batch_copied), cudaEventDestroy(c->batch_copied);
    if (c->batch_host) cudaFreeHost(c->batch_host);
    if (c->batch_dev) cudaFree(c->batch_dev);
    if (c->batch_partials) cudaFree(c->batch_partials);
    if (c->partials) cudaFree(c->partials);
    if (c->esc_idx) cudaFree(c->esc_idx);
    if (c->esc_w) cudaFree(c->esc_w);
    if (c->esc_cnt) cudaFree(c->esc_cnt);
    if (c->amp_esc_list) cudaFree(c->amp_esc_list);
    if (c->amp_esc_count) cudaFree(c->amp_esc_count);
    if (c->flag) cudaFree(c->flag);
    if (c->res_dev) cudaFree(c->res_dev);
    if (c->res_host) cudaFreeHost(c->res_host);
    if (c->hist_parts) cudaFree(c->hist_parts);
    delete c;
}

int heget_set_tile(heget_ctx* ctx, int n, int precision, int kind, int tile) {
    if (!ctx) return fail(HEGET_EINVAL, "context is NULL");
    if (n < kMinN || n > kMaxN) return fail(HEGET_EINVAL, "n = %d outside [2, 8]", n);
    int r = check_precision(precision);
    if (r) return r;
    if (kind != 0 && kind != 1) return fail(HEGET_EINVAL, "kind must be 0 (amp2) or 1 (xsec)");
    const int unit = kBlockThreads >> n;
    if (tile < 0 || tile > 4096 || (tile > 0 && tile % unit != 0))
        return fail(HEGET_EINVAL, "tile %d must be 0 or a multiple of %d up to 4096", tile, unit);
    ctx->tiles[kind][precision == HEGET_FP64][n] = tile;
    return HEGET_OK;
}

int heget_set_shape(heget_ctx* ctx, int n, int precision, int shape) {
    if (!ctx) return fail(HEGET_EINVAL, "context is NULL");
    if (n < kMinN || n > kMaxN) return fail(HEGET_EINVAL, "n = %d outside [2, 8]", n);
    int r = check_precision(precision);
    if (r) return r;
    const int ns = xsec_shape_count(n, precision, kAlgTree);
    if (shape < 0 || shape >= ns) return fail(HEGET_EINVAL, "shape %d: n = %d has shapes 0 .. %d", shape, n, ns - 1);
    ctx->shapes[precision == HEGET_FP64][n] = shape;
    return HEGET_OK;
}

int heget_get_shape(const heget_ctx* ctx, int n, int precision) {
    if (!ctx || n < kMinN || n > kMaxN || (precision != HEGET_FP32 && precision != HEGET_FP64)) return -1;
    return ctx->shapes[precision == HEGET_FP64][n];
}

int heget_shape_info(int n, int precision, int shape, int* threads, int* rows_per_lane, int* groups) {
    if (!threads || !rows_per_lane || !groups) return fail(HEGET_EINVAL, "NULL argument");
    if (n < kMinN || n > kMaxN) return fail(HEGET_EINVAL, "n = %d outside [2, 8]", n);
    int r = check_precision(precision);
    if (r) return r;
    if (shape < 0 || shape >= xsec_shape_count(n, precision, kAlgTree))
        return fail(HEGET_EINVAL, "no shape %d at n = %d", shape, n);
    if (shape == 0) {   // the default: warp-specialised or the tile kernel's default
        *threads = 0;
        *rows_per_lane = 0;
        *groups = 0;
        return HEGET_OK;
    }
    const TileShape t = tree_tile_shape(n, shape);
    *threads = t.block;
    *rows_per_lane = 1 << t.hb;
    *groups = t.g;
    return HEGET_OK;
}

int heget_set_graphs(heget_ctx* ctx, int on) {
    if (!ctx) return fail(HEGET_EINVAL, "context is NULL");
    if (on != 0 && on != 1) return fail(HEGET_EINVAL, "graphs must be 0 or 1, got %d", on);
    DeviceGuard g(ctx->device);
    if (!on) ctx->batch_graphs.clear();
    ctx->graphs = on;
    return HEGET_OK;
}

int heget_get_graphs(const heget_ctx* ctx, int64_t* captures, int64_t* replays) {
    if (!ctx) return -1;
    if (captures) *captures = ctx->batch_graphs.captures;
    if (replays) *replays = ctx->batch_graphs.replays;
    return ctx->graphs;
}

int heget_set_algorithm(heget_ctx* ctx, int alg) {
    if (!ctx) return fail(HEGET_EINVAL, "context is NULL");
    if (alg != HEGET_ALG_TREE && alg != HEGET_ALG_SUBSET) return fail(HEGET_EINVAL, "unknown algorithm %d", alg);
    ctx->alg = alg;
    return HEGET_OK;
}

int heget_get_algorithm(const heget_ctx* ctx) { return ctx ? ctx->alg : -1; }

int heget_set_helicity_sampling(heget_ctx* ctx, int on) {
    if (!ctx) return fail(HEGET_EINVAL, "context is NULL");
    if (on != 0 && on != 1) return fail(HEGET_EINVAL, "helicity sampling must be 0 or 1, got %d", on);
    ctx->hel_sample = on;
    return HEGET_OK;
}

int heget_get_helicity_sampling(const heget_ctx* ctx) { return ctx ? ctx->hel_sample : -1; }

int heget_set_escalation(heget_ctx* ctx, double tau) {
    if (!ctx) return fail(HEGET_EINVAL, "context is NULL");
    if (!(tau >= 0) || !std::isfinite(tau)) return fail(HEGET_EINVAL, "tau must be finite and >= 0");
    ctx->esc_tau = tau;
    return HEGET_OK;
}

int heget_get_escalation(const heget_ctx* ctx, double* tau) {
    if (!ctx || !tau) return fail(HEGET_EINVAL, "NULL argument");
    *tau = ctx->esc_tau;
    return HEGET_OK;
}

int heget_amp2_escalated(heget_ctx* ctx, void* stream, int64_t* count) {
    if (!ctx || !count) return fail(HEGET_EINVAL, "NULL argument");
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, ctx->amp_esc_count, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "heget_amp2_escalated");
    *count = h;
    return HEGET_OK;
}

int heget_get_tile(const heget_ctx* ctx, int n, int precision, int kind) {
    if (!ctx || n < kMinN || n > kMaxN || (kind != 0 && kind != 1)) return -1;
    const int t = ctx->tiles[kind][precision == HEGET_FP64][n];
    if (t > 0) return t;
    return kind == 0 && ctx->alg == kAlgSubset ? subset_amp2_tile(n, precision) : default_tile(n, kind == 1);
}

int heget_set_params(heget_ctx* ctx, const heget_params* p) {
    if (!ctx || !p) return fail(HEGET_EINVAL, "NULL argument");
    int r = check_params(p);
    if (r) return r;
    ctx->params = *p;
    return HEGET_OK;
}

int heget_get_params(const heget_ctx* ctx, heget_params* p) {
    if (!ctx || !p) return fail(HEGET_EINVAL, "NULL argument");
    *p = ctx->params;
    return HEGET_OK;
}

int heget_phase_space_ex(heget_ctx* ctx, uint64_t seed, int64_t i0, int64_t N, int n, const heget_sampler* smp,
                         double* momenta, double* weights, double* sqrt_s_out, double* y_out, uint8_t* mask_out,
                         int32_t* tries_out, void* stream) {
    int r = check_common(ctx, n, N);
    if (r) return r;
    if ((r = check_sampler(smp))) return r;
    if ((r = check_range(i0, N))) return r;
    if (N == 0) return HEGET_OK;
    DeviceGuard g(ctx->device);
    const SamplerArgs S = sampler_args(smp);
    const Physics ph = physics_of(ctx, n);
    cudaStream_t st = (cudaStream_t)stream;
    const long long blocks_needed = (N + kPsBlock - 1) / kPsBlock;
    const int grid = (int)(blocks_needed < kMaxGrid ? blocks_needed : kMaxGrid);
#define PS(NN) \
    phase_space_kernel<NN><<<grid, kPsBlock, 0, st>>>(seed, i0, N, S, ph, momenta, weights, sqrt_s_out, y_out, mask_out, tries_out)
    switch (n) {
        case 2: PS(2); break;
        case 3: PS(3); break;
        case 4: PS(4); break;
        case 5: PS(5); break;
        case 6: PS(6); break;
        case 7: PS(7); break;
        case 8: PS(8); break;
    }
#undef PS
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "phase_space_kernel");
    return HEGET_OK;
}

int heget_phase_space(heget_ctx* ctx, uint64_t seed, int64_t N, int n, double sqrt_s, double* momenta,
                      double* weights, void* stream) {
    heget_sampler s{HEGET_SAMPLER_FIXED, sqrt_s, 0, 0, 7000.0, 100.0, 64};
    return heget_phase_space_ex(ctx, seed, 0, N, n, &s, momenta, weights, nullptr, nullptr, nullptr, nullptr, stream);
}

int heget_amp2(heget_ctx* ctx, int n, int64_t N, const double* momenta, const uint32_t* hel_mask, int precision,
               double* amp2, void* stream) {
    int r = check_common(ctx, n, N);
    if (r) return r;
    if ((r = check_precision(precision))) return r;
    if (N == 0) return HEGET_OK;
    if (!momenta || !amp2) return fail(HEGET_EINVAL, "momenta and amp2 must be non-NULL");
    if (((uintptr_t)momenta & 15) != 0) return fail(HEGET_EINVAL, "momenta must be 16-byte aligned");
    DeviceGuard g(ctx->device);
    AmpLaunch L;
    if ((r = default_amp_launch(n, precision, N, ctx->num_sms, &L, false, ctx->tiles[0][precision == HEGET_FP64][n],
                                ctx->alg)))
        return cuda_fail((cudaError_t)r, "occupancy");
    const Physics ph = physics_of(ctx, n);
    cudaStream_t st = (cudaStream_t)stream;
    const bool esc = precision == HEGET_FP32 && ctx->esc_tau > 0 && N <= INT32_MAX;
    if (esc) {
        if ((r = grow((void**)&ctx->amp_esc_list, &ctx->amp_esc_cap, sizeof(int) * (size_t)N, false))) return r;
        const cudaError_t e = cudaMemsetAsync(ctx->amp_esc_count, 0, sizeof(int), st);
        if (e != cudaSuccess) return cuda_fail(e, "escalation counter");
    }
    r = precision == HEGET_FP32
            ? launch_amp2_f32(n, momenta, N, hel_mask, amp2, ph, ctx->flag, esc ? ctx->amp_esc_list : nullptr,
                              esc ? ctx->amp_esc_count : nullptr, L, st)
            : launch_amp2_f64(n, momenta, N, hel_mask, amp2, ph, ctx->flag, nullptr, nullptr, L, st);
    if (r) return cuda_fail((cudaError_t)r, "amp2_kernel");
    if (esc) {
        // the flagged rows in FP64 (grid-stride over the device-side count)
        const int tile = ctx->tiles[0][1][n] > 0 ? ctx->tiles[0][1][n] : default_tile(n, false);
        r = launch_amp2_list_f64(n, momenta, ctx->amp_esc_list, ctx->amp_esc_count, hel_mask, amp2, ph, ctx->flag,
                                 tile, 2 * ctx->num_sms, st);
        if (r) return cuda_fail((cudaError_t)r, "amp2_list_kernel");
    }
    return HEGET_OK;
}

int heget_ward(heget_ctx* ctx, int n, int64_t N, const double* momenta, int photon, int precision, double* ratio,
               void* stream) {
    int r = check_common(ctx, n, N);
    if (r) return r;
    if ((r = check_precision(precision))) return r;
    if (photon < 0 || photon >= n) return fail(HEGET_EINVAL, "photon must be in [0, n)");
    if (N == 0) return HEGET_OK;
    if (!momenta || !ratio) return fail(HEGET_EINVAL, "momenta and ratio must be non-NULL");
    if (((uintptr_t)momenta & 15) != 0) return fail(HEGET_EINVAL, "momenta must be 16-byte aligned");
    DeviceGuard g(ctx->device);
    AmpLaunch L;
    if ((r = default_amp_launch(n, precision, N, ctx->num_sms, &L, false, ctx->tiles[0][precision == HEGET_FP64][n])))
        return cuda_fail((cudaError_t)r, "occupancy");
    const Physics ph = physics_of(ctx, n);
    cudaStream_t st = (cudaStream_t)stream;
    r = precision == HEGET_FP32 ? launch_ward_f32(n, momenta, N, photon, ratio, ph, ctx->flag, L, st)
                                : launch_ward_f64(n, momenta, N, photon, ratio, ph, ctx->flag, L, st);
    if (r) return cuda_fail((cudaError_t)r, "ward_kernel");
    return HEGET_OK;
}

int heget_log_table(const double* x, double* y, int64_t N, void* stream) {
    if (N < 0) return fail(HEGET_EINVAL, "N < 0");
    if (N == 0) return HEGET_OK;
    if (!x || !y) return fail(HEGET_EINVAL, "x and y must be non-NULL");
    const long long blocks = std::min<long long>((N + 255) / 256, 65536);
    log_table_kernel<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(x, y, N);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "log_table_kernel");
    return HEGET_OK;
}

int heget_sincos_2pi(const uint32_t* words, double* cs, int64_t N, void* stream) {
    if (N < 0) return fail(HEGET_EINVAL, "N < 0");
    if (N == 0) return HEGET_OK;
    if (!words || !cs) return fail(HEGET_EINVAL, "words and cs must be non-NULL");
    const long long blocks = std::min<long long>((N + 255) / 256, 65536);
    sincos_kernel<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(words, cs, N);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "sincos_kernel");
    return HEGET_OK;
}

int heget_f32_round(const double* x, float* y, int64_t N, void* stream) {
    if (N < 0) return fail(HEGET_EINVAL, "N < 0");
    if (N == 0) return HEGET_OK;
    if (!x || !y) return fail(HEGET_EINVAL, "x and y must be non-NULL");
    const long long blocks = std::min<long long>((N + 255) / 256, 65536);
    f32_round_kernel<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(x, y, N);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "f32_round_kernel");
    return HEGET_OK;
}

int heget_check(heget_ctx* ctx, void* stream) {
    if (!ctx) return fail(HEGET_EINVAL, "context is NULL");
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, ctx->flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "heget_check");
    if (h) {
        e = cudaMemsetAsync(ctx->flag, 0, sizeof(int), st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "heget_check reset");
        return fail(HEGET_EINVAL, "input check failed: non-finite momenta, or p1/p2 not massless along +z/-z");
    }
    return HEGET_OK;
}


int heget_xsec_launch(heget_ctx* ctx, int n, uint64_t seed, int64_t i0, int64_t N, const heget_sampler* smp,
                      int precision, double* w_out, void* stream) {
    int r = check_common(ctx, n, N);
    if (r) return r;
    if ((r = check_precision(precision))) return r;
    if ((r = check_sampler(smp))) return r;
    if ((r = check_range(i0, N))) return r;
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    AmpLaunch L;
    if ((r = default_amp_launch(n, precision, N > 0 ? N : 1, ctx->num_sms, &L, true, ctx->tiles[1][precision == HEGET_FP64][n],
                                ctx->alg, ctx->shapes[precision == HEGET_FP64][n])))
        return cuda_fail((cudaError_t)r, "occupancy");
    const Physics ph = physics_of(ctx, n);
    const SamplerArgs S = sampler_args(smp);
    EscArgs esc{nullptr, nullptr, nullptr, 0, 0};
    const bool escalate = precision == HEGET_FP32 && ctx->esc_tau > 0 && N > 0;
    if (escalate) {
        if ((r = reserve_escalation(ctx, L, N))) return r;
        esc = EscArgs{ctx->esc_idx, ctx->esc_w, ctx->esc_cnt, escalation_cap(L, N), 0};
    }
    if (N > 0) {
        r = precision == HEGET_FP32 ? launch_xsec_f32(n, seed, i0, N, S, ph, ctx->partials, w_out, esc, L, st)
                                    : launch_xsec_f64(n, seed, i0, N, S, ph, ctx->partials, w_out, esc, L, st);
        if (r) return cuda_fail((cudaError_t)r, "xsec_kernel");
    }
    if (escalate) {
        // FP64 recomputation of the flagged points (by the subset recursion,
        // whatever the context's algorithm: the same |M|^2, far cheaper at
        // large n); its partials follow the FP32 ones
        r = launch_escalate_f64(n, seed, i0, S, ph, default_tile(n, true), esc, ctx->partials + L.grid, w_out,
                                L.grid, st);
        if (r) return cuda_fail((cudaError_t)r, "xsec_escalate_kernel");
    }
    ctx->last_parts = N > 0 ? (escalate ? 2 * L.grid : L.grid) : 0;
    ctx->last_kind = S.kind;
    ctx->last_ws = L.ws;
    ctx->last_esc = escalate;
    return HEGET_OK;
}

int heget_xsec_finalize(heget_ctx* ctx, heget_xsec_result* result_dev, void* stream) {
    if (!ctx) return fail(HEGET_EINVAL, "context is NULL");
    if (!result_dev) return fail(HEGET_EINVAL, "result_dev is NULL");
    DeviceGuard g(ctx->device);
    finalize_kernel<<<1, 256, 0, (cudaStream_t)stream>>>(ctx->partials, ctx->last_parts, ctx->last_kind, 0,
                                                         result_dev, nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "finalize_kernel");
    return HEGET_OK;
}

int heget_xsec_async(heget_ctx* ctx, int n, uint64_t seed, int64_t i0, int64_t N, const heget_sampler* smp,
                     int precision, heget_xsec_result* result_dev, double* w_out, void* stream) {
    if (!result_dev) return fail(HEGET_EINVAL, "result_dev is NULL");
    int r = heget_xsec_launch(ctx, n, seed, i0, N, smp, precision, w_out, stream);
    if (r) return r;
    return heget_xsec_finalize(ctx, result_dev, stream);
}

int heget_measure_fma_peak(heget_ctx* ctx, int precision, double* tflops) {
    if (!ctx || !tflops) return fail(HEGET_EINVAL, "NULL argument");
    int r = check_precision(precision);
    if (r) return r;
    DeviceGuard g(ctx->device);
    const int blocks = ctx->num_sms * 8, threads = 256;
    const int iters = precision == HEGET_FP32 ? 1024 : 256;
    double* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&sink, sizeof(double) * blocks * threads);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best_ms = 1e30f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        cudaEventRecord(e0);
        if (precision == HEGET_FP32)
            fma_peak_kernel<float><<<blocks, threads>>>(iters, sink);
        else
            fma_peak_kernel<double><<<blocks, threads>>>(iters, sink);
        cudaEventRecord(e1);
        e = cudaEventSynchronize(e1);
        float ms = 0;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best_ms) best_ms = ms;   // rep 0 is warm-up
    }
    if (sink) cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "heget_measure_fma_peak");
    const double fmas = (double)blocks * threads * iters * kPeakChains;
    *tflops = 2.0 * fmas / (best_ms * 1e-3) / 1e12;
    return HEGET_OK;
}

int heget_xsec(heget_ctx* ctx, int n, int64_t N, uint64_t seed, const heget_sampler* smp, int precision,
               heget_xsec_result* out, void* stream) {
    if (!out) return fail(HEGET_EINVAL, "out is NULL");
    if (!ctx) return fail(HEGET_EINVAL, "context is NULL");
    int r = heget_xsec_async(ctx, n, seed, 0, N, smp, precision, ctx->res_dev, nullptr, stream);
    if (r) return r;
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(ctx->res_host, ctx->res_dev, sizeof(heget_xsec_result), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "heget_xsec");
    *out = *ctx->res_host;
    return HEGET_OK;
}

int heget_xsec_combine(const heget_xsec_result* parts, int nparts, int sampler_kind, heget_xsec_result* out) {
    if (!out || nparts < 0 || (nparts > 0 && !parts)) return fail(HEGET_EINVAL, "NULL argument or nparts < 0");
    if (sampler_kind != HEGET_SAMPLER_FIXED && sampler_kind != HEGET_SAMPLER_UNIFORM &&
        sampler_kind != HEGET_SAMPLER_TOY_PDF)
        return fail(HEGET_EINVAL, "unknown sampler kind %d", sampler_kind);
    DD sw{0, 0}, sw2{0, 0};   // (running sum, accumulated TwoSum errors)
    long long npass = 0, ntotal = 0, ntries = 0, nesc = 0;
    for (int k = 0; k < nparts; ++k) {
        double t, e;
        two_sum(sw.hi, parts[k].sum_w, t, e);
        sw.hi = t;
        sw.lo += e;
        two_sum(sw2.hi, parts[k].sum_w2, t, e);
        sw2.hi = t;
        sw2.lo += e;
        npass += parts[k].n_pass;
        ntotal += parts[k].n_total;
        ntries += parts[k].n_tries;
        nesc += parts[k].n_escalated;
    }
    // the formulas of finalize_block (the device's summation step)
    const double s = sw.hi + sw.lo, s2 = sw2.hi + sw2.lo;
    const double N = (double)ntotal;
    const double mean = N > 0 ? s / N : 0.0;
    const double var = N > 1 ? std::fmax(0.0, (s2 - s * mean) / (N - 1.0)) : 0.0;
    const double accept = ntries > 0 ? N / (double)ntries : 1.0;
    const double scale = sampler_kind == HEGET_SAMPLER_TOY_PDF ? 2.0 * accept : 1.0;
    heget_xsec_result o{};
    o.sigma_fb = scale * mean;
    o.err_fb = N > 0 ? scale * std::sqrt(var / N) : 0.0;
    o.sum_w = s;
    o.sum_w2 = s2;
    o.accept = accept;
    o.n_pass = npass;
    o.n_total = ntotal;
    o.n_tries = ntries;
    o.n_escalated = nesc;
    *out = o;
    return HEGET_OK;
}

int heget_hist_combine(const double* const* parts, int nparts, int64_t len, double* out) {
    if (!out || nparts < 0 || len < 0 || (nparts > 0 && !parts)) return fail(HEGET_EINVAL, "bad argument");
    for (int k = 0; k < nparts; ++k)
        if (!parts[k] && len > 0) return fail(HEGET_EINVAL, "part %d is NULL", k);
    for (int64_t i = 0; i < len; ++i) {
        double hi = 0.0, lo = 0.0;
        for (int k = 0; k < nparts; ++k) {
            double sum, err;
            two_sum(hi, parts[k][i], sum, err);
            hi = sum;
            lo += err;
        }
        out[i] = hi + lo;
    }
    return HEGET_OK;
}

int heget_sum(heget_ctx* ctx, const double* x, int64_t N, double* out_dev, void* stream) {
    if (!ctx || !out_dev) return fail(HEGET_EINVAL, "NULL argument");
    if (N < 0) return fail(HEGET_EINVAL, "N < 0");
    if (N > 0 && !x) return fail(HEGET_EINVAL, "x is NULL");
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    long long blocks = (N + 255) / 256;
    const int grid = (int)(blocks < 1 ? 1 : (blocks < 4 * ctx->num_sms ? blocks : 4 * ctx->num_sms));
    if (N > 0) sum_kernel<<<grid, 256, 0, st>>>(x, N, ctx->partials);
    finalize_kernel<<<1, 256, 0, st>>>(ctx->partials, N > 0 ? grid : 0, 0, 1, nullptr, out_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "heget_sum");
    return HEGET_OK;
}

}  // extern "C"


extern "C" int heget_xsec_batch(heget_ctx* ctx, const heget_xsec_request* reqs, int count, void* stream) {
    if (!ctx) return fail(HEGET_EINVAL, "context is NULL");
    if (count < 0 || (count > 0 && !reqs)) return fail(HEGET_EINVAL, "bad request array");
    for (int i = 0; i < count; ++i) {
        const heget_xsec_request& q = reqs[i];
        int r = check_common(ctx, q.n, q.N);
        if (!r) r = check_precision(q.precision);
        if (!r) r = check_sampler(&q.sampler);
        if (!r) r = check_range(q.i0, q.N);
        if (r) return fail(r, "request %d: %s", i, heget_last_error());
        if (!q.result_dev) return fail(HEGET_EINVAL, "request %d: result_dev is NULL", i);
    }
    {   // the work list is staged on the host: bound its length before building it
        long long tiles[2] = {0, 0};
        for (int i = 0; i < count; ++i) {
            const heget_xsec_request& q = reqs[i];
            const int tile_o = ctx->tiles[1][q.precision == HEGET_FP64][q.n];
            const long long tile = tile_o > 0 ? tile_o : batch_default_tile(q.n, q.precision, ctx->alg);
            tiles[q.precision == HEGET_FP64] += (q.N + tile - 1) / tile;
            if (tiles[0] > kMaxBatchTiles || tiles[1] > kMaxBatchTiles)
                return fail(HEGET_EINVAL, "batch needs more than %lld point tiles per precision: split it",
                            (long long)kMaxBatchTiles);
        }
    }
    if (count == 0) return HEGET_OK;
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if (!ctx->batch_copied) {
        e = cudaEventCreateWithFlags(&ctx->batch_copied, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
    }
    for (int prec : {HEGET_FP32, HEGET_FP64}) {
        std::vector<BatchReq> br;
        std::vector<WorkItem> items;
        size_t smem = 0;
        for (int i = 0; i < count; ++i) {
            const heget_xsec_request& q = reqs[i];
            if (q.precision != prec) continue;
            const int tile_o = ctx->tiles[1][prec == HEGET_FP64][q.n];
            const int tile = tile_o > 0 ? tile_o : batch_default_tile(q.n, prec, ctx->alg);
            BatchReq b{};
            b.seed = q.seed;
            b.i0 = q.i0;
            b.S = sampler_args(&q.sampler);
            b.ph = physics_of(ctx, q.n);
            b.w_out = q.w_out;
            b.result = q.result_dev;
            b.n = q.n;
            b.tile = tile;
            b.parts = nullptr;   // set once the partial buffer is sized
            b.pad = (int)items.size();   // first item, until then
            for (long long start = 0; start < q.N; start += tile)
                items.push_back(WorkItem{(int)br.size(), q.n, (int)std::min<long long>(tile, q.N - start), 0, start});
            b.ntiles = (int)items.size() - b.pad;
            br.push_back(b);
            const size_t sm = batch_tile_smem(q.n, prec, ctx->alg, tile);
            smem = std::max(smem, sm);
        }
        if (br.empty()) continue;
        const size_t items_bytes = align16(items.size() * sizeof(WorkItem));
        const size_t bytes = items_bytes + br.size() * sizeof(BatchReq);
        // the previous batch's upload must have left the staging area
        e = cudaEventSynchronize(ctx->batch_copied);
        if (e != cudaSuccess) return cuda_fail(e, "batch staging");
        int r = grow((void**)&ctx->batch_host, &ctx->batch_cap, bytes, true);
        if (r) return r;
        const size_t dcap = ctx->batch_cap;   // device buffer mirrors the pinned one
        if (!ctx->batch_dev || dcap > ctx->batch_dev_cap) {
            ctx->batch_graphs.clear();   // their arguments point into the old buffers
            if (ctx->batch_dev) cudaFree(ctx->batch_dev);
            e = cudaMalloc(&ctx->batch_dev, dcap);
            if (e != cudaSuccess) return fail(HEGET_ENOMEM, "batch workspace: %s", cudaGetErrorString(e));
            ctx->batch_dev_cap = dcap;
        }
        {
            Partial* before = ctx->batch_partials;
            r = grow((void**)&ctx->batch_partials, &ctx->batch_partials_cap, items.size() * sizeof(Partial), false);
            if (r) return r;
            if (before != ctx->batch_partials) ctx->batch_graphs.clear();   // (the request table points there)
        }
        for (auto& b : br) {
            b.parts = ctx->batch_partials + b.pad;
            b.pad = 0;
        }
        std::memcpy(ctx->batch_host, items.data(), items.size() * sizeof(WorkItem));
        std::memcpy(ctx->batch_host + items_bytes, br.data(), br.size() * sizeof(BatchReq));
        e = cudaMemcpyAsync(ctx->batch_dev, ctx->batch_host, bytes, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->batch_copied, st);
        if (e != cudaSuccess) return cuda_fail(e, "batch upload");
        const WorkItem* items_d = reinterpret_cast<const WorkItem*>(ctx->batch_dev);
        const BatchReq* reqs_d = reinterpret_cast<const BatchReq*>(ctx->batch_dev + items_bytes);
        const int nitems = (int)items.size();
        const int grid = std::max(1, std::min(nitems, 8 * ctx->num_sms));
        const int nreq = (int)br.size();
        auto launch = [&](cudaStream_t s2, bool set_attr) {
            int rr = prec == HEGET_FP32 ? launch_batch_f32(items_d, nitems, reqs_d, smem, grid, ctx->alg, s2, set_attr)
                                        : launch_batch_f64(items_d, nitems, reqs_d, smem, grid, ctx->alg, s2, set_attr);
            if (!rr) rr = launch_batch_finalize(reqs_d, nreq, s2);
            return rr;
        };
        if (ctx->graphs) {
            // the kernel's shared-memory attribute is set outside the capture
            r = prec == HEGET_FP32 ? prepare_batch_f32(smem, ctx->alg) : prepare_batch_f64(smem, ctx->alg);
            if (!r)
                r = ctx->batch_graphs.run(BatchGraphKey{prec, ctx->alg, nitems, nreq, grid, smem, items_d, reqs_d, reqs_d}, st,
                                          [&](cudaStream_t s2) { return launch(s2, false); });
        } else {
            r = launch(st, true);
        }
        if (r) return cuda_fail((cudaError_t)r, "xsec_batch_kernel");
        // the next precision's batch reuses the workspace: keep the order
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "heget_xsec_batch");
    }
    return HEGET_OK;
}

// ---------------------------------------------------------------------------
// heget_xsec_noalloc: the cross section without any device allocation.
//
// Its only scratch -- the per-block partial sums that heget_xsec_async keeps
// in the context workspace -- lives in the file-scope array below, which
// every GPU that loads this library holds until the process exits.  Host
// code cannot hand the array's name to a kernel (in host code it names a
// host-side stand-in), so the first call on each device looks up the device
// address with cudaGetSymbolAddress while that device is current and caches
// it together with the CUDA context that was current then.  The address
// belongs to that context: a later call under another context of the same
// device (after cudaDeviceReset, or from a context the caller made current
// through the driver API) looks it up again instead of reusing a stale
// address.  Each call's blocks overwrite exactly the entries its own finalize
// reads, so nothing has to be cleared between calls.
// ---------------------------------------------------------------------------
namespace {
constexpr int kNoAllocMaxBlocks = 4096;   // 4096 partials x 64 B = 256 KiB per device
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) Partial g_noalloc_partials[kNoAllocMaxBlocks];

std::mutex g_noalloc_mu;
struct NoAllocSlot {
    void* ctx;        // the CUDA context current when ptr was looked up
    Partial* ptr;
};
NoAllocSlot g_noalloc_slot[kNoAllocMaxDevices] = {};

// The calling thread's current CUDA context (cuCtxGetCurrent, reached through
// the runtime's driver entry points so that the library needs no link to the
// driver library), or nullptr when there is none or it cannot be queried.
void* current_context() {
    using GetCurrent = int (*)(void**);
    static GetCurrent fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return (GetCurrent) nullptr;
        }
        return reinterpret_cast<GetCurrent>(f);
    }();
    void* c = nullptr;
    if (!fn || fn(&c) != 0) return nullptr;
    return c;
}

int noalloc_scratch(int device, Partial** out) {
    if (device < 0 || device >= kNoAllocMaxDevices) return fail(HEGET_EINVAL, "device %d out of range", device);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoAllocSlot& s = g_noalloc_slot[device];
    void* ctx = current_context();
    if (!s.ptr || !ctx || ctx != s.ctx) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);   // caller made `device` current
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-allocation scratch)");
        s.ptr = static_cast<Partial*>(p);
        s.ctx = current_context();   // the lookup made the primary context current if none was
    }
    *out = s.ptr;
    return HEGET_OK;
}
}  // namespace

extern "C" int heget_xsec_noalloc(int device, int n, uint64_t seed, int64_t i0, int64_t N,
                                  const heget_sampler* smp, const heget_params* params, int precision,
                                  heget_xsec_result* result_dev, void* stream) {
    if (n < kMinN || n > kMaxN) return fail(HEGET_EINVAL, "n = %d outside [2, 8]", n);
    if (N < 0) return fail(HEGET_EINVAL, "N = %lld < 0", (long long)N);
    int r = check_range(i0, N);
    if (r) return r;
    if ((r = check_precision(precision))) return r;
    if ((r = check_sampler(smp))) return r;
    if (!result_dev) return fail(HEGET_EINVAL, "result_dev is NULL");
    const heget_params p = params ? *params : heget_params{1.0 / 137.035999, 2.0 / 3.0, 20.0, 2.5, 0.4};
    if ((r = check_params(&p))) return r;   // the same refusals as heget_set_params
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= count) return fail(HEGET_EINVAL, "device %d not present", device);
    DeviceGuard g(device);
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    AmpLaunch L;
    // the default launch of heget_xsec_async (the tree): the warp-specialised
    // kernel in FP32 up to n = 5 (one resident wave, any N), else the tile
    // kernel with its default tile, whose grid bounds N
    if ((r = default_amp_launch(n, precision, N > 0 ? N : 1, sms, &L, true, 0)))
        return cuda_fail((cudaError_t)r, "occupancy");
    if (N > 0 && L.grid > kNoAllocMaxBlocks)
        return fail(HEGET_EINVAL,
                    "N = %lld needs %d block partials; the no-allocation path holds %d (N <= %lld at n = %d)",
                    (long long)N, L.grid, kNoAllocMaxBlocks, (long long)kNoAllocMaxBlocks * L.tile, n);
    Partial* scratch = nullptr;
    if ((r = noalloc_scratch(device, &scratch))) return r;
    const Physics ph = physics_of(p, n);
    const SamplerArgs S = sampler_args(smp);
    cudaStream_t st = (cudaStream_t)stream;
    if (N > 0) {
        const EscArgs no_esc{nullptr, nullptr, nullptr, 0, 0};
        r = precision == HEGET_FP32 ? launch_xsec_f32(n, seed, i0, N, S, ph, scratch, nullptr, no_esc, L, st)
                                    : launch_xsec_f64(n, seed, i0, N, S, ph, scratch, nullptr, no_esc, L, st);
        if (r) return cuda_fail((cudaError_t)r, "xsec_kernel");
    }
    finalize_kernel<<<1, 256, 0, st>>>(scratch, N > 0 ? L.grid : 0, S.kind, 0, result_dev, nullptr);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "finalize_kernel");
    return HEGET_OK;
}
