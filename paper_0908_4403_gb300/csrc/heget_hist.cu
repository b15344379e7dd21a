// heget_hist.cu -- kinematic distributions (Sec. 5, Fig. 2): weighted
// histograms of photon observables of the generated events.  The events are
// regenerated from the counter-based generator; every block sums each tile's
// entries per bin in a fixed order and folds the tile sums into double-double
// bin sums, and the block partials are combined in block order, so results
// are reproducible bit for bit for a given launch shape (one resident wave,
// set by the GPU).
#include <algorithm>
#include <cmath>

#include "heget_kernels.cuh"
#include "heget_internal.h"

namespace heget {
namespace {

constexpr int kHistBlock = 128;   // points per block tile, one per thread

struct HistSpecDev {
    int kind, nbins, off, pad;   // off: first bin of this histogram in the block's bin array
    double lo, scale;            // scale = nbins / (hi - lo), formed on the host
};

struct HistArgs {
    HistSpecDev spec[HEGET_HIST_MAX_SPECS];
    int nspec, total;
};

// Bin of x: 0 below lo (and NaN), nbins + 1 at or above hi, else
// 1 + floor((x - lo) scale), in FP64 without contraction.
__device__ __forceinline__ int hist_bin(double x, const HistSpecDev& h) {
    if (!(x >= h.lo)) return 0;
    const double t = __dmul_rn(__dsub_rn(x, h.lo), h.scale);
    if (t >= (double)h.nbins) return h.nbins + 1;
    return 1 + (int)t;
}

__host__ __device__ constexpr int hist_entries_max(int n) {
    return n * (n - 1) / 2 > n ? n * (n - 1) / 2 : n;
}

__host__ __device__ constexpr size_t hist_smem_bytes(int n, int total) {
    return (size_t)n * kMomSlots * kHistBlock * sizeof(double)   // momenta, then photon observables
           + 2 * (size_t)total * sizeof(DD)                          // bin sums of w and w^2
           + 2 * (size_t)kHistBlock * sizeof(double)                 // weights, sqrt(s-hat)
           + (size_t)hist_entries_max(n) * kHistBlock * sizeof(short);   // bins of the entries
}

template <int N>
__global__ void __launch_bounds__(kHistBlock)
hist_kernel(uint64_t seed, long long i0, long long npts, SamplerArgs S, Physics ph,
            const double* __restrict__ w, HistArgs H, double* __restrict__ parts) {
    constexpr int NP = N * (N - 1) / 2;
    constexpr int E = hist_entries_max(N);
    extern __shared__ __align__(16) unsigned char smem[];
    double* stage = reinterpret_cast<double*>(smem);
    DD* hw = reinterpret_cast<DD*>(stage + (size_t)N * kMomSlots * kHistBlock);
    DD* hw2 = hw + H.total;
    double* wt = reinterpret_cast<double*>(hw2 + H.total);
    double* rs = wt + kHistBlock;
    short* bins = reinterpret_cast<short*>(rs + kHistBlock);   // [entry][point]
    const int tid = threadIdx.x;
    for (int b = tid; b < H.total; b += kHistBlock) hw[b] = hw2[b] = DD{0.0, 0.0};
    const MomView v{stage + tid, kHistBlock, kMomSlots};
    for (long long t0 = (long long)blockIdx.x * kHistBlock; t0 < npts; t0 += (long long)gridDim.x * kHistBlock) {
        const int cnt = (int)min((long long)kHistBlock, npts - t0);
        wt[tid] = 0.0;
        if (tid < cnt) {
            EventInfo ev;
            generate_event<N>(seed, (uint64_t)(i0 + t0 + tid), S, ph, v, ev);
            const double y = (S.kind == HEGET_SAMPLER_TOY_PDF && ev.ok) ? 0.5 * log(ev.x1 / ev.x2) : 0.0;
            // the photon observables replace the momenta in the point's column:
            // slot 0 pT, 1 eta (lab), 2 phi
#pragma unroll 1
            for (int i = 0; i < N; ++i) {
                const double px = v(i, 1), py = v(i, 2), pz = v(i, 3);
                const double pt = sqrt(__dadd_rn(__dmul_rn(px, px), __dmul_rn(py, py)));
                v(i, 0) = pt;
                v(i, 1) = asinh(pz / pt) + y;
                v(i, 2) = atan2(py, px);
            }
            wt[tid] = w[t0 + tid];
            rs[tid] = ev.rs;
        }
        for (int s = 0; s < H.nspec; ++s) {
            const HistSpecDev& h = H.spec[s];
            int m = 0;
            if (tid < cnt && wt[tid] != 0.0) {   // a zero weight adds nothing
                switch (h.kind) {
                    case HEGET_OBS_PT_MAX: {
                        double x = v(0, 0);
                        for (int i = 1; i < N; ++i) x = v(i, 0) > x ? v(i, 0) : x;
                        bins[tid] = (short)hist_bin(x, h);
                        m = 1;
                        break;
                    }
                    case HEGET_OBS_PT:
                    case HEGET_OBS_ETA: {
                        const int slot = h.kind == HEGET_OBS_PT ? 0 : 1;
                        for (int i = 0; i < N; ++i) bins[i * kHistBlock + tid] = (short)hist_bin(v(i, slot), h);
                        m = N;
                        break;
                    }
                    case HEGET_OBS_DR:
                    case HEGET_OBS_DR_MIN: {
                        double dmin = 0.0;
                        for (int a = 0; a < N; ++a)
                            for (int b = a + 1; b < N; ++b) {
                                double dphi = fabs(v(a, 2) - v(b, 2));
                                if (dphi > M_PI) dphi = 2.0 * M_PI - dphi;
                                const double deta = v(a, 1) - v(b, 1);
                                const double dr = sqrt(__dadd_rn(__dmul_rn(deta, deta), __dmul_rn(dphi, dphi)));
                                if (h.kind == HEGET_OBS_DR) bins[m * kHistBlock + tid] = (short)hist_bin(dr, h);
                                dmin = (m == 0 || dr < dmin) ? dr : dmin;
                                ++m;
                            }
                        if (h.kind == HEGET_OBS_DR_MIN) {
                            bins[tid] = (short)hist_bin(dmin, h);
                            m = 1;
                        }
                        break;
                    }
                    default:
                        bins[tid] = (short)hist_bin(rs[tid], h);
                        m = 1;
                        break;
                }
            }
            for (int e = m; e < E; ++e) bins[e * kHistBlock + tid] = -1;
            __syncthreads();
            // thread b folds bin b (and b + kHistBlock, ...) of this histogram:
            // the tile's points in order, each point's entries in order, into
            // a plain FP64 tile sum, which joins the block's double-double sum
            // once per tile.  (An FP64 instruction occupies the pipe for a whole
            // warp even when one lane runs it, and a match is one lane's work:
            // two FP64 operations per match instead of a double-double update.)
            const int ne = h.kind == HEGET_OBS_PT || h.kind == HEGET_OBS_ETA ? N : h.kind == HEGET_OBS_DR ? NP : 1;
            for (int b = tid; b < h.nbins + 2; b += kHistBlock) {
                double t1 = 0.0, t2 = 0.0;
                for (int p = 0; p < cnt; ++p) {
                    const double wp = wt[p];
                    if (wp == 0.0) continue;
                    for (int e = 0; e < ne; ++e)
                        if (bins[e * kHistBlock + p] == b) {
                            t1 += wp;
                            t2 = fma(wp, wp, t2);
                        }
                }
                hw[h.off + b] = dd_add_d(hw[h.off + b], t1);
                hw2[h.off + b] = dd_add_d(hw2[h.off + b], t2);
            }
            __syncthreads();
        }
    }
    __syncthreads();
    for (int b = tid; b < H.total; b += kHistBlock) {
        double* o = parts + ((size_t)blockIdx.x * H.total + b) * 4;
        o[0] = hw[b].hi;
        o[1] = hw[b].lo;
        o[2] = hw2[b].hi;
        o[3] = hw2[b].lo;
    }
}

// Block partials combined in block order, in two stages so that many
// threads share the work: stage 1 folds groups of kHistGroup consecutive
// blocks (bin-major threads), stage 2 the groups of each bin in order into
// out[2b], out[2b + 1].
constexpr int kHistGroup = 32;

__global__ void __launch_bounds__(128) hist_group_kernel(const double* __restrict__ parts, int nblocks, int total,
                                                         double* __restrict__ groups) {
    const int ngroups = (nblocks + kHistGroup - 1) / kHistGroup;
    const long long items = (long long)ngroups * total;
    for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < items;
         it += (long long)gridDim.x * blockDim.x) {
        const int g = (int)(it / total), b = (int)(it - (long long)g * total);
        DD a{0.0, 0.0}, a2{0.0, 0.0};
        const int k1 = min(nblocks, (g + 1) * kHistGroup);
        for (int k = g * kHistGroup; k < k1; ++k) {
            const double* o = parts + ((size_t)k * total + b) * 4;
            a = dd_add(a, DD{o[0], o[1]});
            a2 = dd_add(a2, DD{o[2], o[3]});
        }
        double* q = groups + ((size_t)g * total + b) * 4;
        q[0] = a.hi;
        q[1] = a.lo;
        q[2] = a2.hi;
        q[3] = a2.lo;
    }
}

__global__ void __launch_bounds__(128) hist_finalize_kernel(const double* __restrict__ groups, int ngroups,
                                                            int total, double* __restrict__ out) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < total; b += gridDim.x * blockDim.x) {
        DD a{0.0, 0.0}, a2{0.0, 0.0};
        for (int g = 0; g < ngroups; ++g) {
            const double* o = groups + ((size_t)g * total + b) * 4;
            a = dd_add(a, DD{o[0], o[1]});
            a2 = dd_add(a2, DD{o[2], o[3]});
        }
        out[2 * b] = a.hi + a.lo;
        out[2 * b + 1] = a2.hi + a2.lo;
    }
}

template <int N>
int launch_hist_n(uint64_t seed, long long i0, long long npts, const SamplerArgs& S, const Physics& ph,
                  const double* w, const HistArgs& H, double* parts, int grid, cudaStream_t st) {
    auto k = hist_kernel<N>;
    const size_t smem = hist_smem_bytes(N, H.total);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    k<<<grid, kHistBlock, smem, st>>>(seed, i0, npts, S, ph, w, H, parts);
    return (int)cudaGetLastError();
}

template <int N>
int occupancy_hist_n(int total, int* bpsm) {
    auto k = hist_kernel<N>;
    const size_t smem = hist_smem_bytes(N, total);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(bpsm, k, kHistBlock, smem);
}

}  // namespace
}  // namespace heget

using namespace heget;

extern "C" {

int heget_hist(heget_ctx* ctx, int n, uint64_t seed, int64_t i0, int64_t N, const heget_sampler* smp,
               const double* w, const heget_hist_spec* specs, int nspec, double* out, void* stream) {
    int r = check_common(ctx, n, N);
    if (r) return r;
    if ((r = check_sampler(smp))) return r;
    if ((r = check_range(i0, N))) return r;
    if (!specs || nspec < 1 || nspec > HEGET_HIST_MAX_SPECS)
        return fail(HEGET_EINVAL, "need 1 <= nspec <= %d histogram specs", HEGET_HIST_MAX_SPECS);
    HistArgs H{};
    H.nspec = nspec;
    int total = 0;
    for (int s = 0; s < nspec; ++s) {
        const heget_hist_spec& q = specs[s];
        if (q.observable < HEGET_OBS_PT_MAX || q.observable > HEGET_OBS_SQRT_S)
            return fail(HEGET_EINVAL, "spec %d: unknown observable %d", s, q.observable);
        if (q.nbins < 1 || q.nbins > HEGET_HIST_MAX_BINS - 2)
            return fail(HEGET_EINVAL, "spec %d: nbins = %d", s, q.nbins);
        if (!std::isfinite(q.lo) || !std::isfinite(q.hi) || !(q.lo < q.hi) || !std::isfinite(q.hi - q.lo) ||
            !std::isfinite((double)q.nbins / (q.hi - q.lo)))
            return fail(HEGET_EINVAL, "spec %d: need finite lo < hi and a finite bins-per-unit scale", s);
        H.spec[s].kind = q.observable;
        H.spec[s].nbins = q.nbins;
        H.spec[s].off = total;
        H.spec[s].lo = q.lo;
        H.spec[s].scale = (double)q.nbins / (q.hi - q.lo);
        total += q.nbins + 2;
    }
    if (total > HEGET_HIST_MAX_BINS) return fail(HEGET_EINVAL, "%d bins in all; at most %d", total, HEGET_HIST_MAX_BINS);
    H.total = total;
    if (!out) return fail(HEGET_EINVAL, "out must be non-NULL");
    if (N > 0 && !w) return fail(HEGET_EINVAL, "w must be non-NULL");
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (N == 0) {
        const cudaError_t e = cudaMemsetAsync(out, 0, 2 * (size_t)total * sizeof(double), st);
        return e == cudaSuccess ? HEGET_OK : cuda_fail(e, "heget_hist");
    }
    int bpsm = 0;
#define OCC(NN) occupancy_hist_n<NN>(total, &bpsm)
    switch (n) {
        case 2: r = OCC(2); break;
        case 3: r = OCC(3); break;
        case 4: r = OCC(4); break;
        case 5: r = OCC(5); break;
        case 6: r = OCC(6); break;
        case 7: r = OCC(7); break;
        default: r = OCC(8); break;
    }
#undef OCC
    if (r) return cuda_fail((cudaError_t)r, "hist occupancy");
    // one resident wave of at most four blocks per SM (16 warps: enough to
    // keep the FP64 pipe busy) keeps the block partials few
    const long long tiles = (N + kHistBlock - 1) / kHistBlock;
    const long long wave = (long long)ctx->num_sms * std::min(std::max(bpsm, 1), 4);
    const int grid = (int)std::min(tiles, wave);
    const int ngroups = (grid + kHistGroup - 1) / kHistGroup;
    const size_t part_bytes = (size_t)grid * total * 4 * sizeof(double);
    if ((r = grow((void**)&ctx->hist_parts, &ctx->hist_parts_cap,
                  part_bytes + (size_t)ngroups * total * 4 * sizeof(double), false)))
        return r;
    double* groups = ctx->hist_parts + (size_t)grid * total * 4;
    const SamplerArgs S = sampler_args(smp);
    const Physics ph = physics_of(ctx, n);
#define RUN(NN) launch_hist_n<NN>(seed, i0, N, S, ph, w, H, ctx->hist_parts, grid, st)
    switch (n) {
        case 2: r = RUN(2); break;
        case 3: r = RUN(3); break;
        case 4: r = RUN(4); break;
        case 5: r = RUN(5); break;
        case 6: r = RUN(6); break;
        case 7: r = RUN(7); break;
        default: r = RUN(8); break;
    }
#undef RUN
    if (r) return cuda_fail((cudaError_t)r, "hist_kernel");
    const long long items = (long long)ngroups * total;
    hist_group_kernel<<<(int)std::min<long long>((items + 127) / 128, 4096), 128, 0, st>>>(ctx->hist_parts, grid,
                                                                                       total, groups);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "hist_group_kernel");
    hist_finalize_kernel<<<(total + 127) / 128, 128, 0, st>>>(groups, ngroups, total, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "hist_finalize_kernel");
    return HEGET_OK;
}

}  // extern "C"
