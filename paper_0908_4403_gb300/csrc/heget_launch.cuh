// heget_launch.cuh -- launch wrappers of the amplitude kernels.  Included by
// the kernel translation units only: each instantiates the per-algorithm
// launchers of one precision and one ordering-sum algorithm
// (HEGET_INSTANTIATE_ALG), or defines the launchers that serve any algorithm
// (mixed-n batch, gauge check, FP64 recomputation of escalated points).
#pragma once

#include "heget_kernels.cuh"

namespace heget {

constexpr int kBlock = 256;

template <class R, int N, int ALG>
static int launch_amp2_n(const double* mom, long long npts, const uint32_t* mask, double* out, const Physics& ph,
                         int* flag, int* esc_list, int* esc_count, const AmpLaunch& L, cudaStream_t st) {
    auto k = amp2_kernel<R, N, kBlock, false, ALG>;
    size_t smem = amp2_smem_bytes<R, N, kBlock, ALG>(L.tile);
    if constexpr (sizeof(R) == sizeof(float))
        if (esc_list) {
            k = amp2_kernel<R, N, kBlock, true, ALG>;
            smem = amp2_smem_bytes<R, N, kBlock, table_alg<ALG, true>()>(L.tile);
        }
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    k<<<L.grid, kBlock, smem, st>>>(mom, npts, mask, out, L.tile, ph, flag, esc_list, esc_count);
    return (int)cudaGetLastError();
}

// The warp-specialised kernel exists where use_ws() can select it: FP32,
// n <= 5 with the tree, every n with the subset recursion.
template <class R, int N, int ALG>
constexpr bool has_ws() {
    return sizeof(R) == sizeof(float) && (N <= 5 || ALG == kAlgSubset);
}

// The fused tile kernel of shape K (tile_shape; K = 0 the default) and its
// dynamic shared memory for `tile` points.
template <class R, int N, int ALG, int K>
struct TileKernel {
    static constexpr TileShape TS = K == 0 ? TileShape{xsec_block<R, N, ALG>(), -1, -1} : tile_shape<R, N, ALG>(K);
    static constexpr auto kernel() { return xsec_kernel<R, N, TS.block, false, ALG, TS.hb, TS.g>; }
    static size_t smem(int tile) { return xsec_smem_bytes<R, N, TS.block, ALG, TS.hb, TS.g>(tile); }
};

template <class R, int N, int ALG, int K>
static int launch_tile_shape(uint64_t seed, long long i0, long long npts, const SamplerArgs& S, const Physics& ph,
                             Partial* partials, double* w_out, const EscArgs& esc, const AmpLaunch& L,
                             cudaStream_t st) {
    using TK = TileKernel<R, N, ALG, K>;
    auto k = TK::kernel();
    const size_t smem = TK::smem(L.tile);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    k<<<L.grid, TK::TS.block, smem, st>>>(seed, i0, npts, S, ph, L.tile, partials, w_out, esc);
    return (int)cudaGetLastError();
}

template <class R, int N, int ALG, int K>
static int occupancy_tile_shape(int tile, int* blocks_per_sm, size_t* smem_out) {
    using TK = TileKernel<R, N, ALG, K>;
    const size_t smem = TK::smem(tile);
    *smem_out = smem;
    auto k = TK::kernel();
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, TK::TS.block, smem);
}

// Dispatch on a run-time shape index to FN<R, N, ALG, K> (the shapes that
// exist for this R, N, ALG; cudaErrorInvalidValue for others).
#define HEGET_DISPATCH_SHAPE(R, N, ALG, shape, FN, ...)                                   \
    switch (shape) {                                                                     \
        case 0: return FN<R, N, ALG, 0>(__VA_ARGS__);                                    \
        case 1:                                                                          \
            if constexpr (num_tile_shapes<R, N, ALG>() > 1) return FN<R, N, ALG, 1>(__VA_ARGS__); \
            break;                                                                       \
        case 2:                                                                          \
            if constexpr (num_tile_shapes<R, N, ALG>() > 2) return FN<R, N, ALG, 2>(__VA_ARGS__); \
            break;                                                                       \
        case 3:                                                                          \
            if constexpr (num_tile_shapes<R, N, ALG>() > 3) return FN<R, N, ALG, 3>(__VA_ARGS__); \
            break;                                                                       \
        default:                                                                         \
            break;                                                                       \
    }                                                                                    \
    return (int)cudaErrorInvalidValue;

template <class R, int N, int ALG>
static int launch_tile(uint64_t seed, long long i0, long long npts, const SamplerArgs& S, const Physics& ph,
                       Partial* partials, double* w_out, const EscArgs& esc, const AmpLaunch& L, cudaStream_t st) {
    HEGET_DISPATCH_SHAPE(R, N, ALG, L.shape, launch_tile_shape, seed, i0, npts, S, ph, partials, w_out, esc, L, st)
}

// The FP32 escalation variant exists for the default shape only: a launch
// with escalation runs shape 0.
template <class R, int N, int ALG>
static int launch_tile_esc(uint64_t seed, long long i0, long long npts, const SamplerArgs& S, const Physics& ph,
                           Partial* partials, double* w_out, const EscArgs& esc, const AmpLaunch& L, cudaStream_t st) {
    constexpr int XB = xsec_block<R, N, ALG>();
    auto k = xsec_kernel<R, N, XB, true, ALG>;
    const size_t smem = xsec_smem_bytes<R, N, XB, table_alg<ALG, true>()>(L.tile);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    k<<<L.grid, XB, smem, st>>>(seed, i0, npts, S, ph, L.tile, partials, w_out, esc);
    return (int)cudaGetLastError();
}

template <class R, int N, int ALG>
static int launch_xsec_n(uint64_t seed, long long i0, long long npts, const SamplerArgs& S, const Physics& ph,
                         Partial* partials, double* w_out, const EscArgs& esc, const AmpLaunch& L, cudaStream_t st) {
    if constexpr (has_ws<R, N, ALG>()) {
        if (L.ws) {
            // the block shape of the instantiation that runs (the escalating
            // kernel keeps more consumers)
            auto k = esc.idx ? xsec_ws_kernel<R, N, true, ALG> : xsec_ws_kernel<R, N, false, ALG>;
            const int threads = esc.idx ? ws_threads<N, ALG, true>() : ws_threads<N, ALG, false>();
            const size_t smem = esc.idx ? ws_smem_bytes<R, N, ALG, table_alg<ALG, true>()>() : ws_smem_bytes<R, N, ALG>();
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return (int)e;
            k<<<L.grid, threads, smem, st>>>(seed, i0, npts, S, ph, partials, w_out, esc);
            return (int)cudaGetLastError();
        }
    } else {
        if (L.ws) return (int)cudaErrorInvalidValue;
    }
    if constexpr (sizeof(R) == sizeof(float))
        if (esc.idx) return launch_tile_esc<R, N, ALG>(seed, i0, npts, S, ph, partials, w_out, esc, L, st);
    return launch_tile<R, N, ALG>(seed, i0, npts, S, ph, partials, w_out, esc, L, st);
}

template <class R, int N, int ALG>
static int occupancy_n(int tile, int shape, int* blocks_per_sm, size_t* smem_out) {
    HEGET_DISPATCH_SHAPE(R, N, ALG, shape, occupancy_tile_shape, tile, blocks_per_sm, smem_out)
}

template <int N, int ALG>
static int occupancy_ws_n(int* blocks_per_sm, size_t* smem_out) {
    if constexpr (has_ws<float, N, ALG>()) {
        const size_t smem = ws_smem_bytes<float, N, ALG>();
        *smem_out = smem;
        auto k = xsec_ws_kernel<float, N, false, ALG>;
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return (int)e;
        return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, ws_threads<N, ALG, false>(), smem);
    } else {
        return (int)cudaErrorInvalidValue;
    }
}

template <int N>
static int launch_amp2_list_n(const double* mom, const int* list, const int* count, const uint32_t* mask,
                              double* out, const Physics& ph, int* flag, int tile, int grid, cudaStream_t st) {
    auto k = amp2_list_kernel<N, kBlock>;
    const size_t smem = amp2_smem_bytes<double, N, kBlock, kAlgSubset>(tile);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    k<<<grid, kBlock, smem, st>>>(mom, list, count, mask, out, tile, ph, flag);
    return (int)cudaGetLastError();
}

template <int N>
static int launch_escalate_n(uint64_t seed, long long i0, const SamplerArgs& S, const Physics& ph, int tile,
                             const EscArgs& esc, Partial* out, double* w_out, int grid, cudaStream_t st) {
    auto k = xsec_escalate_kernel<N, kBlock>;
    const size_t smem = xsec_smem_bytes<double, N, kBlock, kAlgSubset>(tile);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    k<<<grid, kBlock, smem, st>>>(seed, i0, S, ph, tile, esc, out, w_out);
    return (int)cudaGetLastError();
}

template <class R, int N>
static int launch_ward_n(const double* mom, long long npts, int ward, double* out, const Physics& ph, int* flag,
                         const AmpLaunch& L, cudaStream_t st) {
    auto k = ward_kernel<R, N, kBlock>;
    const size_t smem = amp2_smem_bytes<R, N, kBlock, kAlgTree>(L.tile);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    k<<<L.grid, kBlock, smem, st>>>(mom, npts, ward, out, L.tile, ph, flag);
    return (int)cudaGetLastError();
}

template <class R>
static int prepare_batch_t(size_t smem, int alg) {
    return (int)cudaFuncSetAttribute(alg == kAlgSubset ? xsec_batch_kernel<R, kAlgSubset> : xsec_batch_kernel<R, kAlgTree>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// set_attr = false: the caller has run prepare_batch_t for this smem (inside
// a stream capture, where only the launch is recorded).
template <class R>
static int launch_batch_t(const WorkItem* items, int nitems, const BatchReq* reqs, size_t smem, int grid, int alg,
                          cudaStream_t st, bool set_attr) {
    auto k = alg == kAlgSubset ? xsec_batch_kernel<R, kAlgSubset> : xsec_batch_kernel<R, kAlgTree>;
    if (set_attr) {
        const int e = prepare_batch_t<R>(smem, alg);
        if (e) return e;
    }
    k<<<grid, kBatchThreads, smem, st>>>(items, nitems, reqs);
    return (int)cudaGetLastError();
}

#define HEGET_DISPATCH_N(n, CALL)       \
    switch (n) {                        \
        case 2: return CALL(2);         \
        case 3: return CALL(3);         \
        case 4: return CALL(4);         \
        case 5: return CALL(5);         \
        case 6: return CALL(6);         \
        case 7: return CALL(7);         \
        case 8: return CALL(8);         \
        default: return (int)cudaErrorInvalidValue; \
    }

template <class R, int ALG>
int launch_amp2_alg(int n, const double* mom, long long npts, const uint32_t* mask, double* out, const Physics& ph,
                    int* flag, int* esc_list, int* esc_count, const AmpLaunch& L, cudaStream_t st) {
#define CALL(N) launch_amp2_n<R, N, ALG>(mom, npts, mask, out, ph, flag, esc_list, esc_count, L, st)
    HEGET_DISPATCH_N(n, CALL)
#undef CALL
}

template <class R, int ALG>
int launch_xsec_alg(int n, uint64_t seed, long long i0, long long npts, const SamplerArgs& S, const Physics& ph,
                    Partial* partials, double* w_out, const EscArgs& esc, const AmpLaunch& L, cudaStream_t st) {
#define CALL(N) launch_xsec_n<R, N, ALG>(seed, i0, npts, S, ph, partials, w_out, esc, L, st)
    HEGET_DISPATCH_N(n, CALL)
#undef CALL
}

template <class R, int ALG>
int occupancy_alg(int n, int tile, int* bpsm, size_t* smem, int shape) {
#define CALL(N) occupancy_n<R, N, ALG>(tile, shape, bpsm, smem)
    HEGET_DISPATCH_N(n, CALL)
#undef CALL
}

template <int ALG>
int occupancy_ws_alg(int n, int* bpsm, size_t* smem) {
#define CALL(N) occupancy_ws_n<N, ALG>(bpsm, smem)
    HEGET_DISPATCH_N(n, CALL)
#undef CALL
}

// Explicit instantiation of one precision's launchers for one algorithm.
#define HEGET_INSTANTIATE_ALG(R, ALG)                                                                               \
    template int launch_amp2_alg<R, ALG>(int, const double*, long long, const uint32_t*, double*, const Physics&, \
                                         int*, int*, int*, const AmpLaunch&, cudaStream_t);                       \
    template int launch_xsec_alg<R, ALG>(int, uint64_t, long long, long long, const SamplerArgs&, const Physics&,  \
                                         Partial*, double*, const EscArgs&, const AmpLaunch&, cudaStream_t);      \
    template int occupancy_alg<R, ALG>(int, int, int*, size_t*, int);

}  // namespace heget
