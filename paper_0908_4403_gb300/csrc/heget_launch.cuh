// heget_launch.cuh -- per-precision launch wrappers of the amplitude kernels.
// Included by exactly one .cu per precision, which defines HEGET_REAL and
// HEGET_SUFFIX before including it.
#pragma once

#include "heget_kernels.cuh"

namespace heget {

constexpr int kBlock = 256;

template <class R, int N>
static int launch_amp2_n(const double* mom, long long npts, const uint32_t* mask, double* out, const Physics& ph,
                         int* flag, int* esc_list, int* esc_count, const AmpLaunch& L, cudaStream_t st) {
    auto k = amp2_kernel<R, N, kBlock, false>;
    if constexpr (sizeof(R) == sizeof(float))
        if (esc_list) k = amp2_kernel<R, N, kBlock, true>;
    const size_t smem = amp2_smem_bytes<R, N, kBlock>(L.tile);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    k<<<L.grid, kBlock, smem, st>>>(mom, npts, mask, out, L.tile, ph, flag, esc_list, esc_count);
    return (int)cudaGetLastError();
}

template <int N>
static int launch_amp2_list_n(const double* mom, const int* list, const int* count, const uint32_t* mask,
                              double* out, const Physics& ph, int* flag, int tile, int grid, cudaStream_t st) {
    auto k = amp2_list_kernel<N, kBlock>;
    const size_t smem = amp2_smem_bytes<double, N, kBlock>(tile);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    k<<<grid, kBlock, smem, st>>>(mom, list, count, mask, out, tile, ph, flag);
    return (int)cudaGetLastError();
}

template <int N>
static int launch_escalate_n(uint64_t seed, long long i0, const SamplerArgs& S, const Physics& ph, int tile,
                             const EscArgs& esc, Partial* out, double* w_out, int grid, cudaStream_t st) {
    auto k = xsec_escalate_kernel<N, kBlock>;
    const size_t smem = xsec_smem_bytes<double, N, kBlock>(tile);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    k<<<grid, kBlock, smem, st>>>(seed, i0, S, ph, tile, esc, out, w_out);
    return (int)cudaGetLastError();
}

template <class R, int N>
static int launch_ward_n(const double* mom, long long npts, int ward, double* out, const Physics& ph, int* flag,
                         const AmpLaunch& L, cudaStream_t st) {
    auto k = ward_kernel<R, N, kBlock>;
    const size_t smem = amp2_smem_bytes<R, N, kBlock>(L.tile);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    k<<<L.grid, kBlock, smem, st>>>(mom, npts, ward, out, L.tile, ph, flag);
    return (int)cudaGetLastError();
}

template <class R, int N>
static int launch_xsec_n(uint64_t seed, long long i0, long long npts, const SamplerArgs& S, const Physics& ph,
                         Partial* partials, double* w_out, const EscArgs& esc, const AmpLaunch& L, cudaStream_t st) {
    if constexpr (sizeof(R) == sizeof(float)) {
        if (L.ws) {
            auto k = esc.idx ? xsec_ws_kernel<R, N, true> : xsec_ws_kernel<R, N, false>;
            const size_t smem = ws_smem_bytes<R, N>();
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return (int)e;
            k<<<L.grid, kWsConsumers + ws_stage(N), smem, st>>>(seed, i0, npts, S, ph, partials, w_out, esc);
            return (int)cudaGetLastError();
        }
    }
    auto k = xsec_kernel<R, N, kBlock, false>;
    if constexpr (sizeof(R) == sizeof(float))
        if (esc.idx) k = xsec_kernel<R, N, kBlock, true>;
    const size_t smem = xsec_smem_bytes<R, N, kBlock>(L.tile);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    k<<<L.grid, kBlock, smem, st>>>(seed, i0, npts, S, ph, L.tile, partials, w_out, esc);
    return (int)cudaGetLastError();
}

template <class R, int N>
static int occupancy_n(int tile, int* blocks_per_sm, size_t* smem_out) {
    const size_t smem = xsec_smem_bytes<R, N, kBlock>(tile);
    *smem_out = smem;
    auto k = xsec_kernel<R, N, kBlock>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, kBlock, smem);
}

template <int N>
static int occupancy_ws_n(int* blocks_per_sm, size_t* smem_out) {
    const size_t smem = ws_smem_bytes<float, N>();
    *smem_out = smem;
    auto k = xsec_ws_kernel<float, N>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, kWsConsumers + ws_stage(N), smem);
}

template <class R>
static int launch_batch_t(const WorkItem* items, int nitems, const BatchReq* reqs, size_t smem, int grid,
                          cudaStream_t st) {
    auto k = xsec_batch_kernel<R>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
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

}  // namespace heget
