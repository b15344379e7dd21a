// heget_f32.cu -- FP32 spinor-chain instantiations (FP64 phase space,
// propagator denominators and accumulation).
#include "heget_launch.cuh"

namespace heget {

int launch_amp2_f32(int n, const double* mom, long long npts, const uint32_t* mask, double* out,
                    const Physics& ph, int* flag, int* esc_list, int* esc_count, const AmpLaunch& L, cudaStream_t st) {
#define CALL(N) launch_amp2_n<float, N>(mom, npts, mask, out, ph, flag, esc_list, esc_count, L, st)
    HEGET_DISPATCH_N(n, CALL)
#undef CALL
}

int launch_ward_f32(int n, const double* mom, long long npts, int ward, double* out, const Physics& ph,
                    int* flag, const AmpLaunch& L, cudaStream_t st) {
#define CALL(N) launch_ward_n<float, N>(mom, npts, ward, out, ph, flag, L, st)
    HEGET_DISPATCH_N(n, CALL)
#undef CALL
}

int launch_xsec_f32(int n, uint64_t seed, long long i0, long long npts, const SamplerArgs& S,
                    const Physics& ph, Partial* partials, double* w_out, const EscArgs& esc, const AmpLaunch& L,
                    cudaStream_t st) {
#define CALL(N) launch_xsec_n<float, N>(seed, i0, npts, S, ph, partials, w_out, esc, L, st)
    HEGET_DISPATCH_N(n, CALL)
#undef CALL
}

int occupancy_f32(int n, int tile, int* bpsm, size_t* smem) {
#define CALL(N) occupancy_n<float, N>(tile, bpsm, smem)
    HEGET_DISPATCH_N(n, CALL)
#undef CALL
}

int occupancy_ws_f32(int n, int* bpsm, size_t* smem) {
#define CALL(N) occupancy_ws_n<N>(bpsm, smem)
    HEGET_DISPATCH_N(n, CALL)
#undef CALL
}

int launch_batch_f32(const WorkItem* items, int nitems, const BatchReq* reqs, size_t smem, int grid,
                     cudaStream_t st) {
    return launch_batch_t<float>(items, nitems, reqs, smem, grid, st);
}

}  // namespace heget
