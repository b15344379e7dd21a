// heget_f64.cu -- FP64 ("plain FP64") spinor-chain kernels that serve either
// ordering-sum algorithm (the mixed-n batch), the gauge check (prefix tree)
// and the FP64 recomputation of escalated FP32 points (subset recursion).
#include "heget_launch.cuh"

namespace heget {

int launch_ward_f64(int n, const double* mom, long long npts, int ward, double* out, const Physics& ph,
                    int* flag, const AmpLaunch& L, cudaStream_t st) {
#define CALL(N) launch_ward_n<double, N>(mom, npts, ward, out, ph, flag, L, st)
    HEGET_DISPATCH_N(n, CALL)
#undef CALL
}

int launch_batch_f64(const WorkItem* items, int nitems, const BatchReq* reqs, size_t smem, int grid, int alg,
                     cudaStream_t st, bool set_attr) {
    return launch_batch_t<double>(items, nitems, reqs, smem, grid, alg, st, set_attr);
}

int prepare_batch_f64(size_t smem, int alg) { return prepare_batch_t<double>(smem, alg); }

int launch_escalate_f64(int n, uint64_t seed, long long i0, const SamplerArgs& S, const Physics& ph, int tile,
                        const EscArgs& esc, Partial* out, double* w_out, int grid, cudaStream_t st) {
#define CALL(N) launch_escalate_n<N>(seed, i0, S, ph, tile, esc, out, w_out, grid, st)
    HEGET_DISPATCH_N(n, CALL)
#undef CALL
}

int launch_amp2_list_f64(int n, const double* mom, const int* list, const int* count, const uint32_t* mask,
                         double* out, const Physics& ph, int* flag, int tile, int grid, cudaStream_t st) {
#define CALL(N) launch_amp2_list_n<N>(mom, list, count, mask, out, ph, flag, tile, grid, st)
    HEGET_DISPATCH_N(n, CALL)
#undef CALL
}

}  // namespace heget
