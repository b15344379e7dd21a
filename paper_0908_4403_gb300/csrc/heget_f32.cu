// heget_f32.cu -- FP32 spinor-chain kernels that serve either ordering-sum
// algorithm (the mixed-n batch, which reads it from each request) and the
// gauge check (prefix tree).
#include "heget_launch.cuh"

namespace heget {

int launch_ward_f32(int n, const double* mom, long long npts, int ward, double* out, const Physics& ph,
                    int* flag, const AmpLaunch& L, cudaStream_t st) {
#define CALL(N) launch_ward_n<float, N>(mom, npts, ward, out, ph, flag, L, st)
    HEGET_DISPATCH_N(n, CALL)
#undef CALL
}

int launch_batch_f32(const WorkItem* items, int nitems, const BatchReq* reqs, size_t smem, int grid, int alg,
                     cudaStream_t st, bool set_attr) {
    return launch_batch_t<float>(items, nitems, reqs, smem, grid, alg, st, set_attr);
}

int prepare_batch_f32(size_t smem, int alg) { return prepare_batch_t<float>(smem, alg); }

}  // namespace heget
