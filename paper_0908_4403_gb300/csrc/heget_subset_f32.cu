// heget_subset_f32.cu -- subset-recursion kernels of the FP32 spinor chain
// (FP64 phase space, denominators and accumulation): amp2, fused cross
// section and occupancy launchers for n = 2..8.
#include "heget_launch.cuh"

namespace heget {
HEGET_INSTANTIATE_ALG(float, kAlgSubset)
template int occupancy_ws_alg<kAlgSubset>(int, int*, size_t*);
}  // namespace heget
