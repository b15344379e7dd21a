// heget_subset_f64.cu -- subset-recursion kernels of the FP64 spinor chain:
// amp2, fused cross section and occupancy launchers for n = 2..8.
#include "heget_launch.cuh"

namespace heget {
HEGET_INSTANTIATE_ALG(double, kAlgSubset)
}  // namespace heget
