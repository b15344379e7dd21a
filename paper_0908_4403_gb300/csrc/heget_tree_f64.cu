// heget_tree_f64.cu -- prefix-tree kernels (the paper's ordering sum) of the
// FP64 spinor chain: amp2, fused cross section and occupancy launchers for
// n = 2..8.
#include "heget_launch.cuh"

namespace heget {
HEGET_INSTANTIATE_ALG(double, kAlgTree)
}  // namespace heget
