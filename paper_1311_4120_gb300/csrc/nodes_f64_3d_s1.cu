// Interpolation / spreading kernels for double, 3D, bin shape 1 (one translation unit per
// precision, dimension and bin shape so that the width-specialised kernels compile in parallel).
#include "node_kernels.cuh"

namespace nlint {
NLINT_NODE_KERNELS_INSTANTIATE(double, 3, 1)
NLINT_CROWD_MERGE_INSTANTIATE(double, 3)
}  // namespace nlint
