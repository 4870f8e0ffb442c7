// Interpolation / spreading kernels for float, 2D, bin shape 1 (one translation unit per
// precision, dimension and bin shape so that the width-specialised kernels compile in parallel).
#include "node_kernels.cuh"

namespace nlint {
NLINT_NODE_KERNELS_INSTANTIATE(float, 2, 1)
NLINT_CROWD_MERGE_INSTANTIATE(float, 2)
}  // namespace nlint
