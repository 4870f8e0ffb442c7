// Interpolation / spreading kernels for double, 3D, bin shape 2 (one translation unit per
// precision, dimension and bin shape so that the width-specialised kernels compile in parallel).
#include "node_kernels.cuh"

namespace nlint {
NLINT_NODE_KERNELS_INSTANTIATE(double, 3, 2)

}  // namespace nlint
