// Interpolation / spreading kernels for float, 3D, bin shape 3 (one translation unit per
// precision, dimension and bin shape so that the width-specialised kernels compile in parallel).
#include "node_kernels.cuh"

namespace nlint {
NLINT_NODE_KERNELS_INSTANTIATE(float, 3, 3)

}  // namespace nlint
