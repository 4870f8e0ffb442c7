// Interpolation / spreading kernels for double, 3D (one translation unit per precision and
// dimension so that the width-specialised kernels compile in parallel).
#include "node_kernels.cuh"

namespace nlint {
NLINT_NODE_KERNELS_INSTANTIATE(double, 3)
}  // namespace nlint
