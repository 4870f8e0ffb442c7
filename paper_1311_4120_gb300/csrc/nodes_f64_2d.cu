// Interpolation / spreading kernels for double, 2D (one translation unit per precision and
// dimension so that the width-specialised kernels compile in parallel).
#include "node_kernels.cuh"

namespace nlint {
NLINT_NODE_KERNELS_INSTANTIATE(double, 2)
}  // namespace nlint
