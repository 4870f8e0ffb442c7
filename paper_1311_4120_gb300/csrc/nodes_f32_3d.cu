// Interpolation / spreading kernels for float, 3D (one translation unit per precision and
// dimension so that the width-specialised kernels compile in parallel).
#include "node_kernels.cuh"

namespace nlint {
NLINT_NODE_KERNELS_INSTANTIATE(float, 3)
}  // namespace nlint
