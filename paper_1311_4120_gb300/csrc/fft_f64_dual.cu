// FFT column-pass kernels for double that run Algorithm 2's two transforms of one real line
// together (I_1 and I_2 share the density and u), every supported length.
#include "fft_kernels.cuh"

namespace nlint {
template cudaError_t launch_pass_mode_v<double, 6, 0>(const PassDesc &, const void *, void *,
                                                 const void *, cudaStream_t);
template cudaError_t launch_pass_mode_v<double, 7, 0>(const PassDesc &, const void *, void *,
                                                 const void *, cudaStream_t);
}  // namespace nlint
