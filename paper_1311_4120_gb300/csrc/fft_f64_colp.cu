// FFT column-pass kernels for double that carry two real data lines per complex FFT line
// (real input to Hermitian half, and back), every supported length.
#include "fft_kernels.cuh"

namespace nlint {
template cudaError_t launch_pass_mode_v<double, 3, 0>(const PassDesc &, const void *, void *,
                                                 const void *, cudaStream_t);
template cudaError_t launch_pass_mode_v<double, 4, 0>(const PassDesc &, const void *, void *,
                                                 const void *, cudaStream_t);
}  // namespace nlint
