// FFT row-pass kernels for float that convolve each line (forward FFT, multiply, inverse FFT),
// every supported length.
#include "fft_kernels.cuh"

namespace nlint {
template cudaError_t launch_pass_mode_v<float, 5, 0>(const PassDesc &, const void *, void *,
                                                 const void *, cudaStream_t);
}  // namespace nlint
