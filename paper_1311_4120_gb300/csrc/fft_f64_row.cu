// FFT row-pass kernels for double, every supported length (one translation unit per
// precision and pass mode so that they compile in parallel).
#include "fft_kernels.cuh"

namespace nlint {
template cudaError_t launch_pass_mode_v<double, 1, 0>(const PassDesc &, const void *, void *,
                                                 const void *, cudaStream_t);
}  // namespace nlint
