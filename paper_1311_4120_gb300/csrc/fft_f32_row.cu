// FFT pass kernels for float, row passes, every supported length (one
// translation unit per precision and direction so that they compile in parallel).
#include "fft_kernels.cuh"

namespace nlint {
template cudaError_t launch_pass_impl<float, true>(const PassDesc &, const void *, void *,
                                                   const void *, cudaStream_t);
}  // namespace nlint
