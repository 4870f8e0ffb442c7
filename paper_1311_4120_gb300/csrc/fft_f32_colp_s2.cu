// FFT packed real-data column-pass kernels for float whose input is staged in shared memory by
// asynchronous copies (kernel variant 2), every supported length.
#include "fft_kernels.cuh"

namespace nlint {
template cudaError_t launch_pass_mode_v<float, 3, 2>(const PassDesc &, const void *, void *,
                                                 const void *, cudaStream_t);
template cudaError_t launch_pass_mode_v<float, 4, 2>(const PassDesc &, const void *, void *,
                                                 const void *, cudaStream_t);
}  // namespace nlint
