// FFT row-pass kernels for float whose input is read twice over (fold and multiply inputs),
// every supported length (one translation unit per precision and pass mode).
#include "fft_kernels.cuh"

namespace nlint {
template cudaError_t launch_pass_mode_v<float, 2, 0>(const PassDesc &, const void *, void *,
                                                 const void *, cudaStream_t);
}  // namespace nlint
