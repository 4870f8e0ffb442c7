// FFT column-pass kernels for float with the second schedule (nlint_params.fft_sched), every length that has one;
// the other lengths run schedule 0, instantiated in the schedule-0 translation unit.
#include "fft_kernels.cuh"

namespace nlint {
extern template cudaError_t launch_pass_mode_v<float, 0, 0>(const PassDesc &, const void *, void *,
                                                        const void *, cudaStream_t);
template cudaError_t launch_pass_mode_v<float, 0, 1>(const PassDesc &, const void *, void *,
                                                 const void *, cudaStream_t);
}  // namespace nlint
