// float instantiation of the FFT fluid solve (see fft_passes.cuh).
#include "fft_passes.cuh"

namespace ibgb {
IB_FFT_EXTERN(float)
template void fluid_impl<float>(ib_ctx *, const void *, const void *, void *, void *, bool, int, cudaStream_t,
                              cudaEvent_t *);
}  // namespace ibgb
