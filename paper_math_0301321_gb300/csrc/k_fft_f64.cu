// double instantiation of the FFT fluid solve (see fft_passes.cuh).
#include "fft_passes.cuh"

namespace ibgb {
IB_FFT_EXTERN(double)
template void fluid_impl<double>(ib_ctx *, const void *, const void *, void *, void *, bool, int, cudaStream_t,
                              cudaEvent_t *);
}  // namespace ibgb
