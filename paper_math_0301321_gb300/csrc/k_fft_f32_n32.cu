// FFT passes of line length 32, float (see fft_passes.cuh).
#include "fft_passes.cuh"

namespace ibgb {
template struct FftN<float, 32>;
}  // namespace ibgb
