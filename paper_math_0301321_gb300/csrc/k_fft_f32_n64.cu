// FFT passes of line length 64, float (see fft_passes.cuh).
#include "fft_passes.cuh"

namespace ibgb {
template struct FftN<float, 64>;
}  // namespace ibgb
