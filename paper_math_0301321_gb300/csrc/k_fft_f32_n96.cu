// FFT passes of line length 96, float (see fft_passes.cuh).
#include "fft_passes.cuh"

namespace ibgb {
template struct FftN<float, 96>;
}  // namespace ibgb
