// FFT passes of line length 128, float (see fft_passes.cuh).
#include "fft_passes.cuh"

namespace ibgb {
template struct FftN<float, 128>;
}  // namespace ibgb
