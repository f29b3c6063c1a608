// FFT passes of line length 256, float (see fft_passes.cuh).
#include "fft_passes.cuh"

namespace ibgb {
template struct FftN<float, 256>;
}  // namespace ibgb
