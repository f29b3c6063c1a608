// FFT passes of line length 32, double (see fft_passes.cuh).
#include "fft_passes.cuh"

namespace ibgb {
template struct FftN<double, 32>;
}  // namespace ibgb
