// FFT passes of line length 64, double (see fft_passes.cuh).
#include "fft_passes.cuh"

namespace ibgb {
template struct FftN<double, 64>;
}  // namespace ibgb
