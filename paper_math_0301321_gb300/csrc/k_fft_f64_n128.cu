// FFT passes of line length 128, double (see fft_passes.cuh).
#include "fft_passes.cuh"

namespace ibgb {
template struct FftN<double, 128>;
}  // namespace ibgb
