// FFT passes of line length 96, double (see fft_passes.cuh).
#include "fft_passes.cuh"

namespace ibgb {
template struct FftN<double, 96>;
}  // namespace ibgb
