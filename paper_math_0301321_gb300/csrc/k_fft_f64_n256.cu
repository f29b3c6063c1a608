// FFT passes of line length 256, double (see fft_passes.cuh).
#include "fft_passes.cuh"

namespace ibgb {
template struct FftN<double, 256>;
}  // namespace ibgb
