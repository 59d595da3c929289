// Compile-time FFT passes for lines of length 288, 320, 384 (k_fft.cuh).
#include "k_fft.cuh"

namespace ttm {
template struct FftLen<288>;
template struct FftLen<320>;
template struct FftLen<384>;
}  // namespace ttm
