// Compile-time FFT passes for lines of length 640, 768 (k_fft.cuh).
#include "k_fft.cuh"

namespace ttm {
template struct FftLen<640>;
template struct FftLen<768>;
}  // namespace ttm
