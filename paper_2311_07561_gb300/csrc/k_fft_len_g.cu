// Compile-time FFT passes for lines of length 960, 1024 (k_fft.cuh).
#include "k_fft.cuh"

namespace ttm {
template struct FftLen<960>;
template struct FftLen<1024>;
}  // namespace ttm
