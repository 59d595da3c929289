// Compile-time FFT passes for lines of length 96, 128, 144, 160 (k_fft.cuh).
#include "k_fft.cuh"

namespace ttm {
template struct FftLen<96>;
template struct FftLen<128>;
template struct FftLen<144>;
template struct FftLen<160>;
}  // namespace ttm
