// Compile-time FFT passes for lines of length 192, 240, 256 (k_fft.cuh).
#include "k_fft.cuh"

namespace ttm {
template struct FftLen<192>;
template struct FftLen<240>;
template struct FftLen<256>;
}  // namespace ttm
