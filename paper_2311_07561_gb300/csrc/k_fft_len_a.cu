// Compile-time FFT passes for lines of length 16, 32, 48, 64, 80 (k_fft.cuh).
#include "k_fft.cuh"

namespace ttm {
template struct FftLen<16>;
template struct FftLen<32>;
template struct FftLen<48>;
template struct FftLen<64>;
template struct FftLen<80>;
}  // namespace ttm
