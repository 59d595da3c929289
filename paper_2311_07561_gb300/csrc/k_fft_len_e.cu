// Compile-time FFT passes for lines of length 480, 512, 576 (k_fft.cuh).
#include "k_fft.cuh"

namespace ttm {
template struct FftLen<480>;
template struct FftLen<512>;
template struct FftLen<576>;
}  // namespace ttm
