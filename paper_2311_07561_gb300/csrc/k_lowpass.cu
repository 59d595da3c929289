// Optional isotropic low-pass prefilter h (Sec. 2 of the paper: the method
// may work on t' = h * t and f' = h * f for an isotropic h with h * 1 = 1):
// a sampled Gaussian of unit sum, radius int(4 sigma + 0.5), applied along x,
// y and z in turn as a linear convolution with zero outside the volume.
// One thread per output voxel and pass; block (x segment, y, z).
#include <cmath>

#include "ttm_internal.h"

namespace ttm {

namespace {

constexpr int kMaxRadius = 32;

struct LowpassArgs {
    const float* in;
    float* out;
    int X, Y, Z;
    int axis;                     // 0 x, 1 y, 2 z
    int r;                        // kernel radius
    float w[2 * kMaxRadius + 1];  // w[j] for offset j - r
};

__global__ void __launch_bounds__(128) lowpass_axis_kernel(LowpassArgs a) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= a.X) return;
    const size_t v = ((size_t)z * a.Y + y) * a.X + x;
    const int pos = a.axis == 0 ? x : (a.axis == 1 ? y : z);
    const int n = a.axis == 0 ? a.X : (a.axis == 1 ? a.Y : a.Z);
    const long long stride = a.axis == 0 ? 1 : (a.axis == 1 ? (long long)a.X : (long long)a.X * a.Y);
    float acc = 0.f;
    for (int j = 0; j <= 2 * a.r; ++j) {
        const int p = pos + j - a.r;
        if (p >= 0 && p < n) acc = fmaf(a.w[j], __ldg(a.in + (long long)v + (long long)(j - a.r) * stride), acc);
    }
    a.out[v] = acc;
}

}  // namespace

bool lowpass_sigma_ok(float sigma) {
    return std::isfinite(sigma) && sigma > 0.f && (int)(4.0 * sigma + 0.5) <= kMaxRadius;
}

ttm_status launch_lowpass(const float* in, int X, int Y, int Z, float sigma, float* tmp,
                          float* out, cudaStream_t st, long long* cnt) {
    if (!lowpass_sigma_ok(sigma)) return TTM_ERR_INVALID_ARG;
    if (Y > 65535 || Z > 65535) return TTM_ERR_UNSUPPORTED;
    LowpassArgs a;
    a.X = X; a.Y = Y; a.Z = Z;
    a.r = (int)(4.0 * sigma + 0.5);
    double sum = 0.0;
    double wd[2 * kMaxRadius + 1];
    for (int j = 0; j <= 2 * a.r; ++j) {
        const double d = (double)(j - a.r) / sigma;
        wd[j] = std::exp(-0.5 * d * d);
        sum += wd[j];
    }
    for (int j = 0; j <= 2 * a.r; ++j) a.w[j] = (float)(wd[j] / sum);
    dim3 grid((unsigned)((X + 127) / 128), (unsigned)Y, (unsigned)Z);
    const float* src[3] = {in, out, tmp};
    float* dst[3] = {out, tmp, out};
    for (int axis = 0; axis < 3; ++axis) {
        a.axis = axis;
        a.in = src[axis];
        a.out = dst[axis];
        lowpass_axis_kernel<<<grid, 128, 0, st>>>(a);
        TTM_TRY(after_launch(cnt));
    }
    return TTM_OK;
}

}  // namespace ttm
