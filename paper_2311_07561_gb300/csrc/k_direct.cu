// Direct correlation with the K tensor-template components over the mask
// support (Sec. 2 cross-correlation, Sec. 3.2: C_n(x)_alpha = w(x) <tau_x f, T_alpha>):
//
//   Corr_alpha(x) = sum_u f(x + u - c) T_alpha(u),   u over the mask voxels.
//
// A CTA owns a 64 x 4 tile of voxels in one z-plane and up to kKC components;
// every thread keeps its voxel's kKC accumulators in registers.  For every
// mask plane dz the CTA stages the input rows its windows touch and the
// template values of that plane (tap-major, components contiguous, read as
// shared-memory broadcasts), then walks the plane's x-runs.  FP32 throughout.
#include "ttm_internal.h"

namespace ttm {

namespace {

constexpr int kTX = 64;
constexpr int kTY = 4;
constexpr int kThreads = kTX * kTY;
constexpr int kKC = 36;           // components per pass
constexpr int kTapChunk = 384;    // taps staged at once

struct DirectArgs {
    const float* f;
    float* corr;              // K x nvox
    int X, Y, Z;
    const MaskRun* runs;
    const int* run_tap0;
    const int* dz_run0;
    const float* taps;        // n_taps x K
    int K, a0, na;
    int dz_min, dz_max, dy_min, dy_max, x_min, x_max;
};

__global__ void __launch_bounds__(kThreads) direct_corr_kernel(DirectArgs a) {
    extern __shared__ float smem[];
    const int rows = kTY + (a.dy_max - a.dy_min);
    const int width = kTX + (a.x_max - a.x_min);
    float* F = smem;                                  // rows x width
    float* Tt = smem + ((rows * width + 3) & ~3);     // kTapChunk x kKC

    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY, z = blockIdx.z;
    const int lx = threadIdx.x % kTX, ly = threadIdx.x / kTX;
    float acc[kKC];
#pragma unroll
    for (int k = 0; k < kKC; ++k) acc[k] = 0.f;

    for (int dz = a.dz_min; dz <= a.dz_max; ++dz) {
        const int zz = z + dz;
        const int rb = a.dz_run0[dz - a.dz_min], re = a.dz_run0[dz - a.dz_min + 1];
        if (rb == re) continue;
        __syncthreads();
        for (int e = threadIdx.x; e < rows * width; e += kThreads) {
            const int r = e / width, i = e % width;
            const int yy = y0 + a.dy_min + r, xx = x0 + a.x_min + i;
            float v = 0.f;
            if (zz >= 0 && zz < a.Z && yy >= 0 && yy < a.Y && xx >= 0 && xx < a.X)
                v = __ldg(a.f + ((size_t)zz * a.Y + yy) * a.X + xx);
            F[e] = v;
        }
        // taps of this plane, staged in chunks of whole runs
        int k = rb;
        while (k < re) {
            const int tap0 = a.run_tap0[k];
            int kend = k;
            while (kend < re && a.run_tap0[kend] + (a.runs[kend].x1 - a.runs[kend].x0 + 1) - tap0 <= kTapChunk)
                ++kend;
            if (kend == k) kend = k + 1;   // a single run longer than the chunk cannot occur (s <= 128 < chunk)
            const int ntap = a.run_tap0[kend - 1] + (a.runs[kend - 1].x1 - a.runs[kend - 1].x0 + 1) - tap0;
            __syncthreads();
            for (int e = threadIdx.x; e < ntap * kKC; e += kThreads) {
                const int t = e / kKC, c = e % kKC;
                Tt[e] = c < a.na ? __ldg(a.taps + (size_t)(tap0 + t) * a.K + a.a0 + c) : 0.f;
            }
            __syncthreads();
            for (int kk = k; kk < kend; ++kk) {
                const MaskRun run = a.runs[kk];
                const float* frow = F + (ly + run.dy - a.dy_min) * width + lx - a.x_min;
                const float* trow = Tt + (a.run_tap0[kk] - tap0) * kKC;
                for (int dx = run.x0; dx <= run.x1; ++dx) {
                    const float v = frow[dx];
                    const float4* t4 = reinterpret_cast<const float4*>(trow + (dx - run.x0) * kKC);
#pragma unroll
                    for (int c4 = 0; c4 < kKC / 4; ++c4) {
                        const float4 t = t4[c4];
                        acc[4 * c4 + 0] = fmaf(t.x, v, acc[4 * c4 + 0]);
                        acc[4 * c4 + 1] = fmaf(t.y, v, acc[4 * c4 + 1]);
                        acc[4 * c4 + 2] = fmaf(t.z, v, acc[4 * c4 + 2]);
                        acc[4 * c4 + 3] = fmaf(t.w, v, acc[4 * c4 + 3]);
                    }
                }
            }
            k = kend;
        }
    }
    const int x = x0 + lx, y = y0 + ly;
    if (x >= a.X || y >= a.Y) return;
    const size_t nvox = (size_t)a.X * a.Y * a.Z;
    const size_t v = ((size_t)z * a.Y + y) * a.X + x;
#pragma unroll
    for (int c = 0; c < kKC; ++c)
        if (c < a.na) a.corr[(size_t)(a.a0 + c) * nvox + v] = acc[c];
}

}  // namespace

ttm_status launch_direct_corr(const float* f, int X, int Y, int Z, const TemplateData& T, int K,
                              float* corr, cudaStream_t st, long long* cnt) {
    DirectArgs a;
    a.f = f; a.corr = corr; a.X = X; a.Y = Y; a.Z = Z;
    a.runs = T.d_runs; a.run_tap0 = T.d_run_tap0; a.dz_run0 = T.d_dz_run0; a.taps = T.d_taps;
    a.K = K;
    a.dz_min = T.dz_min; a.dz_max = T.dz_max; a.dy_min = T.dy_min; a.dy_max = T.dy_max;
    a.x_min = T.x_min; a.x_max = T.x_max;
    const int rows = kTY + (T.dy_max - T.dy_min);
    const int width = kTX + (T.x_max - T.x_min);
    const size_t smem = (size_t)(((rows * width + 3) & ~3) + kTapChunk * kKC) * sizeof(float);
    if (smem > 220 * 1024) return TTM_ERR_UNSUPPORTED;
    TTM_CUDA_TRY(cudaFuncSetAttribute(direct_corr_kernel,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((X + kTX - 1) / kTX, (Y + kTY - 1) / kTY, Z);
    for (int a0 = 0; a0 < K; a0 += kKC) {
        a.a0 = a0;
        a.na = K - a0 < kKC ? K - a0 : kKC;
        direct_corr_kernel<<<grid, kThreads, smem, st>>>(a);
        TTM_TRY(after_launch(cnt));
    }
    return TTM_OK;
}

}  // namespace ttm
