// Local statistics: the NCC denominators (Sec. 2 of the paper,
//   ||P_S tau_x f||_S^2 = <(tau_x f)^2, m> - <tau_x f, m>^2 / <1, m>,
// Algorithm 1, image block), for a binary mask given as x-runs.
//
// A CTA owns a 64 x 8 tile of output voxels in one z-plane.  For every mask
// plane dz it stages the rows the tile's windows touch, subtracts a reference
// value (the input voxel at the tile centre; the variance does not change under
// a constant shift and the shift removes the cancellation of large offsets),
// and builds exclusive prefix sums of (f - mu) and (f - mu)^2 along x in
// shared memory.  Each x-run of the mask then costs two prefix lookups per
// statistic.  The prefix sums and S1, S2 are FP64: a difference of two prefix
// sums cancels whatever the row holds before the run, which in FP32 loses a
// quiet run next to a bright one.  V = S2 - S1^2/m_sum is formed in FP64.
// The degenerate-variance floor is 1e-6 * m_sum * var(f) with var(f) from
// launch_volume_moments.
#include "ttm_internal.h"

namespace ttm {

namespace {

constexpr int kTX = 64;
constexpr int kTY = 8;
constexpr int kStatThreads = 256;   // each thread: x = tid % 64, y = tid / 64 and +4

__global__ void __launch_bounds__(256) moments_kernel(const float* __restrict__ f, size_t n,
                                                      double* acc) {
    __shared__ double r1[8], r2[8];
    // float4 loads with four independent FP32 partial sums each, flushed to
    // FP64 every 16 vectors; the scalar tail (n % 4, or an unaligned f) after
    double d1 = 0.0, d2 = 0.0;
    const size_t tid = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    const size_t nthr = (size_t)gridDim.x * blockDim.x;
    const bool vec = ((uintptr_t)f & 15) == 0;
    const size_t n4 = vec ? n / 4 : 0;
    const float4* f4 = reinterpret_cast<const float4*>(f);
    float4 s1 = make_float4(0.f, 0.f, 0.f, 0.f), s2 = s1;
    int cntr = 0;
    for (size_t i = tid; i < n4; i += nthr) {
        const float4 v = __ldg(f4 + i);
        s1.x += v.x; s1.y += v.y; s1.z += v.z; s1.w += v.w;
        s2.x = fmaf(v.x, v.x, s2.x); s2.y = fmaf(v.y, v.y, s2.y);
        s2.z = fmaf(v.z, v.z, s2.z); s2.w = fmaf(v.w, v.w, s2.w);
        if (++cntr == 16) {
            d1 += (double)s1.x + s1.y + s1.z + s1.w;
            d2 += (double)s2.x + s2.y + s2.z + s2.w;
            s1 = make_float4(0.f, 0.f, 0.f, 0.f); s2 = s1; cntr = 0;
        }
    }
    d1 += (double)s1.x + s1.y + s1.z + s1.w;
    d2 += (double)s2.x + s2.y + s2.z + s2.w;
    for (size_t i = 4 * n4 + tid; i < n; i += nthr) {
        const float v = f[i];
        d1 += v;
        d2 += (double)v * v;
    }
    for (int o = 16; o > 0; o >>= 1) {
        d1 += __shfl_down_sync(0xffffffffu, d1, o);
        d2 += __shfl_down_sync(0xffffffffu, d2, o);
    }
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { r1[wid] = d1; r2[wid] = d2; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { a += r1[k]; b += r2[k]; }
        atomicAdd(acc, a);
        atomicAdd(acc + 1, b);
    }
}

struct StatsArgs {
    const float* f;
    float* w;
    int X, Y, Z, s;
    const MaskRun* runs;
    const int* dz_run0;      // runs of plane dz start at dz_run0[dz - dz_min]
    int dz_min, dz_max, dy_min, dy_max, x_min, x_max;
    double mask_sum;
    const double* moments;   // sum f, sum f^2 over the volume
};

__global__ void __launch_bounds__(kStatThreads) local_stats_kernel(StatsArgs a) {
    extern __shared__ double smem[];
    const int rows = kTY + (a.dy_max - a.dy_min);
    const int width = kTX + (a.x_max - a.x_min);     // staged values per row
    const int pitch = width + 1;                     // exclusive prefix length
    double* P1 = smem;
    double* P2 = smem + rows * pitch;

    const int x0 = blockIdx.x * kTX;
    const int y0 = blockIdx.y * kTY;
    const int z = blockIdx.z;
    const int lx = threadIdx.x % kTX;
    const int ly = threadIdx.x / kTX;                // 0..3, second voxel at ly + 4

    // reference value: the input voxel nearest the tile centre (clamped)
    const int cx = min(x0 + kTX / 2, a.X - 1), cy = min(y0 + kTY / 2, a.Y - 1);
    const double mu = __ldg(a.f + ((size_t)z * a.Y + cy) * a.X + cx);

    double s1[2] = {0.0, 0.0}, s2[2] = {0.0, 0.0};
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = kStatThreads / 32;

    for (int dz = a.dz_min; dz <= a.dz_max; ++dz) {
        const int zz = z + dz;
        __syncthreads();
        // stage rows and build exclusive prefix sums, one warp per row
        for (int r = warp; r < rows; r += nwarps) {
            const int yy = y0 + a.dy_min + r;
            const bool row_ok = zz >= 0 && zz < a.Z && yy >= 0 && yy < a.Y;
            const float* src = a.f + ((size_t)(row_ok ? zz : 0) * a.Y + (row_ok ? yy : 0)) * a.X;
            double run1 = 0.0, run2 = 0.0;
            for (int base = 0; base < width; base += 32) {
                const int i = base + lane;
                const int xx = x0 + a.x_min + i;
                double v = 0.0;
                if (i < width && row_ok && xx >= 0 && xx < a.X) v = (double)__ldg(src + xx) - mu;
                double v2 = v * v;
                // inclusive warp scan
                double c1 = v, c2 = v2;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    double t1 = __shfl_up_sync(0xffffffffu, c1, o);
                    double t2 = __shfl_up_sync(0xffffffffu, c2, o);
                    if (lane >= o) { c1 += t1; c2 += t2; }
                }
                if (i < width) {
                    P1[r * pitch + i + 1] = run1 + c1;
                    P2[r * pitch + i + 1] = run2 + c2;
                }
                run1 += __shfl_sync(0xffffffffu, c1, 31);
                run2 += __shfl_sync(0xffffffffu, c2, 31);
            }
            if (lane == 0) {
                P1[r * pitch] = 0.0;
                P2[r * pitch] = 0.0;
            }
        }
        __syncthreads();
        const int rb = a.dz_run0[dz - a.dz_min], re = a.dz_run0[dz - a.dz_min + 1];
        for (int k = rb; k < re; ++k) {
            const MaskRun run = a.runs[k];
            const int i0 = lx + run.x0 - a.x_min;        // first staged index
            const int i1 = lx + run.x1 - a.x_min + 1;    // one past the last
#pragma unroll
            for (int v = 0; v < 2; ++v) {
                const int r = ly + 4 * v + run.dy - a.dy_min;
                s1[v] += P1[r * pitch + i1] - P1[r * pitch + i0];
                s2[v] += P2[r * pitch + i1] - P2[r * pitch + i0];
            }
        }
    }

    // volume statistics and the variance floor once per CTA (FP64 divisions are slow here)
    __shared__ double sh[2];
    if (threadIdx.x == 0) {
        const double nvox = (double)a.X * a.Y * a.Z;
        const double mean = a.moments[0] / nvox;
        const double var_f = fmax(a.moments[1] / nvox - mean * mean, 0.0);
        sh[0] = 1.0 / a.mask_sum;
        sh[1] = 1e-6 * a.mask_sum * var_f;
    }
    __syncthreads();
    const double inv_msum = sh[0];
    const double floor_v = sh[1];
    const int x = x0 + lx;
    if (x >= a.X) return;
#pragma unroll
    for (int v = 0; v < 2; ++v) {
        const int y = y0 + ly + 4 * v;
        if (y >= a.Y) continue;
        float wv = 0.f;
        if (interior(x, a.X, a.s) && interior(y, a.Y, a.s) && interior(z, a.Z, a.s)) {
            const double S1 = s1[v], S2 = s2[v];
            const double V = S2 - S1 * S1 * inv_msum;
            if (V > floor_v) wv = rsqrtf((float)V);
        }
        a.w[((size_t)z * a.Y + y) * a.X + x] = wv;
    }
}

// Exact local statistics at the voxels flagged by the FFT window sums (w = -1
// there; flagged voxels are interior).  One warp per flagged voxel: the lanes
// split the s^3 mask box and accumulate m (f - f(x)) and m (f - f(x))^2 in
// FP64 (a shift by the voxel's own value; the variance does not change under
// it), then V = S2 - S1^2 / m_sum and w as in every other path.  Warps scan
// the w map 32 voxels at a time; with no flagged voxel the kernel returns at
// once.
__global__ void __launch_bounds__(256) exact_stats_kernel(
    const float* __restrict__ f, float* __restrict__ w, int X, int Y, int Z, int s,
    const float* __restrict__ mask, double mask_sum, const double* __restrict__ moments,
    const unsigned int* __restrict__ flagged) {
    if (*flagged == 0u) return;
    const double nvox = (double)X * Y * Z;
    const double mean = moments[0] / nvox;
    const double floor_v = 1e-6 * mask_sum * fmax(moments[1] / nvox - mean * mean, 0.0);
    const int lane = threadIdx.x & 31;
    const size_t n = (size_t)X * Y * Z;
    const size_t warp0 = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const size_t nwarps = ((size_t)gridDim.x * blockDim.x) >> 5;
    const int c = s / 2, s3 = s * s * s;
    for (size_t base = warp0 * 32; base < n; base += nwarps * 32) {
        const size_t v = base + lane;
        uint32_t bits = __ballot_sync(0xffffffffu, v < n && w[v] < 0.f);
        while (bits) {
            const int src = __ffs(bits) - 1;
            bits &= bits - 1;
            const size_t vv = base + src;
            const int x = (int)(vv % (size_t)X);
            const int y = (int)((vv / (size_t)X) % (size_t)Y);
            const int z = (int)(vv / ((size_t)X * Y));
            const double ref = f[vv];
            double a1 = 0.0, a2 = 0.0;
            for (int u = lane; u < s3; u += 32) {
                const float mu = __ldg(mask + u);
                if (mu == 0.f) continue;
                const int ux = u % s, uy = (u / s) % s, uz = u / (s * s);
                const double d = (double)__ldg(f + ((size_t)(z + uz - c) * Y + (y + uy - c)) * X +
                                               (x + ux - c)) - ref;
                a1 = fma((double)mu, d, a1);
                a2 = fma((double)mu * d, d, a2);
            }
            for (int o = 16; o > 0; o >>= 1) {
                a1 += __shfl_down_sync(0xffffffffu, a1, o);
                a2 += __shfl_down_sync(0xffffffffu, a2, o);
            }
            if (lane == 0) {
                const double V = a2 - a1 * a1 / mask_sum;
                w[vv] = V > floor_v ? (float)(1.0 / sqrt(V)) : 0.f;
            }
        }
    }
}

// integer hash of (index, seed) -> uniform float in [-1, 1)
__global__ void fill_random_kernel(float* __restrict__ f, size_t n, uint32_t seed) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        uint32_t h = (uint32_t)i * 0x9E3779B1u ^ (uint32_t)(i >> 32) ^ seed;
        h ^= h >> 16; h *= 0x7FEB352Du; h ^= h >> 15; h *= 0x846CA68Bu; h ^= h >> 16;
        f[i] = (float)(h >> 8) * (2.0f / 16777216.0f) - 1.0f;
    }
}

}  // namespace

ttm_status launch_fill_random(float* f, size_t n, uint32_t seed, cudaStream_t st, long long* cnt) {
    fill_random_kernel<<<152 * 8, 256, 0, st>>>(f, n, seed);
    return after_launch(cnt);
}

ttm_status launch_volume_moments(const float* f, size_t n, double* d_acc, cudaStream_t st,
                                 long long* cnt) {
    int blocks = (int)((n + 255) / 256);
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (blocks < 1) blocks = 1;
    moments_kernel<<<blocks, 256, 0, st>>>(f, n, d_acc);
    return after_launch(cnt);
}

ttm_status launch_exact_stats(const float* f, float* w, int X, int Y, int Z,
                              const TemplateData& T, const double* moments,
                              const unsigned int* flagged, cudaStream_t st, long long* cnt) {
    exact_stats_kernel<<<152 * 8, 256, 0, st>>>(f, w, X, Y, Z, T.desc.s, T.d_mask,
                                                T.desc.mask_sum, moments, flagged);
    return after_launch(cnt);
}

ttm_status launch_local_stats(const float* f, int X, int Y, int Z, const TemplateData& T,
                              const double* d_moments, float* w, cudaStream_t st,
                              long long* cnt) {
    StatsArgs a;
    a.f = f; a.w = w; a.X = X; a.Y = Y; a.Z = Z; a.s = T.desc.s;
    a.runs = T.d_runs; a.dz_run0 = T.d_dz_run0;
    a.dz_min = T.dz_min; a.dz_max = T.dz_max; a.dy_min = T.dy_min; a.dy_max = T.dy_max;
    a.x_min = T.x_min; a.x_max = T.x_max;
    a.mask_sum = T.desc.mask_sum;
    a.moments = d_moments;
    const int rows = kTY + (T.dy_max - T.dy_min);
    const int pitch = kTX + (T.x_max - T.x_min) + 1;
    const size_t smem = (size_t)2 * rows * pitch * sizeof(double);
    if (smem > 200 * 1024) return TTM_ERR_UNSUPPORTED;
    TTM_CUDA_TRY(cudaFuncSetAttribute(local_stats_kernel,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((X + kTX - 1) / kTX, (Y + kTY - 1) / kTY, Z);
    local_stats_kernel<<<grid, kStatThreads, smem, st>>>(a);
    return after_launch(cnt);
}

}  // namespace ttm
