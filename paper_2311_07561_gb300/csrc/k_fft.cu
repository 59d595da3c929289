// Batched 3D FFTs for the correlation with the K tensor components (Sec. 2 of
// the paper: <f, g> = F^-1(F f . conj F g)(0); Algorithm 1 uses it for every
// rotation, TTM for every component, Sec. 3.2).
//
// Layouts.  A real volume is [Zp][Yp][Xp] (padded sizes, zero beyond the
// data); its half spectrum is [Zp][Yp][Xh] complex64 with Xh = Xp/2 + 1.
//
// Every pass moves a tile of whole 1D lines into shared memory, transforms
// them there with Stockham autosort stages (radix 4, one radix-2 stage when
// the length needs it; two shared-memory buffers ping-pong between stages),
// and writes the tile back, so each pass reads and writes HBM once:
//   rows_r2c      x lines of the real volume -> half-spectrum rows
//   cols          y or z lines of a half spectrum (strided), in place
//   cols_mul      z lines of the image spectrum times conj(template spectrum)
//                 for all K components: the image tile is read once and kept
//                 in shared memory while the K component tiles stream through
//   rows_c2r      half-spectrum rows -> real x lines (Hermitian extension)
// Twiddles exp(-2 pi i k / L) come from a table computed on the host in FP64.
#include <cuda_bf16.h>

#include <type_traits>

#include "ttm_internal.h"

namespace ttm {

namespace {

constexpr int kFftThreads = 256;
constexpr int kTileElems = 4096;   // complex elements per shared-memory buffer

struct Radices {
    int n;          // number of stages
    int r[16];      // radix of each stage (4 or 2), in order
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {   // a * conj(b)
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }

// Storage types of spectra (float2 or bf16 pairs) and real maps (float or
// bf16); arithmetic is always FP32.
__device__ __forceinline__ float2 ldc(const float2* p) { return *p; }
__device__ __forceinline__ float2 ldc(const __nv_bfloat162* p) { return __bfloat1622float2(*p); }
__device__ __forceinline__ float2 ldgc(const float2* p) { return __ldg(p); }
__device__ __forceinline__ float2 ldgc(const __nv_bfloat162* p) { return __bfloat1622float2(__ldg(p)); }
__device__ __forceinline__ void stc(float2* p, float2 v) { *p = v; }
__device__ __forceinline__ void stc(__nv_bfloat162* p, float2 v) { *p = __float22bfloat162_rn(v); }
__device__ __forceinline__ void str(float* p, float v) { *p = v; }
__device__ __forceinline__ void str(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// NB independent transforms of length L stored as buf[i * pitch + b].  The
// result ends in *out (one of a, b).  sign = -1 forward, +1 inverse.
__device__ void fft_lines(float2* a, float2* b, float2** out, int L, int NB, int pitch,
                          const Radices& rd, const float2* __restrict__ tw, int sign) {
    float2* src = a;
    float2* dst = b;
    int Ns = 1;
    for (int st = 0; st < rd.n; ++st) {
        const int R = rd.r[st];
        const int nbf = L / R;                    // butterflies per line
        const int stride_tw = L / (Ns * R);
        for (int idx = threadIdx.x; idx < nbf * NB; idx += blockDim.x) {
            const int line = idx % NB;
            const int j = idx / NB;
            const int jm = j % Ns;
            const int idxD = (j / Ns) * Ns * R + jm;
            if (R == 4) {
                float2 v[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    float2 x = src[(j + r * nbf) * pitch + line];
                    if (r) {
                        float2 w = __ldg(tw + jm * r * stride_tw);
                        w.y *= (float)(-sign);      // forward: table value, inverse: conjugate
                        x = cmul(x, w);
                    }
                    v[r] = x;
                }
                float2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
                float2 s13 = cadd(v[1], v[3]), d13 = csub(v[1], v[3]);
                // d = -i*d13 (forward) or +i*d13 (inverse)
                float2 d = sign < 0 ? make_float2(d13.y, -d13.x) : make_float2(-d13.y, d13.x);
                dst[(idxD + 0 * Ns) * pitch + line] = cadd(s02, s13);
                dst[(idxD + 1 * Ns) * pitch + line] = cadd(d02, d);
                dst[(idxD + 2 * Ns) * pitch + line] = csub(s02, s13);
                dst[(idxD + 3 * Ns) * pitch + line] = csub(d02, d);
            } else {  // R == 2
                float2 x0 = src[j * pitch + line];
                float2 x1 = src[(j + nbf) * pitch + line];
                float2 w = __ldg(tw + jm * stride_tw);
                w.y *= (float)(-sign);
                x1 = cmul(x1, w);
                dst[(idxD) * pitch + line] = cadd(x0, x1);
                dst[(idxD + Ns) * pitch + line] = csub(x0, x1);
            }
        }
        __syncthreads();
        float2* t = src; src = dst; dst = t;
        Ns *= R;
    }
    *out = src;
}

// ---- compile-time-length Stockham stages with radix up to 16 in registers ----
// Small DFTs (sign -1 forward, +1 inverse).  DFT16 = 4 x 4 with the internal
// twiddles W16^(n2 k1); its outputs come back in transposed order.
constexpr float kC8 = 0.92387953251128674f;   // cos(pi/8)
constexpr float kS8 = 0.38268343236508978f;   // sin(pi/8)
constexpr float kR2 = 0.70710678118654752f;   // sqrt(2)/2

template <int SIGN>
__device__ __forceinline__ float2 mul_mi(float2 a) {   // a * (SIGN * i)
    return SIGN < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

template <int SIGN>
__device__ __forceinline__ void dft4(float2& a, float2& b, float2& c, float2& d) {
    float2 s02 = cadd(a, c), d02 = csub(a, c), s13 = cadd(b, d), d13 = csub(b, d);
    float2 t = mul_mi<SIGN>(d13);
    a = cadd(s02, s13);
    b = cadd(d02, t);
    c = csub(s02, s13);
    d = csub(d02, t);
}

// W16^m for the forward transform (conjugated for the inverse)
template <int SIGN>
__device__ __forceinline__ float2 w16(int m) {
    float c, s;
    switch (m & 15) {
        case 0: c = 1.f; s = 0.f; break;
        case 1: c = kC8; s = kS8; break;
        case 2: c = kR2; s = kR2; break;
        case 3: c = kS8; s = kC8; break;
        case 4: c = 0.f; s = 1.f; break;
        case 5: c = -kS8; s = kC8; break;
        case 6: c = -kR2; s = kR2; break;
        case 7: c = -kC8; s = kS8; break;
        case 8: c = -1.f; s = 0.f; break;
        default: c = -kC8; s = -kS8; break;   // 9
    }
    // forward: exp(-2 pi i m / 16) = c - i s
    return SIGN < 0 ? make_float2(c, -s) : make_float2(c, s);
}

template <int R, int SIGN>
__device__ __forceinline__ void dft_small(float2 (&v)[R]) {
    if constexpr (R == 2) {
        float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if constexpr (R == 4) {
        dft4<SIGN>(v[0], v[1], v[2], v[3]);
    } else if constexpr (R == 8) {
        // n = 2 n1 + n2, k = k1 + 4 k2
        float2 u[8];
#pragma unroll
        for (int n2 = 0; n2 < 2; ++n2) {
            float2 a = v[n2], b = v[n2 + 2], c = v[n2 + 4], d = v[n2 + 6];
            dft4<SIGN>(a, b, c, d);
            u[n2 + 0] = a; u[n2 + 2] = b; u[n2 + 4] = c; u[n2 + 6] = d;   // u[n2 + 2 k1]
        }
        // twiddle W8^(n2 k1) = W16^(2 n2 k1)
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) u[1 + 2 * k1] = cmul(u[1 + 2 * k1], w16<SIGN>(2 * k1));
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            float2 a = u[2 * k1], b = u[2 * k1 + 1];
            v[k1] = cadd(a, b);          // k2 = 0 -> k = k1
            v[k1 + 4] = csub(a, b);      // k2 = 1 -> k = k1 + 4
        }
    } else {  // R == 16: n = 4 n1 + n2, k = k1 + 4 k2
        float2 u[16];
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) {
            float2 a = v[n2], b = v[n2 + 4], c = v[n2 + 8], d = v[n2 + 12];
            dft4<SIGN>(a, b, c, d);
            u[4 * 0 + n2] = a; u[4 * 1 + n2] = b; u[4 * 2 + n2] = c; u[4 * 3 + n2] = d;  // u[4 k1 + n2]
        }
#pragma unroll
        for (int k1 = 1; k1 < 4; ++k1)
#pragma unroll
            for (int n2 = 1; n2 < 4; ++n2) u[4 * k1 + n2] = cmul(u[4 * k1 + n2], w16<SIGN>(n2 * k1));
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            float2 a = u[4 * k1], b = u[4 * k1 + 1], c = u[4 * k1 + 2], d = u[4 * k1 + 3];
            dft4<SIGN>(a, b, c, d);
            v[k1] = a; v[k1 + 4] = b; v[k1 + 8] = c; v[k1 + 12] = d;     // k = k1 + 4 k2
        }
    }
}

// radix of stage st for length L: 16s first, the remaining factor last
__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n >> 1); }
__host__ __device__ constexpr int n_stages(int L) {
    return ilog2c(L) / 4 + ((ilog2c(L) % 4) ? 1 : 0);
}
__host__ __device__ constexpr int stage_radix(int L, int st) {
    return (st < ilog2c(L) / 4) ? 16 : (1 << (ilog2c(L) % 4));
}

// One Stockham stage of radix R on NB lines of length L, buf[i * PITCH + line].
template <int L, int R, int NS, int NB, int PITCH, int SIGN>
__device__ __forceinline__ void stockham_stage(const float2* __restrict__ src, float2* __restrict__ dst,
                                               const float2* __restrict__ tw) {
    constexpr int NBF = L / R;
    constexpr int STRIDE_TW = L / (NS * R);
    for (int idx = threadIdx.x; idx < NBF * NB; idx += blockDim.x) {
        const int line = idx & (NB - 1);
        const int j = idx / NB;                      // NB is a power of two
        const int jm = j & (NS - 1);
        const int idxD = (j - jm) * R + jm;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[(j + r * NBF) * PITCH + line];
        if constexpr (NS > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float2 w = __ldg(tw + jm * r * STRIDE_TW);
                if (SIGN > 0) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        dft_small<R, SIGN>(v);
#pragma unroll
        for (int r = 0; r < R; ++r) dst[(idxD + r * NS) * PITCH + line] = v[r];
    }
}

template <int L, int ST, int NB, int PITCH, int SIGN>
__device__ __forceinline__ float2* stockham_from(float2* a, float2* b, const float2* tw) {
    if constexpr (ST >= n_stages(L)) {
        return a;
    } else {
        constexpr int R = stage_radix(L, ST);
        constexpr int NS = [] { int ns = 1; for (int s = 0; s < ST; ++s) ns *= stage_radix(L, s); return ns; }();
        stockham_stage<L, R, NS, NB, PITCH, SIGN>(a, b, tw);
        __syncthreads();
        return stockham_from<L, ST + 1, NB, PITCH, SIGN>(b, a, tw);
    }
}

template <int L, int NB, int PITCH, int SIGN>
__device__ __forceinline__ float2* fft_lines_t(float2* a, float2* b, const float2* tw) {
    return stockham_from<L, 0, NB, PITCH, SIGN>(a, b, tw);
}

template <int L> constexpr int rows_nb() { return (4096 / L) > 16 ? 16 : (4096 / L < 1 ? 1 : 4096 / L); }
template <int L> constexpr int cols_tb() { return (4096 / L) > 32 ? 32 : (4096 / L < 1 ? 1 : 4096 / L); }

struct FftGeom {
    int Xp, Yp, Zp, Xh;
};

// ---- rows: real x lines -> half-spectrum rows --------------------------
// The source volume has X, Y, Z <= Xp, Yp, Zp; lines and samples beyond the
// data are zero.  Rows are (y, z) pairs of the padded volume.
__global__ void __launch_bounds__(kFftThreads) rows_r2c_kernel(
    const float* __restrict__ f, int X, int Y, int Z, FftGeom g, float2* __restrict__ out,
    Radices rd, const float2* __restrict__ tw, int NB) {
    extern __shared__ float2 sm[];
    const int pitch = NB + 1;
    float2* A = sm;
    float2* B = sm + g.Xp * pitch;
    const int row0 = blockIdx.x * NB;
    const int nrows = g.Yp * g.Zp;
    for (int e = threadIdx.x; e < NB * g.Xp; e += blockDim.x) {
        const int r = e / g.Xp, x = e % g.Xp;
        const int row = row0 + r;
        float v = 0.f;
        if (row < nrows) {
            const int y = row % g.Yp, z = row / g.Yp;
            if (x < X && y < Y && z < Z) v = __ldg(f + ((size_t)z * Y + y) * X + x);
        }
        A[x * pitch + r] = make_float2(v, 0.f);
    }
    __syncthreads();
    float2* res;
    fft_lines(A, B, &res, g.Xp, NB, pitch, rd, tw, -1);
    for (int e = threadIdx.x; e < NB * g.Xh; e += blockDim.x) {
        const int r = e / g.Xh, k = e % g.Xh;
        const int row = row0 + r;
        if (row < nrows) out[(size_t)row * g.Xh + k] = res[k * pitch + r];
    }
}

// ---- columns: lines of length L with element stride B, batch A ----------
// data[(a * L + l) * B + b]; CTA = (b tile of TB, a).
__global__ void __launch_bounds__(kFftThreads) cols_kernel(float2* __restrict__ data, int L,
                                                           int B, Radices rd,
                                                           const float2* __restrict__ tw, int TB,
                                                           int sign) {
    extern __shared__ float2 sm[];
    float2* P = sm;
    float2* Q = sm + L * TB;
    const int b0 = blockIdx.x * TB;
    const size_t base = (size_t)blockIdx.y * L * B;
    const int tb = min(TB, B - b0);
    for (int e = threadIdx.x; e < L * TB; e += blockDim.x) {
        const int l = e / TB, bb = e % TB;
        P[e] = bb < tb ? data[base + (size_t)l * B + b0 + bb] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2* res;
    fft_lines(P, Q, &res, L, TB, TB, rd, tw, sign);
    for (int e = threadIdx.x; e < L * TB; e += blockDim.x) {
        const int l = e / TB, bb = e % TB;
        if (bb < tb) data[base + (size_t)l * B + b0 + bb] = res[e];
    }
}

// ---- z lines of F(f) * conj(T^_k) for every component k, inverse -------
// spec: image spectrum [Zp][Yp*Xh]; tspec: K template spectra (same shape,
// already scaled by 1/N); out: K products after the inverse z transform.
__global__ void __launch_bounds__(kFftThreads) cols_mul_kernel(
    const float2* __restrict__ spec, const float2* __restrict__ tspec, float2* __restrict__ out,
    int L, int B, int K, Radices rd, const float2* __restrict__ tw, int TB) {
    extern __shared__ float2 sm[];
    float2* Fimg = sm;
    float2* P = sm + L * TB;
    float2* Q = sm + 2 * L * TB;
    const int b0 = blockIdx.x * TB;
    const int tb = min(TB, B - b0);
    const size_t plane = (size_t)L * B;
    for (int e = threadIdx.x; e < L * TB; e += blockDim.x) {
        const int l = e / TB, bb = e % TB;
        Fimg[e] = bb < tb ? spec[(size_t)l * B + b0 + bb] : make_float2(0.f, 0.f);
    }
    for (int k = 0; k < K; ++k) {
        __syncthreads();
        const float2* ts = tspec + (size_t)k * plane;
        for (int e = threadIdx.x; e < L * TB; e += blockDim.x) {
            const int l = e / TB, bb = e % TB;
            float2 t = bb < tb ? __ldg(ts + (size_t)l * B + b0 + bb) : make_float2(0.f, 0.f);
            P[e] = cmulc(Fimg[e], t);
        }
        __syncthreads();
        float2* res;
        fft_lines(P, Q, &res, L, TB, TB, rd, tw, +1);
        float2* o = out + (size_t)k * plane;
        for (int e = threadIdx.x; e < L * TB; e += blockDim.x) {
            const int l = e / TB, bb = e % TB;
            if (bb < tb) o[(size_t)l * B + b0 + bb] = res[e];
        }
    }
}

// ---- half-spectrum rows -> real x lines (inverse) ------------------------
// in: batch of nb_planes * Yp rows of Xh complex; writes the X x Y x Z data
// region of every plane into out (batch-major, X*Y*Z floats per batch item).
__global__ void __launch_bounds__(kFftThreads) rows_c2r_kernel(
    const float2* __restrict__ in, int X, int Y, int Z, FftGeom g, float* __restrict__ out,
    int n_batch, Radices rd, const float2* __restrict__ tw, int NB) {
    extern __shared__ float2 sm[];
    const int pitch = NB + 1;
    float2* A = sm;
    float2* Bf = sm + g.Xp * pitch;
    const size_t rows_per_item = (size_t)g.Yp * g.Zp;
    const size_t nrows = rows_per_item * n_batch;
    const size_t row0 = (size_t)blockIdx.x * NB;
    for (int e = threadIdx.x; e < NB * g.Xp; e += blockDim.x) {
        const int r = e / g.Xp, x = e % g.Xp;
        const size_t row = row0 + r;
        float2 v = make_float2(0.f, 0.f);
        if (row < nrows) {
            const float2* src = in + row * g.Xh;
            if (x < g.Xh) v = src[x];
            else { float2 c = src[g.Xp - x]; v = make_float2(c.x, -c.y); }
        }
        A[x * pitch + r] = v;
    }
    __syncthreads();
    float2* res;
    fft_lines(A, Bf, &res, g.Xp, NB, pitch, rd, tw, +1);
    const size_t vox = (size_t)X * Y * Z;
    for (int e = threadIdx.x; e < NB * g.Xp; e += blockDim.x) {
        const int r = e / g.Xp, x = e % g.Xp;
        const size_t row = row0 + r;
        if (row >= nrows || x >= X) continue;
        const size_t item = row / rows_per_item;
        const int rr = (int)(row % rows_per_item);
        const int y = rr % g.Yp, z = rr / g.Yp;
        if (y < Y && z < Z) out[item * vox + ((size_t)z * Y + y) * X + x] = res[x * pitch + r].x;
    }
}

// place a component box into a zeroed padded volume at (u - c) mod N
__global__ void scatter_component_kernel(const float* __restrict__ comp, int s, FftGeom g,
                                         float* __restrict__ pad) {
    const int s3 = s * s * s;
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= s3) return;
    const int c = s / 2;
    const int ux = u % s, uy = (u / s) % s, uz = u / (s * s);
    const int x = ((ux - c) % g.Xp + g.Xp) % g.Xp;
    const int y = ((uy - c) % g.Yp + g.Yp) % g.Yp;
    const int z = ((uz - c) % g.Zp + g.Zp) % g.Zp;
    pad[((size_t)z * g.Yp + y) * g.Xp + x] = comp[u];
}

__global__ void scale_kernel(float2* __restrict__ a, size_t n, float s) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) { a[i].x *= s; a[i].y *= s; }
}

// ---- the four passes with a compile-time line length ---------------------
// mode 0 transforms f, mode 1 (f - mean), mode 2 (f - mean)^2 with mean =
// moments[0] / (X Y Z) (the shift removes the cancellation in the local variance)
template <int L>
__global__ void __launch_bounds__(kFftThreads) rows_r2c_t(const float* __restrict__ f, int X, int Y,
                                                          int Z, FftGeom g, float2* __restrict__ out,
                                                          const float2* __restrict__ tw, int mode,
                                                          const double* __restrict__ moments) {
    constexpr int NB = rows_nb<L>();
    constexpr int PITCH = NB + 1;
    constexpr int XH = L / 2 + 1;
    extern __shared__ float2 sm[];
    float2* A = sm;
    float2* B = sm + L * PITCH;
    const int row0 = blockIdx.x * NB;
    const int nrows = g.Yp * g.Zp;
    const float mean = mode ? (float)(moments[0] / ((double)X * Y * Z)) : 0.f;
    constexpr int PER = (NB * L + kFftThreads - 1) / kFftThreads;
    __shared__ long long row_in[NB];         // input offset of each row, -1 = zero row
    if (threadIdx.x < NB) {
        const int row = row0 + threadIdx.x;
        long long off = -1;
        if (row < nrows) {
            const int y = row % g.Yp, z = row / g.Yp;
            if (y < Y && z < Z) off = (long long)(((size_t)z * Y + y) * X);
        }
        row_in[threadIdx.x] = off;
    }
    __syncthreads();
    float vv[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int e = threadIdx.x + i * kFftThreads;
        const int r = e / L, x = e & (L - 1);
        float v = 0.f;
        if (e < NB * L && x < X) {
            const long long off = row_in[r];
            if (off >= 0) {
                v = __ldg(f + off + x) - mean;
                if (mode == 2) v = v * v;
            }
        }
        vv[i] = v;
    }
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int e = threadIdx.x + i * kFftThreads;
        const int r = e / L, x = e & (L - 1);
        if (e < NB * L) A[x * PITCH + r] = make_float2(vv[i], 0.f);
    }
    __syncthreads();
    float2* res = fft_lines_t<L, NB, PITCH, -1>(A, B, tw);
    for (int e = threadIdx.x; e < NB * XH; e += blockDim.x) {
        const int r = e / XH, k = e % XH;
        const int row = row0 + r;
        if (row < nrows) out[(size_t)row * XH + k] = res[k * PITCH + r];
    }
}

template <int L, int SIGN, typename PS>
__global__ void __launch_bounds__(kFftThreads) cols_t(PS* __restrict__ data, int B,
                                                      const float2* __restrict__ tw) {
    constexpr int TB = cols_tb<L>();
    extern __shared__ float2 sm[];
    float2* P = sm;
    float2* Q = sm + L * TB;
    constexpr int PER = (L * TB + kFftThreads - 1) / kFftThreads;
    const int b0 = blockIdx.x * TB;
    const size_t base = (size_t)blockIdx.y * L * B;
    const int tb = min(TB, B - b0);
    float2 v[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) {          // all loads in flight before any store
        const int e = threadIdx.x + i * kFftThreads;
        const int l = e / TB, bb = e & (TB - 1);
        v[i] = (e < L * TB && bb < tb) ? ldc(data + base + (size_t)l * B + b0 + bb) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int e = threadIdx.x + i * kFftThreads;
        if (e < L * TB) P[e] = v[i];
    }
    __syncthreads();
    float2* res = fft_lines_t<L, TB, TB, SIGN>(P, Q, tw);
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int e = threadIdx.x + i * kFftThreads;
        const int l = e / TB, bb = e & (TB - 1);
        if (e < L * TB && bb < tb) stc(data + base + (size_t)l * B + b0 + bb, res[e]);
    }
}

template <int L, typename TS, typename PS>
__global__ void __launch_bounds__(kFftThreads) cols_mul_t(const float2* __restrict__ spec,
                                                          const TS* __restrict__ tspec,
                                                          PS* __restrict__ out, int B, int K,
                                                          const float2* __restrict__ tw) {
    constexpr int TB = cols_tb<L>();
    extern __shared__ float2 sm[];
    float2* P = sm;
    float2* Q = sm + L * TB;
    constexpr int PER = (L * TB + kFftThreads - 1) / kFftThreads;
    const int b0 = blockIdx.x * TB;
    const int tb = min(TB, B - b0);
    const size_t plane = (size_t)L * B;
    // this thread's elements of the image tile stay in registers
    float2 fi[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int e = threadIdx.x + i * kFftThreads;
        const int l = e / TB, bb = e & (TB - 1);
        fi[i] = (e < L * TB && bb < tb) ? spec[(size_t)l * B + b0 + bb] : make_float2(0.f, 0.f);
    }
    // component tiles: the next one is fetched while the current one is transformed
    float2 tv[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int e = threadIdx.x + i * kFftThreads;
        const int l = e / TB, bb = e & (TB - 1);
        tv[i] = (K > 0 && e < L * TB && bb < tb) ? ldgc(tspec + (size_t)l * B + b0 + bb)
                                                  : make_float2(0.f, 0.f);
    }
    for (int k = 0; k < K; ++k) {
        __syncthreads();
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int e = threadIdx.x + i * kFftThreads;
            if (e < L * TB) P[e] = cmulc(fi[i], tv[i]);
        }
        if (k + 1 < K) {
            const TS* ts = tspec + (size_t)(k + 1) * plane;
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                const int e = threadIdx.x + i * kFftThreads;
                const int l = e / TB, bb = e & (TB - 1);
                tv[i] = (e < L * TB && bb < tb) ? ldgc(ts + (size_t)l * B + b0 + bb)
                                                 : make_float2(0.f, 0.f);
            }
        }
        __syncthreads();
        float2* res = fft_lines_t<L, TB, TB, +1>(P, Q, tw);
        PS* o = out + (size_t)k * plane;
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int e = threadIdx.x + i * kFftThreads;
            const int l = e / TB, bb = e & (TB - 1);
            if (e < L * TB && bb < tb) stc(o + (size_t)l * B + b0 + bb, res[e]);
        }
    }
}

template <int L, typename PS, typename RT>
__global__ void __launch_bounds__(kFftThreads) rows_c2r_t(const PS* __restrict__ in, int X, int Y,
                                                          int Z, FftGeom g, RT* __restrict__ out,
                                                          int n_batch, const float2* __restrict__ tw) {
    constexpr int NB = rows_nb<L>();
    constexpr int PITCH = NB + 1;
    constexpr int XH = L / 2 + 1;
    extern __shared__ float2 sm[];
    float2* A = sm;
    float2* Bf = sm + L * PITCH;
    constexpr int PER = (NB * L + kFftThreads - 1) / kFftThreads;
    __shared__ long long row_out[NB];        // output offset of each row, -1 = not written
    const size_t rows_per_item = (size_t)g.Yp * g.Zp;
    const size_t nrows = rows_per_item * n_batch;
    const size_t row0 = (size_t)blockIdx.x * NB;
    if (threadIdx.x < NB) {
        const size_t row = row0 + threadIdx.x;
        long long off = -1;
        if (row < nrows) {
            const size_t item = row / rows_per_item;
            const int rr = (int)(row - item * rows_per_item);
            const int y = rr % g.Yp, z = rr / g.Yp;
            if (y < Y && z < Z) off = (long long)(item * ((size_t)X * Y * Z) + ((size_t)z * Y + y) * X);
        }
        row_out[threadIdx.x] = off;
    }
    float2 v[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) {          // loads first, Hermitian extension on the fly
        const int e = threadIdx.x + i * kFftThreads;
        const int r = e / L, x = e & (L - 1);
        const size_t row = row0 + r;
        v[i] = make_float2(0.f, 0.f);
        if (e < NB * L && row < nrows) {
            const PS* src = in + row * XH;
            if (x < XH) v[i] = ldc(src + x);
            else { float2 c = ldc(src + (L - x)); v[i] = make_float2(c.x, -c.y); }
        }
    }
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int e = threadIdx.x + i * kFftThreads;
        const int r = e / L, x = e & (L - 1);
        if (e < NB * L) A[x * PITCH + r] = v[i];
    }
    __syncthreads();
    float2* res = fft_lines_t<L, NB, PITCH, +1>(A, Bf, tw);   // ends with a barrier
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int e = threadIdx.x + i * kFftThreads;
        const int r = e / L, x = e & (L - 1);
        if (e >= NB * L || x >= X) continue;
        const long long off = row_out[r];
        if (off >= 0) str(out + off + x, res[x * PITCH + r].x);
    }
}


struct RunRowsR2C {
    const float* f; int X, Y, Z; FftGeom g; float2* spec; const float2* tw; cudaStream_t st;
    cudaError_t* err; int mode; const double* moments;
    template <int L> void operator()() {
        constexpr int NB = rows_nb<L>();
        const size_t smem = (size_t)2 * L * (NB + 1) * sizeof(float2);
        *err = cudaFuncSetAttribute(rows_r2c_t<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        const int nrows = g.Yp * g.Zp;
        rows_r2c_t<L><<<(nrows + NB - 1) / NB, kFftThreads, smem, st>>>(f, X, Y, Z, g, spec, tw, mode, moments);
    }
};

template <typename TS, typename PS>
struct RunColsMul {
    const float2* spec; const TS* tspec; PS* prod; int Bz, K; const float2* tw;
    cudaStream_t st; cudaError_t* err;
    template <int L> void operator()() {
        constexpr int TB = cols_tb<L>();
        const size_t smem = (size_t)2 * L * TB * sizeof(float2);
        *err = cudaFuncSetAttribute(cols_mul_t<L, TS, PS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        dim3 grid((Bz + TB - 1) / TB, 1);
        cols_mul_t<L, TS, PS><<<grid, kFftThreads, smem, st>>>(spec, tspec, prod, Bz, K, tw);
    }
};

template <typename PS, typename RT>
struct RunRowsC2R {
    const PS* prod; int X, Y, Z; FftGeom g; RT* corr; int K; const float2* tw;
    cudaStream_t st; cudaError_t* err;
    template <int L> void operator()() {
        constexpr int NB = rows_nb<L>();
        const size_t smem = (size_t)2 * L * (NB + 1) * sizeof(float2);
        *err = cudaFuncSetAttribute(rows_c2r_t<L, PS, RT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        const size_t nrows = (size_t)g.Yp * g.Zp * K;
        rows_c2r_t<L, PS, RT><<<(unsigned)((nrows + NB - 1) / NB), kFftThreads, smem, st>>>(
            prod, X, Y, Z, g, corr, K, tw);
    }
};

template <typename PS>
struct RunCols {
    PS* d; int B, na; const float2* tw; int sign; cudaStream_t st; cudaError_t* err;
    template <int LL> void operator()() {
        constexpr int TB = cols_tb<LL>();
        const size_t smem = (size_t)2 * LL * TB * sizeof(float2);
        dim3 grid((B + TB - 1) / TB, na);
        if (sign < 0) {
            *err = cudaFuncSetAttribute(cols_t<LL, -1, PS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            cols_t<LL, -1, PS><<<grid, kFftThreads, smem, st>>>(d, B, tw);
        } else {
            *err = cudaFuncSetAttribute(cols_t<LL, +1, PS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            cols_t<LL, +1, PS><<<grid, kFftThreads, smem, st>>>(d, B, tw);
        }
    }
};

// Dispatch helpers: call F.template operator()<L>() for a supported length.
template <typename F>
bool with_length(int L, F&& f) {
    switch (L) {
        case 16: f.template operator()<16>(); return true;
        case 32: f.template operator()<32>(); return true;
        case 64: f.template operator()<64>(); return true;
        case 128: f.template operator()<128>(); return true;
        case 256: f.template operator()<256>(); return true;
        case 512: f.template operator()<512>(); return true;
        case 1024: f.template operator()<1024>(); return true;
        default: return false;
    }
}

Radices radices_for(int L) {
    Radices rd{};
    int n = L;
    while (n % 4 == 0 && n > 1) { rd.r[rd.n++] = 4; n /= 4; }
    while (n % 2 == 0 && n > 1) { rd.r[rd.n++] = 2; n /= 2; }
    return rd;
}

int rows_per_cta(int L) {
    int nb = kTileElems / L;
    if (nb > 16) nb = 16;
    if (nb < 1) nb = 1;
    return nb;
}

int cols_per_cta(int L) {
    int tb = kTileElems / L;
    if (tb > 32) tb = 32;
    if (tb < 1) tb = 1;
    return tb;
}

}  // namespace

// Column lines (length L, element stride B) of `batch` consecutive blocks.
template <typename PS>
static ttm_status launch_cols_t(PS* data, int L, int B, int batch, const float2* tw, int sign,
                                cudaStream_t st, long long* cnt) {
    for (int a0 = 0; a0 < batch; a0 += 65535) {
        const int na = batch - a0 < 65535 ? batch - a0 : 65535;
        PS* d = data + (size_t)a0 * L * B;
        cudaError_t err = cudaSuccess;
        RunCols<PS> run{d, B, na, tw, sign, st, &err};
        if (!with_length(L, run)) {
            if constexpr (!std::is_same<PS, float2>::value) return TTM_ERR_UNSUPPORTED;
            else {
                const int TB = cols_per_cta(L);
                const size_t smem = (size_t)2 * L * TB * sizeof(float2);
                TTM_CUDA_TRY(cudaFuncSetAttribute(cols_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
                dim3 grid((B + TB - 1) / TB, na);
                cols_kernel<<<grid, kFftThreads, smem, st>>>(d, L, B, radices_for(L), tw, TB, sign);
            }
        }
        TTM_CUDA_TRY(err);
        TTM_TRY(after_launch(cnt));
    }
    return TTM_OK;
}

static ttm_status launch_cols(float2* data, int L, int B, int batch, const float2* tw, int sign,
                              cudaStream_t st, long long* cnt) {
    return launch_cols_t<float2>(data, L, B, batch, tw, sign, st, cnt);
}

bool fft_length_ok(int L) { return L >= 2 && L <= 4096 && (L & (L - 1)) == 0; }

int fft_good_length(int n) {
    int L = 2;
    while (L < n) L <<= 1;
    return L;
}

ttm_status launch_fft_forward(const float* f, int X, int Y, int Z, const FftShape& S,
                              float2* spec, cudaStream_t st, long long* cnt, int mode,
                              const double* moments) {
    FftGeom g{S.Xp, S.Yp, S.Zp, S.Xp / 2 + 1};
    cudaError_t err = cudaSuccess;
    {
        RunRowsR2C run{f, X, Y, Z, g, spec, S.d_tw_x, st, &err, mode, moments};
        if (mode != 0 && !fft_template_length(S.Xp)) return TTM_ERR_UNSUPPORTED;
        if (!with_length(S.Xp, run)) {
            const int NB = rows_per_cta(S.Xp);
            const size_t smem = (size_t)2 * S.Xp * (NB + 1) * sizeof(float2);
            TTM_CUDA_TRY(cudaFuncSetAttribute(rows_r2c_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            const int nrows = S.Yp * S.Zp;
            rows_r2c_kernel<<<(nrows + NB - 1) / NB, kFftThreads, smem, st>>>(
                f, X, Y, Z, g, spec, radices_for(S.Xp), S.d_tw_x, NB);
        }
        TTM_CUDA_TRY(err);
        TTM_TRY(after_launch(cnt));
    }
    TTM_TRY(launch_cols(spec, S.Yp, g.Xh, S.Zp, S.d_tw_y, -1, st, cnt));            // y lines
    TTM_TRY(launch_cols(spec, S.Zp, S.Yp * g.Xh, 1, S.d_tw_z, -1, st, cnt));       // z lines
    return TTM_OK;
}

template <typename TS, typename PS>
static ttm_status spectrum_inverse_z_t(const float2* spec, const TS* tspec, int K, const FftShape& S,
                                       PS* prod, cudaStream_t st, long long* cnt) {
    const int Xh = S.Xp / 2 + 1;
    const int Bz = S.Yp * Xh;
    cudaError_t err = cudaSuccess;
    RunColsMul<TS, PS> run{spec, tspec, prod, Bz, K, S.d_tw_z, st, &err};
    if (!with_length(S.Zp, run)) {
        if constexpr (!std::is_same<TS, float2>::value || !std::is_same<PS, float2>::value)
            return TTM_ERR_UNSUPPORTED;
        else {
            const int TB = cols_per_cta(S.Zp);
            const size_t smem = (size_t)3 * S.Zp * TB * sizeof(float2);
            TTM_CUDA_TRY(cudaFuncSetAttribute(cols_mul_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            dim3 grid((Bz + TB - 1) / TB, 1);
            cols_mul_kernel<<<grid, kFftThreads, smem, st>>>(spec, tspec, prod, S.Zp, Bz, K,
                                                             radices_for(S.Zp), S.d_tw_z, TB);
        }
    }
    TTM_CUDA_TRY(err);
    return after_launch(cnt);
}

template <typename PS, typename RT>
static ttm_status inverse_yx_t(PS* prod, int K, int X, int Y, int Z, const FftShape& S, RT* corr,
                               cudaStream_t st, long long* cnt) {
    FftGeom g{S.Xp, S.Yp, S.Zp, S.Xp / 2 + 1};
    TTM_TRY(launch_cols_t<PS>(prod, S.Yp, g.Xh, K * S.Zp, S.d_tw_y, +1, st, cnt));
    cudaError_t err = cudaSuccess;
    RunRowsC2R<PS, RT> run{prod, X, Y, Z, g, corr, K, S.d_tw_x, st, &err};
    if (!with_length(S.Xp, run)) {
        if constexpr (!std::is_same<PS, float2>::value || !std::is_same<RT, float>::value)
            return TTM_ERR_UNSUPPORTED;
        else {
            const int NB = rows_per_cta(S.Xp);
            const size_t smem = (size_t)2 * S.Xp * (NB + 1) * sizeof(float2);
            TTM_CUDA_TRY(cudaFuncSetAttribute(rows_c2r_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            const size_t nrows = (size_t)S.Yp * S.Zp * K;
            rows_c2r_kernel<<<(unsigned)((nrows + NB - 1) / NB), kFftThreads, smem, st>>>(
                prod, X, Y, Z, g, corr, K, radices_for(S.Xp), S.d_tw_x, NB);
        }
    }
    TTM_CUDA_TRY(err);
    return after_launch(cnt);
}

ttm_status launch_fft_spectrum_inverse_z(const float2* spec, const float2* tspec, int K,
                                         const FftShape& S, float2* prod, cudaStream_t st,
                                         long long* cnt) {
    return spectrum_inverse_z_t<float2, float2>(spec, tspec, K, S, prod, st, cnt);
}

ttm_status launch_fft_inverse_yx(float2* prod, int K, int X, int Y, int Z, const FftShape& S,
                                 float* corr, cudaStream_t st, long long* cnt) {
    return inverse_yx_t<float2, float>(prod, K, X, Y, Z, S, corr, st, cnt);
}

// mixed precision: bf16 template spectra, products and correlation maps
ttm_status launch_fft_spectrum_inverse_z_bf16(const float2* spec, const void* tspec, int K,
                                              const FftShape& S, void* prod, cudaStream_t st,
                                              long long* cnt) {
    return spectrum_inverse_z_t<__nv_bfloat162, __nv_bfloat162>(
        spec, reinterpret_cast<const __nv_bfloat162*>(tspec), K, S,
        reinterpret_cast<__nv_bfloat162*>(prod), st, cnt);
}

ttm_status launch_fft_inverse_yx_bf16(void* prod, int K, int X, int Y, int Z, const FftShape& S,
                                      void* corr, cudaStream_t st, long long* cnt) {
    return inverse_yx_t<__nv_bfloat162, __nv_bfloat16>(
        reinterpret_cast<__nv_bfloat162*>(prod), K, X, Y, Z, S,
        reinterpret_cast<__nv_bfloat16*>(corr), st, cnt);
}

__global__ void to_bf16_kernel(const float2* __restrict__ a, __nv_bfloat162* __restrict__ b, size_t n) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = __float22bfloat162_rn(a[i]);
}

ttm_status launch_spectra_to_bf16(const float2* a, void* b, size_t n, cudaStream_t st, long long* cnt) {
    to_bf16_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, reinterpret_cast<__nv_bfloat162*>(b), n);
    return after_launch(cnt);
}

bool fft_template_length(int L) {
    return L == 16 || L == 32 || L == 64 || L == 128 || L == 256 || L == 512 || L == 1024;
}

// w from the FFT-based window sums of (f - mean) and (f - mean)^2 (Algorithm 1):
// V = S2 - S1^2 / m_sum in FP64; interior only; floor 1e-6 m_sum var(f).
__global__ void stats_from_sums_kernel(const float* __restrict__ s1, const float* __restrict__ s2,
                                       float* __restrict__ w, int X, int Y, int Z, int s,
                                       double mask_sum, const double* __restrict__ moments) {
    const size_t n = (size_t)X * Y * Z;
    const size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int x = (int)(v % X), y = (int)((v / X) % Y), z = (int)(v / ((size_t)X * Y));
    float out = 0.f;
    if (interior(x, X, s) && interior(y, Y, s) && interior(z, Z, s)) {
        const double nv = (double)n;
        const double mean = moments[0] / nv;
        const double var_f = fmax(moments[1] / nv - mean * mean, 0.0);
        const double S1 = s1[v], S2 = s2[v];
        const double V = S2 - S1 * S1 / mask_sum;
        if (V > 1e-6 * mask_sum * var_f) out = rsqrtf((float)V);
    }
    w[v] = out;
}

ttm_status launch_stats_from_sums(const float* s1, const float* s2, float* w, int X, int Y, int Z,
                                  int s, double mask_sum, const double* moments, cudaStream_t st,
                                  long long* cnt) {
    const size_t n = (size_t)X * Y * Z;
    stats_from_sums_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(s1, s2, w, X, Y, Z, s,
                                                                        mask_sum, moments);
    return after_launch(cnt);
}

ttm_status launch_template_spectra(const float* comp, int K, int s, const FftShape& S,
                                   float* pad, float2* tspec, cudaStream_t st, long long* cnt) {
    FftGeom g{S.Xp, S.Yp, S.Zp, S.Xp / 2 + 1};
    const size_t nreal = (size_t)S.Xp * S.Yp * S.Zp;
    const size_t nspec = (size_t)g.Xh * S.Yp * S.Zp;
    const int s3 = s * s * s;
    for (int k = 0; k < K; ++k) {
        TTM_CUDA_TRY(cudaMemsetAsync(pad, 0, nreal * sizeof(float), st));
        scatter_component_kernel<<<(s3 + 255) / 256, 256, 0, st>>>(comp + (size_t)k * s3, s, g, pad);
        TTM_TRY(after_launch(cnt));
        float2* dst = tspec + (size_t)k * nspec;
        TTM_TRY(launch_fft_forward(pad, S.Xp, S.Yp, S.Zp, S, dst, st, cnt, 0, nullptr));
        scale_kernel<<<(unsigned)((nspec + 255) / 256), 256, 0, st>>>(dst, nspec, 1.0f / (float)nreal);
        TTM_TRY(after_launch(cnt));
    }
    return TTM_OK;
}

}  // namespace ttm
