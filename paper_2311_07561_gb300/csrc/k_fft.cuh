// Compile-time-length FFT passes (header of k_fft.cu and the k_fft_len*.cu
// files, which instantiate FftLen<L> for the supported lengths).
//
// Every pass moves a tile of whole 1D lines into shared memory, transforms
// them there with Stockham autosort stages whose radices (16, 8, 4, 2, 3, 5)
// are fixed at compile time for the length (the small DFTs run in registers,
// two shared-memory buffers ping-pong between stages), and writes the tile
// back, so each pass reads and writes HBM once:
//   rows_r2c_t    x lines of the real volume -> half-spectrum rows
//   cols_t        y or z lines of a half spectrum (strided), in place
//   cols_mul_t    z lines of the image spectrum times conj(template spectrum)
//                 for all K components: the image tile is read once and kept
//                 in registers while the K component tiles stream through
//   rows_c2r_t    half-spectrum rows -> real x lines (Hermitian extension)
// Twiddles exp(-2 pi i k / L) come from a table computed on the host in FP64.
// Lengths: 2^p 3^a 5^b, even, listed in TTM_FFT_LENGTHS.
#pragma once

#include <cuda_bf16.h>

#include "ttm_internal.h"

// supported compile-time lengths (x, y and z extents of padded FFT boxes)
#define TTM_FFT_LENGTHS(X) \
    X(16) X(32) X(48) X(64) X(80) X(96) X(128) X(144) X(160) X(192) X(240) X(256) X(288) \
    X(320) X(384) X(480) X(512) X(576) X(640) X(768) X(960) X(1024)

namespace ttm {

struct FftGeom {
    int Xp, Yp, Zp, Xh;
};

// Lines of a column pass: plane p = p0 + blockIdx.y (or the persistent tile's
// plane) is plane z0 + (p % nz) of item p / nz, items zstride planes apart;
// line samples lo..hi are stored (the rest are computed and dropped).
struct ColsMap {
    int p0, nz, zstride, z0, lo, hi;
};

namespace fftk {

constexpr int kFftThreads = 256;

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

// ---- compile-time-length Stockham stages with radix up to 16 in registers ----
// Small DFTs (sign -1 forward, +1 inverse).  DFT16 = 4 x 4 with the internal
// twiddles W16^(n2 k1); its outputs come back in transposed order.
constexpr float kC8 = 0.92387953251128674f;   // cos(pi/8)
constexpr float kS8 = 0.38268343236508978f;   // sin(pi/8)
constexpr float kR2 = 0.70710678118654752f;   // sqrt(2)/2
constexpr float kS3 = 0.86602540378443865f;   // sin(2 pi/3)
constexpr float kC51 = 0.30901699437494742f;  // cos(2 pi/5)
constexpr float kC52 = -0.80901699437494742f; // cos(4 pi/5)
constexpr float kS51 = 0.95105651629515357f;  // sin(2 pi/5)
constexpr float kS52 = 0.58778525229247313f;  // sin(4 pi/5)

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
        // twiddle W8^(n2 k1) = W16^(2 n2 k1) (k1 = 2: -i, a swap)
#pragma unroll
        for (int k1 = 1; k1 < 4; ++k1)
            u[1 + 2 * k1] = k1 == 2 ? mul_mi<SIGN>(u[1 + 2 * k1]) : cmul(u[1 + 2 * k1], w16<SIGN>(2 * k1));
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            float2 a = u[2 * k1], b = u[2 * k1 + 1];
            v[k1] = cadd(a, b);          // k2 = 0 -> k = k1
            v[k1 + 4] = csub(a, b);      // k2 = 1 -> k = k1 + 4
        }
    } else if constexpr (R == 3) {
        // X1,2 = x0 - (x1 + x2)/2 +- SIGN i (sqrt(3)/2) (x1 - x2)
        const float2 s = cadd(v[1], v[2]);
        const float2 d = mul_mi<SIGN>(csub(v[1], v[2]));
        const float2 m = make_float2(v[0].x - 0.5f * s.x, v[0].y - 0.5f * s.y);
        v[0] = cadd(v[0], s);
        v[1] = make_float2(m.x + kS3 * d.x, m.y + kS3 * d.y);
        v[2] = make_float2(m.x - kS3 * d.x, m.y - kS3 * d.y);
    } else if constexpr (R == 5) {
        // with t1 = x1 + x4, t2 = x2 + x3, t3 = x1 - x4, t4 = x2 - x3:
        //   X1,4 = x0 + c1 t1 + c2 t2 +- SIGN i (s1 t3 + s2 t4)
        //   X2,3 = x0 + c2 t1 + c1 t2 +- SIGN i (s2 t3 - s1 t4)
        const float2 t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
        const float2 t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
        const float2 a1 = make_float2(v[0].x + kC51 * t1.x + kC52 * t2.x, v[0].y + kC51 * t1.y + kC52 * t2.y);
        const float2 a2 = make_float2(v[0].x + kC52 * t1.x + kC51 * t2.x, v[0].y + kC52 * t1.y + kC51 * t2.y);
        const float2 b1 = mul_mi<SIGN>(make_float2(kS51 * t3.x + kS52 * t4.x, kS51 * t3.y + kS52 * t4.y));
        const float2 b2 = mul_mi<SIGN>(make_float2(kS52 * t3.x - kS51 * t4.x, kS52 * t3.y - kS51 * t4.y));
        v[0] = cadd(v[0], cadd(t1, t2));
        v[1] = cadd(a1, b1);
        v[4] = csub(a1, b1);
        v[2] = cadd(a2, b2);
        v[3] = csub(a2, b2);
    } else {
        static_assert(R == 16, "radix 2, 3, 4, 5, 8 or 16");
        // n = 4 n1 + n2, k = k1 + 4 k2
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
            for (int n2 = 1; n2 < 4; ++n2)   // W16^4 = -i: a swap
                u[4 * k1 + n2] = n2 * k1 == 4 ? mul_mi<SIGN>(u[4 * k1 + n2])
                                              : cmul(u[4 * k1 + n2], w16<SIGN>(n2 * k1));
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            float2 a = u[4 * k1], b = u[4 * k1 + 1], c = u[4 * k1 + 2], d = u[4 * k1 + 3];
            dft4<SIGN>(a, b, c, d);
            v[k1] = a; v[k1 + 4] = b; v[k1 + 8] = c; v[k1 + 12] = d;     // k = k1 + 4 k2
        }
    }
}

// radix of stage st for length L: 16s first, the remaining factor last
// Stage radices of a length L = 2^p 3^a 5^b: radix 16 while it divides the
// power of two, the remaining power of two (2, 4 or 8), then a radix-3 and
// b radix-5 stages.
__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n >> 1); }
__host__ __device__ constexpr int pow2_part(int L) { return L & -L; }
__host__ __device__ constexpr int count_factor(int L, int f) {
    return (L > 1 && L % f == 0) ? 1 + count_factor(L / f, f) : 0;
}
__host__ __device__ constexpr bool smooth235(int L) {
    int m = L / pow2_part(L);
    while (m % 3 == 0) m /= 3;
    while (m % 5 == 0) m /= 5;
    return L >= 2 && m == 1;
}
__host__ __device__ constexpr int n_stages(int L) {
    return ilog2c(pow2_part(L)) / 4 + ((ilog2c(pow2_part(L)) % 4) ? 1 : 0) + count_factor(L, 3) +
           count_factor(L, 5);
}
__host__ __device__ constexpr int stage_radix(int L, int st) {
    const int p = ilog2c(pow2_part(L));
    if (st < p / 4) return 16;
    st -= p / 4;
    if (p % 4) {
        if (st == 0) return 1 << (p % 4);
        st -= 1;
    }
    return st < count_factor(L, 3) ? 3 : 5;
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
        const int jm = j % NS;
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

// lines per CTA: the largest power of two with at most 4096 elements per
// shared-memory buffer (16 rows, 32 columns at most)
__host__ __device__ constexpr int pow2_floor(int n) { return n < 2 ? 1 : 2 * pow2_floor(n / 2); }
template <int L> constexpr int rows_nb() { return pow2_floor(4096 / L) > 16 ? 16 : pow2_floor(4096 / L); }
template <int L> constexpr int cols_tb() { return pow2_floor(4096 / L) > 32 ? 32 : pow2_floor(4096 / L); }
// column passes over bf16 storage (4 bytes per complex) take at least 8
// columns, so that every row segment of a tile is a whole 32-byte sector
template <int L, typename PS>
constexpr int cols_tb_s() { return (sizeof(PS) < 8 && cols_tb<L>() < 8) ? 8 : cols_tb<L>(); }

// ---- the four passes with a compile-time line length ---------------------
// mode 0 transforms f, mode 1 (f - mean), mode 2 (f - mean)^2 with mean =
// moments[0] / (X Y Z) (the shift removes the cancellation in the local
// variance); mode 2 also adds sum (f - mean)^4 into moments[2] (the size of
// the FFT rounding error of the window sums, see stats_from_sums_kernel)
template <int L>
__global__ void __launch_bounds__(kFftThreads) rows_r2c_t(const float* __restrict__ f, int X, int Y,
                                                          int Z, FftGeom g, float2* __restrict__ out,
                                                          const float2* __restrict__ tw, int mode,
                                                          double* __restrict__ moments) {
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
        const int r = e / L, x = e % L;
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
        const int r = e / L, x = e % L;
        if (e < NB * L) A[x * PITCH + r] = make_float2(vv[i], 0.f);
    }
    if (mode == 2) {
        __shared__ double part[kFftThreads / 32];
        float q = 0.f;
#pragma unroll
        for (int i = 0; i < PER; ++i) q = fmaf(vv[i], vv[i], q);
        double d = q;
        for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
        if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = d;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int k = 0; k < kFftThreads / 32; ++k) t += part[k];
            if (t != 0.0) atomicAdd(moments + 2, t);
        }
    }
    __syncthreads();
    float2* res = fft_lines_t<L, NB, PITCH, -1>(A, B, tw);
    for (int e = threadIdx.x; e < NB * XH; e += blockDim.x) {
        const int r = e / XH, k = e % XH;
        const int row = row0 + r;
        if (row < nrows) out[(size_t)row * XH + k] = res[k * PITCH + r];
    }
}

__device__ __forceinline__ size_t cols_plane_base(const ColsMap& mp, size_t p, int L, int B) {
    const size_t item = p / (size_t)mp.nz;
    const size_t zz = p - item * (size_t)mp.nz;
    return (item * (size_t)mp.zstride + (size_t)mp.z0 + zz) * (size_t)L * (size_t)B;
}

template <int L, int SIGN, typename PS>
__global__ void __launch_bounds__(kFftThreads) cols_t(PS* __restrict__ data, int B,
                                                      const float2* __restrict__ tw, ColsMap mp) {
    constexpr int TB = cols_tb_s<L, PS>();
    extern __shared__ float2 sm[];
    float2* P = sm;
    float2* Q = sm + L * TB;
    constexpr int PER = (L * TB + kFftThreads - 1) / kFftThreads;
    const int b0 = blockIdx.x * TB;
    const size_t base = cols_plane_base(mp, (size_t)mp.p0 + blockIdx.y, L, B);
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
        if (e < L * TB && bb < tb && l >= mp.lo && l <= mp.hi)
            stc(data + base + (size_t)l * B + b0 + bb, res[e]);
    }
}

// The same pass for long lines (one or two CTAs per SM): persistent CTAs walk
// the (column tile, plane) tiles with a stride of gridDim.x, and the raw
// elements of the next tile are loaded into registers while the current one
// is transformed, so loads stay in flight through the Stockham stages.
template <int L, int SIGN, typename PS>
__global__ void __launch_bounds__(kFftThreads, 1) cols_pf_t(PS* __restrict__ data, int B,
                                                            const float2* __restrict__ tw,
                                                            ColsMap mp, int ntb, size_t ntiles) {
    constexpr int TB = cols_tb_s<L, PS>();
    extern __shared__ float2 sm[];
    float2* P = sm;
    float2* Q = sm + L * TB;
    constexpr int PER = (L * TB + kFftThreads - 1) / kFftThreads;
    PS nv[PER];
    auto load = [&](size_t tile) {
        const size_t plane = tile / (size_t)ntb;
        const int b0 = (int)(tile - plane * (size_t)ntb) * TB;
        const size_t base = cols_plane_base(mp, (size_t)mp.p0 + plane, L, B);
        const int tb = min(TB, B - b0);
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int e = threadIdx.x + i * kFftThreads;
            const int l = e / TB, bb = e & (TB - 1);
            if (e < L * TB && bb < tb) nv[i] = data[base + (size_t)l * B + b0 + bb];
        }
    };
    size_t tile = blockIdx.x;
    if (tile >= ntiles) return;
    load(tile);
    for (; tile < ntiles; tile += gridDim.x) {
        const size_t plane = tile / (size_t)ntb;
        const int b0 = (int)(tile - plane * (size_t)ntb) * TB;
        const size_t base = cols_plane_base(mp, (size_t)mp.p0 + plane, L, B);
        const int tb = min(TB, B - b0);
        __syncthreads();                      // the previous tile's result is stored
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int e = threadIdx.x + i * kFftThreads;
            const int bb = e & (TB - 1);
            if (e < L * TB) P[e] = bb < tb ? ldc(&nv[i]) : make_float2(0.f, 0.f);
        }
        if (tile + gridDim.x < ntiles) load(tile + gridDim.x);
        __syncthreads();
        float2* res = fft_lines_t<L, TB, TB, SIGN>(P, Q, tw);
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int e = threadIdx.x + i * kFftThreads;
            const int l = e / TB, bb = e & (TB - 1);
            if (e < L * TB && bb < tb && l >= mp.lo && l <= mp.hi)
                stc(data + base + (size_t)l * B + b0 + bb, res[e]);
        }
    }
}

template <int L, typename TS, typename PS>
__global__ void __launch_bounds__(kFftThreads, 2) cols_mul_t(const float2* __restrict__ spec,
                                                          const TS* __restrict__ tspec,
                                                          PS* __restrict__ out, int B, int K,
                                                          const float2* __restrict__ tw, int lo,
                                                          int hi) {
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
            if (e < L * TB && bb < tb && l >= lo && l <= hi) stc(o + (size_t)l * B + b0 + bb, res[e]);
        }
    }
}

// ---- stages with functor input/output (first stage reads a staged tile,
// last stage writes global memory) --------------------------------------
template <int L, int ST>
constexpr int ns_before() {
    int ns = 1;
    for (int s = 0; s < ST; ++s) ns *= stage_radix(L, s);
    return ns;
}

// One Stockham stage of radix R: element x of line `line` comes from
// src(x, line) and goes to dst(x, line, v).  LINE_FAST: consecutive threads
// take consecutive lines (shared-memory destinations), else consecutive
// butterflies, so that a stage writing global memory stores consecutive x.
template <int L, int R, int NS, int NB, int SIGN, bool LINE_FAST, class Src, class Dst>
__device__ __forceinline__ void stage_io(const Src& src, const Dst& dst,
                                         const float2* __restrict__ tw) {
    constexpr int NBF = L / R;
    constexpr int STRIDE_TW = L / (NS * R);
    for (int idx = threadIdx.x; idx < NBF * NB; idx += blockDim.x) {
        const int line = LINE_FAST ? (idx & (NB - 1)) : idx / NBF;
        const int j = LINE_FAST ? idx / NB : idx % NBF;
        const int jm = j % NS;
        const int idxD = (j - jm) * R + jm;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src(j + r * NBF, line);
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
        for (int r = 0; r < R; ++r) dst(idxD + r * NS, line, v[r]);
    }
}

// All stages of NB lines: the first reads src, the middle ones ping-pong
// between a and b (pitch PITCH, x-major), the last writes out.
template <int L, int ST, int NB, int PITCH, int SIGN, class Src, class Out>
__device__ __forceinline__ void stages_io(const Src& src, float2* a, float2* b, const Out& out,
                                          const float2* __restrict__ tw) {
    constexpr int R = stage_radix(L, ST);
    constexpr int NS = ns_before<L, ST>();
    if constexpr (ST + 1 == n_stages(L)) {
        stage_io<L, R, NS, NB, SIGN, false>(src, out, tw);
    } else {
        stage_io<L, R, NS, NB, SIGN, true>(
            src, [a](int x, int line, float2 v) { a[x * PITCH + line] = v; }, tw);
        __syncthreads();
        stages_io<L, ST + 1, NB, PITCH, SIGN>(
            [a](int x, int line) { return a[x * PITCH + line]; }, b, a, out, tw);
    }
}

// ---- half-spectrum rows -> real x lines (inverse), persistent -----------
// A tile is NB consecutive half-spectrum rows (contiguous in memory) of one z
// plane of one batch item; only the planes z0..z1 and the rows y0..y1 of the
// keep box are visited (tiles start at multiples of NB rows, so every tile is
// one aligned bulk copy).  Each CTA walks tiles with a stride of gridDim.x;
// the next NST - 1 tiles are in flight in a ring of staging buffers (bulk
// copies completing on one mbarrier each) while the current one is
// transformed.  The first stage reads the staged rows with the Hermitian
// extension X[L - x] = conj X[x]; the last stage stores the real parts of the
// kept samples x0..x1 straight to the X x Y x Z maps (out is batch-major,
// X Y Z floats per item).  Copy waits are bounded: on expiry the CTA records
// TTM_ERR_TIMEOUT, waits once more for its copies in flight and exits.
template <int L>
constexpr int c2r_stages_buffers() { return n_stages(L) >= 3 ? 2 : 1; }

template <int L, typename PS>
constexpr uint32_t c2r_tile_bytes() { return (uint32_t)(rows_nb<L>() * (L / 2 + 1) * sizeof(PS)); }

template <int L>
constexpr size_t c2r_fft_bytes() {
    return (size_t)c2r_stages_buffers<L>() * L * (rows_nb<L>() + 1) * sizeof(float2);
}

// staging ring depth: as deep as 4 while two CTAs still fit on an SM
template <int L, typename PS>
constexpr int c2r_ring() {
    constexpr size_t budget = 113u * 1024u;
    return (4 * (size_t)c2r_tile_bytes<L, PS>() + c2r_fft_bytes<L>() <= budget) ? 4
         : (3 * (size_t)c2r_tile_bytes<L, PS>() + c2r_fft_bytes<L>() <= budget) ? 3 : 2;
}

template <int L, typename PS>
constexpr size_t c2r_smem() {
    return (size_t)c2r_ring<L, PS>() * c2r_tile_bytes<L, PS>() + c2r_fft_bytes<L>();
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void bulk_to_smem(uint32_t dst, const void* src, uint32_t bytes,
                                             uint32_t bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
        ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t phase) {
    for (long it = 0; it < (1L << 24); ++it) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}

template <int L, typename PS, typename RT>
__global__ void __launch_bounds__(kFftThreads) rows_c2r_t(const PS* __restrict__ in, int X, int Y,
                                                          int Z, FftGeom g, RT* __restrict__ out,
                                                          int n_batch, const float2* __restrict__ tw,
                                                          int* status, FftKeep keep) {
    constexpr int NB = rows_nb<L>();
    constexpr int PITCH = NB + 1;
    constexpr int XH = L / 2 + 1;
    constexpr int NST = c2r_ring<L, PS>();
    constexpr uint32_t TILE = c2r_tile_bytes<L, PS>();
    static_assert(TILE % 16 == 0, "bulk copies move multiples of 16 bytes");
    extern __shared__ __align__(128) unsigned char smraw[];
    float2* a = reinterpret_cast<float2*>(smraw + NST * TILE);
    float2* b = a + (c2r_stages_buffers<L>() == 2 ? L * PITCH : 0);
    __shared__ __align__(8) uint64_t bars[NST];
    __shared__ long long row_out[NB];        // output offset of each row, -1 = not written
    // kept rows: planes z0..z1, rows from y0 rounded down to a multiple of NB
    // (every tile starts on a 16-byte boundary) up to y1
    const int y_first = keep.y0 & ~(NB - 1);
    const int nty = (keep.y1 - y_first) / NB + 1;
    const int nz = keep.z1 - keep.z0 + 1;
    const size_t ntiles = (size_t)n_batch * nz * nty;
    auto tile_src = [&](size_t t, int& y_start, size_t& item, int& z) {
        const size_t per_item = (size_t)nz * nty;
        item = t / per_item;
        const size_t r = t - item * per_item;
        const int zz = (int)(r / (size_t)nty);
        y_start = y_first + (int)(r - (size_t)zz * nty) * NB;
        z = keep.z0 + zz;
        return in + ((item * (size_t)g.Zp + (size_t)z) * (size_t)g.Yp + (size_t)y_start) * XH;
    };
    const uint32_t sbase = smem_addr(smraw);
    if (threadIdx.x == 0) {
        for (int q = 0; q < NST; ++q)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&bars[q])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    }
    __syncthreads();
    if ((size_t)blockIdx.x >= ntiles) return;
    uint32_t pending = 0u;                   // thread 0: buffers with a copy in flight
    if (threadIdx.x == 0) {
        for (int q = 0; q < NST - 1; ++q) {
            const size_t t = blockIdx.x + (size_t)q * gridDim.x;
            if (t >= ntiles) break;
            int ys, z;
            size_t item;
            bulk_to_smem(sbase + (uint32_t)q * TILE, tile_src(t, ys, item, z), TILE,
                         smem_addr(&bars[q]));
            pending |= 1u << q;
        }
    }
    uint32_t phase = 0u;
    int it = 0;
    for (size_t tile = blockIdx.x; tile < ntiles; ++it, tile += gridDim.x) {
        const int buf = it % NST;
        if (threadIdx.x == 0) {
            const size_t ahead = tile + (size_t)(NST - 1) * gridDim.x;
            if (ahead < ntiles) {
                const int nb = (it + NST - 1) % NST;
                int ys, z;
                size_t item;
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                bulk_to_smem(sbase + (uint32_t)nb * TILE, tile_src(ahead, ys, item, z), TILE,
                             smem_addr(&bars[nb]));
                pending |= 1u << nb;
            }
        }
        if (threadIdx.x < NB) {
            int ys, z;
            size_t item;
            tile_src(tile, ys, item, z);
            const int y = ys + threadIdx.x;
            row_out[threadIdx.x] = (y >= keep.y0 && y <= keep.y1 && y < Y && z < Z)
                ? (long long)(item * ((size_t)X * Y * Z) + ((size_t)z * Y + y) * X) : -1;
        }
        const bool ok = bar_wait(smem_addr(&bars[buf]), (phase >> buf) & 1u);
        phase ^= 1u << buf;
        if (threadIdx.x == 0) pending &= ~(1u << buf);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                atomicExch(status, TTM_ERR_TIMEOUT);
                for (int q = 0; q < NST; ++q)
                    if ((pending >> q) & 1u) bar_wait(smem_addr(&bars[q]), (phase >> q) & 1u);
            }
            return;
        }
        const PS* S = reinterpret_cast<const PS*>(smraw + (size_t)buf * TILE);
        const int xk0 = keep.x0, xk1 = min(keep.x1, X - 1);
        stages_io<L, 0, NB, PITCH, +1>(
            [S](int x, int line) {
                if (x < XH) return ldc(S + line * XH + x);
                const float2 c = ldc(S + line * XH + (L - x));
                return make_float2(c.x, -c.y);
            },
            a, b,
            [out, xk0, xk1](int x, int line, float2 v) {
                const long long off = row_out[line];
                if (x >= xk0 && x <= xk1 && off >= 0) str(out + off + x, v.x);
            },
            tw);
        __syncthreads();     // staging buffer, a/b and row_out are reused
    }
}

}  // namespace fftk
}  // namespace ttm

#include "k_fft2.cuh"

namespace ttm {

// Launchers of the four passes for one compile-time length L.  Each returns
// the CUDA error of its attribute call or launch.  Defined out of line so that
// `extern template` keeps the kernels in the k_fft_len*.cu objects.  The
// column passes take a ColsMap (na planes), the fused multiply the range of
// stored z, the row inverse the keep box.
template <int L>
struct FftLen {
    static cudaError_t rows_r2c(const float* f, int X, int Y, int Z, FftGeom g, float2* spec,
                                const float2* tw, int mode, double* moments, cudaStream_t st);
    static cudaError_t cols(float2* d, int B, int na, ColsMap mp, const float2* tw, int sign,
                            cudaStream_t st);
    static cudaError_t cols_bf(__nv_bfloat162* d, int B, int na, ColsMap mp, const float2* tw,
                               int sign, cudaStream_t st);
    static cudaError_t cols_mul(const float2* spec, const float2* tspec, float2* prod, int Bz, int K,
                                const float2* tw, int lo, int hi, cudaStream_t st);
    static cudaError_t cols_mul_bf(const float2* spec, const __nv_bfloat162* tspec,
                                   __nv_bfloat162* prod, int Bz, int K, const float2* tw, int lo,
                                   int hi, cudaStream_t st);
    static cudaError_t rows_c2r(const float2* prod, int X, int Y, int Z, FftGeom g, float* corr,
                                int K, const float2* tw, int* status, FftKeep keep, cudaStream_t st);
    static cudaError_t rows_c2r_bf(const __nv_bfloat162* prod, int X, int Y, int Z, FftGeom g,
                                   __nv_bfloat16* corr, int K, const float2* tw, int* status,
                                   FftKeep keep, cudaStream_t st);
};

namespace fftk {

inline cudaError_t sm_count(int* sms) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    return cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev);
}

// lengths whose column tiles leave one CTA per SM take the persistent pass
template <int L, typename PS>
constexpr bool cols_persistent() { return 2 * (size_t)L * cols_tb_s<L, PS>() * sizeof(float2) > 100u * 1024u; }

// persistent grid of a kernel: SMs x resident CTAs per SM, at most `work`
template <class Kern>
inline cudaError_t persistent_grid(Kern kern, size_t smem, size_t work, unsigned* grid) {
    int sms = 0, per_sm = 0;
    cudaError_t e = sm_count(&sms);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTwoThreads, smem);
    if (e != cudaSuccess) return e;
    const size_t cap = (size_t)sms * (per_sm > 0 ? per_sm : 1);
    *grid = (unsigned)(work < cap ? work : cap);
    return cudaSuccess;
}

template <int L, int SIGN, typename PS>
cudaError_t run_cols(PS* d, int B, int na, ColsMap mp, const float2* tw, cudaStream_t st) {
    if constexpr (two_level<L>()) {
        constexpr int L1 = TwoLevel<L>::L1, L2 = TwoLevel<L>::L2;
        constexpr int TB = kTwoThreads / L1;
        constexpr size_t smem = two_cols_smem<L1, L2>();
        auto kern = cols2_t<L1, L2, SIGN, PS>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        const int ntb = (B + TB - 1) / TB;
        const size_t ntiles = (size_t)ntb * na;
        unsigned grid = 0;
        if ((e = persistent_grid(kern, smem, ntiles, &grid)) != cudaSuccess) return e;
        if (grid == 0) return cudaSuccess;
        kern<<<grid, kTwoThreads, smem, st>>>(d, B, tw, mp, ntb, ntiles);
        return cudaGetLastError();
    }
    constexpr int TB = cols_tb_s<L, PS>();
    const size_t smem = (size_t)2 * L * TB * sizeof(float2);
    const int ntb = (B + TB - 1) / TB;
    if constexpr (cols_persistent<L, PS>()) {
        cudaError_t e = cudaFuncSetAttribute(cols_pf_t<L, SIGN, PS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int sms = 0;
        if ((e = sm_count(&sms)) != cudaSuccess) return e;
        const size_t ntiles = (size_t)ntb * na;
        const unsigned grid = (unsigned)(ntiles < (size_t)sms ? ntiles : (size_t)sms);
        if (grid == 0) return cudaSuccess;
        cols_pf_t<L, SIGN, PS><<<grid, kFftThreads, smem, st>>>(d, B, tw, mp, ntb, ntiles);
        return cudaGetLastError();
    } else {
        cudaError_t e = cudaFuncSetAttribute(cols_t<L, SIGN, PS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        for (int a0 = 0; a0 < na; a0 += 65535) {
            const int n = na - a0 < 65535 ? na - a0 : 65535;
            ColsMap m2 = mp;
            m2.p0 = mp.p0 + a0;
            dim3 grid(ntb, n);
            cols_t<L, SIGN, PS><<<grid, kFftThreads, smem, st>>>(d, B, tw, m2);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
}

template <int L, typename TS, typename PS>
cudaError_t run_cols_mul(const float2* spec, const TS* tspec, PS* prod, int Bz, int K,
                         const float2* tw, int lo, int hi, cudaStream_t st) {
    if constexpr (two_level<L>()) {
        constexpr int L1 = MulSplit<L>::L1, L2 = MulSplit<L>::L2;
        constexpr int TB = kTwoThreads / L1;
        constexpr size_t smem = mul2_smem<L1, L2, TS>();
        auto kern = cols_mul2_t<L1, L2, TS, PS>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        dim3 grid((Bz + TB - 1) / TB, 1);
        kern<<<grid, kTwoThreads, smem, st>>>(spec, tspec, prod, Bz, K, tw, lo, hi);
        return cudaGetLastError();
    }
    constexpr int TB = cols_tb<L>();
    const size_t smem = (size_t)2 * L * TB * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(cols_mul_t<L, TS, PS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((Bz + TB - 1) / TB, 1);
    cols_mul_t<L, TS, PS><<<grid, kFftThreads, smem, st>>>(spec, tspec, prod, Bz, K, tw, lo, hi);
    return cudaGetLastError();
}

template <int L, typename PS, typename RT>
cudaError_t run_rows_c2r(const PS* prod, int X, int Y, int Z, FftGeom g, RT* corr, int K,
                         const float2* tw, int* status, FftKeep keep, cudaStream_t st) {
    if constexpr (c2r_half<L>()) {
        constexpr int L1 = RowSplit<L / 2>::L1, L2 = RowSplit<L / 2>::L2;
        constexpr int NR = kTwoThreads / L1 * c2r_groups<L1, L2, PS>();   // rows per tile
        constexpr size_t smem = c2r_half_smem<L1, L2, PS>();
        auto kern = rows_c2r_half_t<L1, L2, PS, RT>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        if (keep.z1 < keep.z0 || keep.y1 < keep.y0 || keep.x1 < keep.x0) return cudaSuccess;
        const size_t nrows = (size_t)K * (keep.z1 - keep.z0 + 1) * (keep.y1 - keep.y0 + 1);
        unsigned grid = 0;
        if ((e = persistent_grid(kern, smem, (nrows + NR - 1) / NR, &grid)) != cudaSuccess) return e;
        if (grid == 0) return cudaSuccess;
        (void)status;                       // no device-side waits in this pass
        kern<<<grid, kTwoThreads, smem, st>>>(prod, X, Y, Z, g, corr, K, tw, keep);
        return cudaGetLastError();
    } else if constexpr (two_level<L>()) {
        constexpr int L1 = TwoLevel<L>::L1, L2 = TwoLevel<L>::L2;
        constexpr int NR = kTwoThreads / L1;
        constexpr size_t smem = two_rows_smem<L1, L2>();
        auto kern = rows_c2r2_t<L1, L2, PS, RT>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        if (keep.z1 < keep.z0 || keep.y1 < keep.y0 || keep.x1 < keep.x0) return cudaSuccess;
        const size_t nrows = (size_t)K * (keep.z1 - keep.z0 + 1) * (keep.y1 - keep.y0 + 1);
        unsigned grid = 0;
        if ((e = persistent_grid(kern, smem, (nrows + NR - 1) / NR, &grid)) != cudaSuccess) return e;
        if (grid == 0) return cudaSuccess;
        (void)status;                       // no device-side waits in this pass
        kern<<<grid, kTwoThreads, smem, st>>>(prod, X, Y, Z, g, corr, K, tw, keep);
        return cudaGetLastError();
    }
    constexpr int NB = rows_nb<L>();
    constexpr size_t smem = c2r_smem<L, PS>();
    cudaError_t e = cudaFuncSetAttribute(rows_c2r_t<L, PS, RT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int sms = 0, per_sm = 0;
    if ((e = sm_count(&sms)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rows_c2r_t<L, PS, RT>,
                                                           kFftThreads, smem)) != cudaSuccess)
        return e;
    if (keep.z1 < keep.z0 || keep.y1 < keep.y0 || keep.x1 < keep.x0) return cudaSuccess;
    const int nty = (keep.y1 - (keep.y0 & ~(NB - 1))) / NB + 1;
    const size_t ntiles = (size_t)K * (keep.z1 - keep.z0 + 1) * nty;
    const size_t cap = (size_t)sms * (per_sm > 0 ? per_sm : 1);
    const unsigned grid = (unsigned)(ntiles < cap ? ntiles : cap);
    if (grid == 0) return cudaSuccess;
    rows_c2r_t<L, PS, RT><<<grid, kFftThreads, smem, st>>>(prod, X, Y, Z, g, corr, K, tw, status,
                                                          keep);
    return cudaGetLastError();
}

}  // namespace fftk

template <int L>
cudaError_t FftLen<L>::rows_r2c(const float* f, int X, int Y, int Z, FftGeom g, float2* spec,
                                const float2* tw, int mode, double* moments,
                                cudaStream_t st) {
    if constexpr (fftk::r2c_half<L>()) {
        constexpr int L1 = fftk::RowSplit<L / 2>::L1, L2 = fftk::RowSplit<L / 2>::L2;
        constexpr int NR = fftk::kTwoThreads / L1;
        constexpr size_t smem = fftk::two_rows_smem<L1, L2>();
        auto kern = fftk::rows_r2c_half_t<L1, L2>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        const size_t nrows = (size_t)g.Yp * g.Zp;
        unsigned grid = 0;
        if ((e = fftk::persistent_grid(kern, smem, (nrows + NR - 1) / NR, &grid)) != cudaSuccess)
            return e;
        if (grid == 0) return cudaSuccess;
        kern<<<grid, fftk::kTwoThreads, smem, st>>>(f, X, Y, Z, g, spec, tw, mode, moments);
        return cudaGetLastError();
    }
    constexpr int NB = fftk::rows_nb<L>();
    const size_t smem = (size_t)2 * L * (NB + 1) * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(fftk::rows_r2c_t<L>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int nrows = g.Yp * g.Zp;
    fftk::rows_r2c_t<L><<<(nrows + NB - 1) / NB, fftk::kFftThreads, smem, st>>>(f, X, Y, Z, g, spec,
                                                                               tw, mode, moments);
    return cudaGetLastError();
}

template <int L>
cudaError_t FftLen<L>::cols(float2* d, int B, int na, ColsMap mp, const float2* tw, int sign,
                            cudaStream_t st) {
    return sign < 0 ? fftk::run_cols<L, -1, float2>(d, B, na, mp, tw, st)
                    : fftk::run_cols<L, +1, float2>(d, B, na, mp, tw, st);
}

template <int L>
cudaError_t FftLen<L>::cols_bf(__nv_bfloat162* d, int B, int na, ColsMap mp, const float2* tw,
                               int sign, cudaStream_t st) {
    // bf16 storage is used by the inverse passes only
    if (sign < 0) return cudaErrorInvalidValue;
    return fftk::run_cols<L, +1, __nv_bfloat162>(d, B, na, mp, tw, st);
}

template <int L>
cudaError_t FftLen<L>::cols_mul(const float2* spec, const float2* tspec, float2* prod, int Bz,
                                int K, const float2* tw, int lo, int hi, cudaStream_t st) {
    return fftk::run_cols_mul<L, float2, float2>(spec, tspec, prod, Bz, K, tw, lo, hi, st);
}

template <int L>
cudaError_t FftLen<L>::cols_mul_bf(const float2* spec, const __nv_bfloat162* tspec,
                                   __nv_bfloat162* prod, int Bz, int K, const float2* tw, int lo,
                                   int hi, cudaStream_t st) {
    return fftk::run_cols_mul<L, __nv_bfloat162, __nv_bfloat162>(spec, tspec, prod, Bz, K, tw, lo,
                                                                 hi, st);
}

template <int L>
cudaError_t FftLen<L>::rows_c2r(const float2* prod, int X, int Y, int Z, FftGeom g, float* corr,
                                int K, const float2* tw, int* status, FftKeep keep,
                                cudaStream_t st) {
    return fftk::run_rows_c2r<L, float2, float>(prod, X, Y, Z, g, corr, K, tw, status, keep, st);
}

template <int L>
cudaError_t FftLen<L>::rows_c2r_bf(const __nv_bfloat162* prod, int X, int Y, int Z, FftGeom g,
                                   __nv_bfloat16* corr, int K, const float2* tw, int* status,
                                   FftKeep keep, cudaStream_t st) {
    return fftk::run_rows_c2r<L, __nv_bfloat162, __nv_bfloat16>(prod, X, Y, Z, g, corr, K, tw,
                                                                 status, keep, st);
}

}  // namespace ttm
