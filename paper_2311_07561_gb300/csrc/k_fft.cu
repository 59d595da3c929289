// Batched 3D FFTs for the correlation with the K tensor components (Sec. 2 of
// the paper: <f, g> = F^-1(F f . conj F g)(0); Algorithm 1 uses it for every
// rotation, TTM for every component, Sec. 3.2).
//
// Layouts.  A real volume is [Zp][Yp][Xp] (padded sizes, zero beyond the
// data); its half spectrum is [Zp][Yp][Xh] complex64 with Xh = Xp/2 + 1.
//
// The passes for the lengths of TTM_FFT_LENGTHS have their line length fixed
// at compile time (k_fft.cuh, instantiated in k_fft_len*.cu).  Other powers of
// two up to 4096 take the runtime-length kernels below (radix 4 and 2, same
// tiling, FP32 storage only).
#include <cmath>
#include <type_traits>

#include "k_fft.cuh"

namespace ttm {

#define TTM_FFT_EXTERN(L) extern template struct FftLen<L>;
TTM_FFT_LENGTHS(TTM_FFT_EXTERN)
#undef TTM_FFT_EXTERN

namespace {

using fftk::cmul;
using fftk::cmulc;
using fftk::cadd;
using fftk::csub;
using fftk::kFftThreads;
constexpr int kTileElems = 4096;   // complex elements per shared-memory buffer

struct Radices {
    int n;          // number of stages
    int r[16];      // radix of each stage (4 or 2), in order
};

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

// ---- dispatch to the compile-time lengths (false: length not listed) ----
#define TTM_FFT_CASE(L, CALL) case L: *err = FftLen<L>::CALL; return true;

bool fixed_rows_r2c(int L, const float* f, int X, int Y, int Z, FftGeom g, float2* spec,
                    const float2* tw, int mode, double* moments, cudaStream_t st,
                    cudaError_t* err) {
    switch (L) {
#define C(L) TTM_FFT_CASE(L, rows_r2c(f, X, Y, Z, g, spec, tw, mode, moments, st))
        TTM_FFT_LENGTHS(C)
#undef C
        default: return false;
    }
}

bool fixed_cols(int L, float2* d, int B, int na, ColsMap mp, const float2* tw, int sign,
                cudaStream_t st, cudaError_t* err) {
    switch (L) {
#define C(L) TTM_FFT_CASE(L, cols(d, B, na, mp, tw, sign, st))
        TTM_FFT_LENGTHS(C)
#undef C
        default: return false;
    }
}

bool fixed_cols(int L, __nv_bfloat162* d, int B, int na, ColsMap mp, const float2* tw, int sign,
                cudaStream_t st, cudaError_t* err) {
    switch (L) {
#define C(L) TTM_FFT_CASE(L, cols_bf(d, B, na, mp, tw, sign, st))
        TTM_FFT_LENGTHS(C)
#undef C
        default: return false;
    }
}

bool fixed_cols_mul(int L, const float2* spec, const float2* tspec, float2* prod, int Bz, int K,
                    const float2* tw, int lo, int hi, cudaStream_t st, cudaError_t* err) {
    switch (L) {
#define C(L) TTM_FFT_CASE(L, cols_mul(spec, tspec, prod, Bz, K, tw, lo, hi, st))
        TTM_FFT_LENGTHS(C)
#undef C
        default: return false;
    }
}

bool fixed_cols_mul(int L, const float2* spec, const __nv_bfloat162* tspec, __nv_bfloat162* prod,
                    int Bz, int K, const float2* tw, int lo, int hi, cudaStream_t st,
                    cudaError_t* err) {
    switch (L) {
#define C(L) TTM_FFT_CASE(L, cols_mul_bf(spec, tspec, prod, Bz, K, tw, lo, hi, st))
        TTM_FFT_LENGTHS(C)
#undef C
        default: return false;
    }
}

bool fixed_rows_c2r(int L, const float2* prod, int X, int Y, int Z, FftGeom g, float* corr, int K,
                    const float2* tw, int* status, FftKeep keep, cudaStream_t st,
                    cudaError_t* err) {
    switch (L) {
#define C(L) TTM_FFT_CASE(L, rows_c2r(prod, X, Y, Z, g, corr, K, tw, status, keep, st))
        TTM_FFT_LENGTHS(C)
#undef C
        default: return false;
    }
}

bool fixed_rows_c2r(int L, const __nv_bfloat162* prod, int X, int Y, int Z, FftGeom g,
                    __nv_bfloat16* corr, int K, const float2* tw, int* status, FftKeep keep,
                    cudaStream_t st, cudaError_t* err) {
    switch (L) {
#define C(L) TTM_FFT_CASE(L, rows_c2r_bf(prod, X, Y, Z, g, corr, K, tw, status, keep, st))
        TTM_FFT_LENGTHS(C)
#undef C
        default: return false;
    }
}
#undef TTM_FFT_CASE

}  // namespace


// Column lines (length L, element stride B): planes z0 .. z0 + nz - 1 of each
// of n_items items (items zstride planes apart), storing line samples lo..hi.
template <typename PS>
static ttm_status launch_cols_t(PS* data, int L, int B, int n_items, int zstride, int z0, int nz,
                                int lo, int hi, const float2* tw, int sign, cudaStream_t st,
                                long long* cnt) {
    if (n_items <= 0 || nz <= 0) return TTM_OK;
    cudaError_t err = cudaSuccess;
    const ColsMap mp{0, nz, zstride, z0, lo, hi};
    if (fixed_cols(L, data, B, n_items * nz, mp, tw, sign, st, &err)) {
        TTM_CUDA_TRY(err);
        return after_launch(cnt);
    }
    if constexpr (!std::is_same<PS, float2>::value) {
        return TTM_ERR_UNSUPPORTED;
    } else {
        // runtime-length kernel: every sample of the selected planes is stored
        const int TB = cols_per_cta(L);
        const size_t smem = (size_t)2 * L * TB * sizeof(float2);
        TTM_CUDA_TRY(cudaFuncSetAttribute(cols_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        for (int item = 0; item < n_items; ++item) {
            for (int a0 = 0; a0 < nz; a0 += 65535) {
                const int na = nz - a0 < 65535 ? nz - a0 : 65535;
                PS* d = data + ((size_t)item * zstride + z0 + a0) * L * B;
                dim3 grid((B + TB - 1) / TB, na);
                cols_kernel<<<grid, kFftThreads, smem, st>>>(d, L, B, radices_for(L), tw, TB, sign);
                TTM_TRY(after_launch(cnt));
            }
        }
        return TTM_OK;
    }
}

static ttm_status launch_cols(float2* data, int L, int B, int batch, const float2* tw, int sign,
                              cudaStream_t st, long long* cnt) {
    return launch_cols_t<float2>(data, L, B, 1, batch, 0, batch, 0, L - 1, tw, sign, st, cnt);
}

// lengths with a compile-time pass (TTM_FFT_LENGTHS)
bool fft_template_length(int L) {
    switch (L) {
#define C(L) case L:
        TTM_FFT_LENGTHS(C)
#undef C
        return true;
        default: return false;
    }
}

// compile-time lengths, or powers of two up to 4096 (runtime-length kernels)
bool fft_length_ok(int L) {
    return fft_template_length(L) || (L >= 2 && L <= 4096 && (L & (L - 1)) == 0);
}

// smallest compile-time length >= n (2^p 3^a 5^b), else the next power of two
int fft_good_length(int n) {
    static const int lengths[] = {
#define C(L) L,
        TTM_FFT_LENGTHS(C)
#undef C
    };
    for (int L : lengths)
        if (L >= n) return L;
    int L = 2;
    while (L < n) L <<= 1;
    return L;
}

ttm_status launch_fft_forward(const float* f, int X, int Y, int Z, const FftShape& S,
                              float2* spec, cudaStream_t st, long long* cnt, int mode,
                              double* moments) {
    FftGeom g{S.Xp, S.Yp, S.Zp, S.Xp / 2 + 1};
    cudaError_t err = cudaSuccess;
    {
        if (mode != 0 && !fft_template_length(S.Xp)) return TTM_ERR_UNSUPPORTED;
        if (!fixed_rows_r2c(S.Xp, f, X, Y, Z, g, spec, S.d_tw_x, mode, moments, st, &err)) {
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
                                       PS* prod, const FftKeep& keep, cudaStream_t st,
                                       long long* cnt) {
    const int Xh = S.Xp / 2 + 1;
    const int Bz = S.Yp * Xh;
    cudaError_t err = cudaSuccess;
    if (!fixed_cols_mul(S.Zp, spec, tspec, prod, Bz, K, S.d_tw_z, keep.z0, keep.z1, st, &err)) {
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
                               int* status, const FftKeep& keep, cudaStream_t st, long long* cnt) {
    FftGeom g{S.Xp, S.Yp, S.Zp, S.Xp / 2 + 1};
    // y lines of the kept z planes; the kept rows y are the ones stored
    TTM_TRY(launch_cols_t<PS>(prod, S.Yp, g.Xh, K, S.Zp, keep.z0, keep.z1 - keep.z0 + 1, keep.y0,
                              keep.y1, S.d_tw_y, +1, st, cnt));
    cudaError_t err = cudaSuccess;
    if (!fixed_rows_c2r(S.Xp, prod, X, Y, Z, g, corr, K, S.d_tw_x, status, keep, st, &err)) {
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
                                         const FftShape& S, float2* prod, const FftKeep& keep,
                                         cudaStream_t st, long long* cnt) {
    return spectrum_inverse_z_t<float2, float2>(spec, tspec, K, S, prod, keep, st, cnt);
}

ttm_status launch_fft_inverse_yx(float2* prod, int K, int X, int Y, int Z, const FftShape& S,
                                 float* corr, int* status, const FftKeep& keep, cudaStream_t st,
                                 long long* cnt) {
    return inverse_yx_t<float2, float>(prod, K, X, Y, Z, S, corr, status, keep, st, cnt);
}

// mixed precision: bf16 template spectra, products and correlation maps
ttm_status launch_fft_spectrum_inverse_z_bf16(const float2* spec, const void* tspec, int K,
                                              const FftShape& S, void* prod, const FftKeep& keep,
                                              cudaStream_t st, long long* cnt) {
    return spectrum_inverse_z_t<__nv_bfloat162, __nv_bfloat162>(
        spec, reinterpret_cast<const __nv_bfloat162*>(tspec), K, S,
        reinterpret_cast<__nv_bfloat162*>(prod), keep, st, cnt);
}

ttm_status launch_fft_inverse_yx_bf16(void* prod, int K, int X, int Y, int Z, const FftShape& S,
                                      void* corr, int* status, const FftKeep& keep,
                                      cudaStream_t st, long long* cnt) {
    return inverse_yx_t<__nv_bfloat162, __nv_bfloat16>(
        reinterpret_cast<__nv_bfloat162*>(prod), K, X, Y, Z, S,
        reinterpret_cast<__nv_bfloat16*>(corr), status, keep, st, cnt);
}

__global__ void to_bf16_kernel(const float2* __restrict__ a, __nv_bfloat162* __restrict__ b, size_t n) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = __float22bfloat162_rn(a[i]);
}

ttm_status launch_spectra_to_bf16(const float2* a, void* b, size_t n, cudaStream_t st, long long* cnt) {
    to_bf16_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, reinterpret_cast<__nv_bfloat162*>(b), n);
    return after_launch(cnt);
}


// w from the FFT-based window sums of (f - mean) and (f - mean)^2 (Algorithm 1):
// V = S2 - S1^2 / m_sum; interior only; floor 1e-6 m_sum var(f).
//
// The FP32 FFT window sums carry a rounding error set by the whole volume,
// not by the window: |dS| <= kappa eps m_sum rms(a) for a = f - mean (S1) and
// a = (f - mean)^2 (S2), eps = 2^-24, kappa = 2 log2(N) (measured worst cases
// stay near log2(N)).  A window whose bound on |dV| exceeds 2e-5 V (the 1e-5
// tolerance of w), or which lies within the bound of the floor, is flagged
// (w = -1, counted in *flagged) and recomputed exactly by direct FP64 sums
// (launch_exact_stats).  Large offsets never flag (the mean is removed); a
// quiet window in a volume of large dynamic range does.
// Persistent CTAs over x-segments of 128 voxels: the volume statistics and
// the bounds (FP64 divisions, slow on this GPU) are formed once per CTA; per
// voxel V and its bound are FP32 (a window that needs more than that is
// flagged and recomputed in FP64).
__global__ void __launch_bounds__(128) stats_from_sums_kernel(
    const float* __restrict__ s1, const float* __restrict__ s2, float* __restrict__ w, int X,
    int Y, int Z, int s, double mask_sum, const double* __restrict__ moments, double kappa,
    unsigned int* __restrict__ flagged) {
    __shared__ double sh[4];
    if (threadIdx.x == 0) {
        const double nv = (double)X * Y * Z;
        const double mean = moments[0] / nv;
        const double var_f = fmax(moments[1] / nv - mean * mean, 0.0);
        const double eps = 5.9604644775390625e-8;          // 2^-24
        sh[0] = 1.0 / mask_sum;
        sh[1] = 1e-6 * mask_sum * var_f;
        sh[2] = kappa * eps * mask_sum * sqrt(var_f);       // bound on |dS1|
        sh[3] = kappa * eps * mask_sum * sqrt(fmax(moments[2], 0.0) / nv);   // on |dS2|
    }
    __syncthreads();
    const float fim = (float)sh[0], ffl = (float)sh[1], fe1 = (float)sh[2], fe2 = (float)sh[3];
    const uint32_t xt = (uint32_t)((X + 127) / 128);
    const uint32_t segs = xt * (uint32_t)Y * (uint32_t)Z;
    unsigned int nflag = 0;
    for (uint32_t sg = blockIdx.x; sg < segs; sg += gridDim.x) {
        const uint32_t row = sg / xt;
        const int x = (int)(sg - row * xt) * 128 + threadIdx.x;
        const int y = (int)(row % (uint32_t)Y), z = (int)(row / (uint32_t)Y);
        if (x >= X) continue;
        const size_t v = ((size_t)z * Y + y) * X + x;
        float out = 0.f;
        if (interior(x, X, s) && interior(y, Y, s) && interior(z, Z, s)) {
            // V in FP32; its own rounding (eps (S2 + S1^2/m)) joins the bound
            const float S1 = s1[v], S2 = s2[v];
            const float q = S1 * S1 * fim;
            const float V = S2 - q;
            const float dv = fe2 + (2.f * fabsf(S1) * fe1 + fe1 * fe1) * fim +
                             1.2e-7f * (fabsf(S2) + q);
            if (dv > 2e-5f * V || fabsf(V - ffl) <= dv) {
                out = -1.f;
                ++nflag;
            } else if (V > ffl) {
                out = rsqrtf(V);
            }
        }
        w[v] = out;
    }
    for (int o = 16; o > 0; o >>= 1) nflag += __shfl_down_sync(0xffffffffu, nflag, o);
    if ((threadIdx.x & 31) == 0 && nflag) atomicAdd(flagged, nflag);
}

ttm_status launch_stats_from_sums(const float* s1, const float* s2, float* w, int X, int Y, int Z,
                                  int s, double mask_sum, const double* moments,
                                  unsigned int* flagged, cudaStream_t st, long long* cnt) {
    const size_t segs = (size_t)((X + 127) / 128) * Y * Z;
    if (segs > 0xFFFFFFFFull) return TTM_ERR_UNSUPPORTED;
    const unsigned grid = (unsigned)(segs < 152 * 16 ? segs : 152 * 16);
    const double kappa = 2.0 * std::log2((double)X * Y * Z);
    stats_from_sums_kernel<<<grid, 128, 0, st>>>(s1, s2, w, X, Y, Z, s, mask_sum, moments, kappa,
                                                 flagged);
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