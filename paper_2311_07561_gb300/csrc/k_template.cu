// Tensor template build (Sec. 3.2 of the paper; template normalisation as in
// Algorithm 1 and the formulas for ||P_S t||_S and <t, 1>_S in Sec. 2).
//
//   t~_j = m (t_{R_j} - <t_{R_j}, m>/<1, m>) / sqrt(<t_{R_j}^2, m> - <t_{R_j}, m>^2/<1, m>)
//   T_alpha(u) = sum_j w_j q_j^alpha t~_j(u)
//
// Kernel 1 rotates and normalises a chunk of quadrature nodes, one CTA per
// node (the per-node reductions stay inside the CTA, in FP64).  Kernel 2 folds
// the chunk into the K components: a [K x J] x [J x s^3] product on CUDA cores
// with the coefficients w_j q_j^alpha staged in shared memory.
#include "ttm_internal.h"

namespace ttm {

namespace {

constexpr int kRotThreads = 512;

__device__ __forceinline__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x < 32) {
        r = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
        if (threadIdx.x == 0) red[0] = r;
    }
    __syncthreads();
    return red[0];
}

__global__ void __launch_bounds__(kRotThreads) mask_sum_kernel(const float* __restrict__ m,
                                                               int n, double* out) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += (double)m[i];
    double s = block_sum(acc, red);
    if (threadIdx.x == 0) *out = s;
}

// t_R(u) = t(c + R^-1 (u - c)), trilinear, zero outside the s^3 box.  The
// eight taps are read unconditionally from clamped indices, a tap outside
// the box carrying weight zero (the same sum, term by term, as skipping it),
// so that every load of a voxel can be in flight at once.
__device__ __forceinline__ float sample_rotated(const float* __restrict__ t, int s, float c,
                                                const float Rt[9], int ux, int uy, int uz) {
    float vx = ux - c, vy = uy - c, vz = uz - c;
    // R^-1 = R^T: p_i = sum_k R[k][i] v_k
    float px = Rt[0] * vx + Rt[1] * vy + Rt[2] * vz + c;
    float py = Rt[3] * vx + Rt[4] * vy + Rt[5] * vz + c;
    float pz = Rt[6] * vx + Rt[7] * vy + Rt[8] * vz + c;
    float fx0 = floorf(px), fy0 = floorf(py), fz0 = floorf(pz);
    int x0 = (int)fx0, y0 = (int)fy0, z0 = (int)fz0;
    float ax = px - fx0, ay = py - fy0, az = pz - fz0;
    float tap[8], wt[8];
#pragma unroll
    for (int dz = 0; dz < 2; ++dz) {
        const int zz = z0 + dz;
        const bool iz = zz >= 0 && zz < s;
        const int zc = min(max(zz, 0), s - 1);
        const float wz = dz ? az : 1.0f - az;
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
            const int yy = y0 + dy;
            const bool iy = yy >= 0 && yy < s;
            const int yc = min(max(yy, 0), s - 1);
            const float wy = dy ? ay : 1.0f - ay;
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                const int xx = x0 + dx;
                const bool ix = xx >= 0 && xx < s;
                const int xc = min(max(xx, 0), s - 1);
                const float wx = dx ? ax : 1.0f - ax;
                const int k = (dz * 2 + dy) * 2 + dx;
                tap[k] = __ldg(t + ((size_t)zc * s + yc) * s + xc);
                wt[k] = (iz && iy && ix) ? wz * wy * wx : 0.0f;
            }
        }
    }
    float acc = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) acc += wt[k] * tap[k];
    return acc;
}

__global__ void __launch_bounds__(kRotThreads) rotate_normalise_kernel(
    const float* __restrict__ t, const float* __restrict__ m, int s,
    const float* __restrict__ quats, int j0, float* __restrict__ out, double mask_sum,
    int* bad) {
    __shared__ double red[32];
    __shared__ float Rt[9];
    const int j = j0 + blockIdx.x;
    if (threadIdx.x == 0) {
        float a = quats[4 * j], b = quats[4 * j + 1], cc = quats[4 * j + 2], d = quats[4 * j + 3];
        float inv = rsqrtf(a * a + b * b + cc * cc + d * d);
        a *= inv; b *= inv; cc *= inv; d *= inv;
        // rows of R stored transposed: Rt[3*i + k] = R[k][i]
        float R00 = 1.f - 2.f * (cc * cc + d * d), R01 = 2.f * (b * cc - a * d), R02 = 2.f * (b * d + a * cc);
        float R10 = 2.f * (b * cc + a * d), R11 = 1.f - 2.f * (b * b + d * d), R12 = 2.f * (cc * d - a * b);
        float R20 = 2.f * (b * d - a * cc), R21 = 2.f * (cc * d + a * b), R22 = 1.f - 2.f * (b * b + cc * cc);
        Rt[0] = R00; Rt[1] = R10; Rt[2] = R20;
        Rt[3] = R01; Rt[4] = R11; Rt[5] = R21;
        Rt[6] = R02; Rt[7] = R12; Rt[8] = R22;
    }
    __syncthreads();
    float R[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) R[i] = Rt[i];
    const int s3 = s * s * s;
    const float c = (float)(s / 2);
    float* o = out + (size_t)blockIdx.x * s3;
    double t1 = 0.0, t2 = 0.0;
#pragma unroll 4
    for (int u = threadIdx.x; u < s3; u += blockDim.x) {
        int ux = u % s, uy = (u / s) % s, uz = u / (s * s);
        float v = sample_rotated(t, s, c, R, ux, uy, uz);
        o[u] = v;
        float mm = m[u];
        t1 += (double)(mm * v);
        t2 += (double)(mm * v) * v;
    }
    double T1 = block_sum(t1, red);
    double T2 = block_sum(t2, red);
    double var = T2 - T1 * T1 / mask_sum;
    if (!(var > 0.0)) {
        if (threadIdx.x == 0) atomicOr(bad, 1);
        var = 1.0;
    }
    const float off = (float)(T1 / mask_sum);
    const float scl = (float)(1.0 / sqrt(var));
    for (int u = threadIdx.x; u < s3; u += blockDim.x) o[u] = m[u] * (o[u] - off) * scl;
}

constexpr int kFoldThreads = 256;
constexpr int kFoldJ = 32;        // quadrature nodes staged per step
constexpr int kFoldA = 40;        // components per pass (registers per thread)

// Components A0 .. A0 + kFoldA - 1 (a compile-time range, so the exponent
// table is indexed by constants and stays out of local memory).
template <int N, int A0>
__global__ void __launch_bounds__(kFoldThreads, 2) fold_kernel(
    const float* __restrict__ quats, const float* __restrict__ weights, float inv_nrot, int j0,
    int nj, const float* __restrict__ rot, int s3, float* __restrict__ comp, int first) {
    constexpr Sym<N> S{};
    constexpr int K = n_comp(N);
    constexpr int na = K - A0 < kFoldA ? K - A0 : kFoldA;
    const int a0 = A0;
    __shared__ __align__(16) float coef[kFoldJ][kFoldA];
    static_assert(kFoldA % 4 == 0, "coefficients are read as float4");
    static_assert(kFoldJ <= kFoldThreads, "one thread per staged node");
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    float acc[kFoldA];
#pragma unroll
    for (int a = 0; a < kFoldA; ++a) acc[a] = 0.0f;
    for (int jb = 0; jb < nj; jb += kFoldJ) {
        __syncthreads();
        if (threadIdx.x < kFoldJ) {
            // thread jj: w_j q_j^alpha of its node for the pass's components
            const int jj = threadIdx.x;
            const bool live = jb + jj < nj;
            const int j = j0 + jb + (live ? jj : 0);
            float q[4] = {quats[4 * j], quats[4 * j + 1], quats[4 * j + 2], quats[4 * j + 3]};
            const float inv = rsqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
#pragma unroll
            for (int i = 0; i < 4; ++i) q[i] *= inv;
            const float w = weights ? weights[j] : inv_nrot;
#pragma unroll
            for (int a = 0; a < kFoldA; ++a) {
                float p = 0.0f;
                if (live && a < na) {
                    p = w;
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int r = 0; r < S.e[(A0 + a) % K][i]; ++r) p *= q[i];
                }
                coef[jj][a] = p;
            }
        }
        __syncthreads();
        if (u < s3) {
            const int jn = min(kFoldJ, nj - jb);
            // the block's kFoldJ samples of this voxel, all loads in flight at
            // once (nodes past jn carry zero coefficients)
            float rr[kFoldJ];
#pragma unroll
            for (int jj = 0; jj < kFoldJ; ++jj)
                rr[jj] = jj < jn ? __ldg(rot + (size_t)(jb + jj) * s3 + u) : 0.f;
#pragma unroll
            for (int jj = 0; jj < kFoldJ; ++jj) {
                const float r = rr[jj];
                // one 16-byte broadcast read per four FMAs
                const float4* c4 = reinterpret_cast<const float4*>(&coef[jj][0]);
#pragma unroll
                for (int a4 = 0; a4 < kFoldA / 4; ++a4) {
                    const float4 c = c4[a4];
                    acc[4 * a4 + 0] = fmaf(c.x, r, acc[4 * a4 + 0]);
                    acc[4 * a4 + 1] = fmaf(c.y, r, acc[4 * a4 + 1]);
                    acc[4 * a4 + 2] = fmaf(c.z, r, acc[4 * a4 + 2]);
                    acc[4 * a4 + 3] = fmaf(c.w, r, acc[4 * a4 + 3]);
                }
            }
        }
    }
    if (u < s3) {
        for (int a = 0; a < na; ++a) {
            float* dst = comp + (size_t)(a0 + a) * s3 + u;
            *dst = first ? acc[a] : *dst + acc[a];
        }
    }
}

}  // namespace

ttm_status launch_mask_sum(const float* m, int s, double* d_out, cudaStream_t st, long long* cnt) {
    mask_sum_kernel<<<1, kRotThreads, 0, st>>>(m, s * s * s, d_out);
    return after_launch(cnt);
}

ttm_status launch_rotate_normalise(const float* t, const float* m, int s, const float* quats,
                                   int j0, int nj, float* out, double mask_sum, int* d_bad,
                                   cudaStream_t st, long long* cnt) {
    if (nj <= 0) return TTM_OK;
    rotate_normalise_kernel<<<nj, kRotThreads, 0, st>>>(t, m, s, quats, j0, out, mask_sum, d_bad);
    return after_launch(cnt);
}

// one launch per kFoldA components: A0 = 0, kFoldA, ... below K
template <int N, int A0 = 0>
static ttm_status fold_passes(const float* quats, const float* weights, float inv, int j0, int nj,
                              const float* rot, int s3, float* comp, bool first, dim3 grid,
                              cudaStream_t st, long long* cnt) {
    if constexpr (A0 < n_comp(N)) {
        fold_kernel<N, A0><<<grid, kFoldThreads, 0, st>>>(quats, weights, inv, j0, nj, rot, s3, comp,
                                                         first);
        TTM_TRY(after_launch(cnt));
        return fold_passes<N, A0 + kFoldA>(quats, weights, inv, j0, nj, rot, s3, comp, first, grid,
                                          st, cnt);
    } else {
        return TTM_OK;
    }
}

ttm_status launch_fold_components(int n_order, const float* quats, const float* weights,
                                  int n_rot_total, int j0, int nj, const float* rot, int s3,
                                  float* comp, bool first, cudaStream_t st, long long* cnt) {
    const float inv = 1.0f / (float)n_rot_total;
    const dim3 grid((s3 + kFoldThreads - 1) / kFoldThreads);
    switch (n_order) {
        case 2: return fold_passes<2>(quats, weights, inv, j0, nj, rot, s3, comp, first, grid, st, cnt);
        case 4: return fold_passes<4>(quats, weights, inv, j0, nj, rot, s3, comp, first, grid, st, cnt);
        case 6: return fold_passes<6>(quats, weights, inv, j0, nj, rot, s3, comp, first, grid, st, cnt);
        case 8: return fold_passes<8>(quats, weights, inv, j0, nj, rot, s3, comp, first, grid, st, cnt);
        default: return TTM_ERR_UNSUPPORTED;
    }
}

}  // namespace ttm
