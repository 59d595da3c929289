// Per-voxel TTM score and rotation (kernel template; instantiated per order n
// in k_rotation_n*.cu) (Sec. 3.2-3.4 of the paper).
//
//   C_alpha(x) = w(x) Corr_alpha(x)
//   score(x)   = ||C_n(x)||_F = sqrt(sum_alpha mu_alpha C_alpha^2)          (Sec. 3.4)
//   lambda(x)  = max_{|Q|=1} phi(Q),  phi(Q) = C_n(x) . Q^(n)                (Sec. 3.3)
//   q(x)       = argmax, the dominant Z-eigenvector of C_n(x)                (Sec. 3.1)
//
// One thread per interior voxel.  The maximum is searched on a fixed grid of unit
// quaternions (half sphere, sorted into regions of equal size): phi at every grid point is a
// dot product with a precomputed row mu_alpha q_g^alpha staged in shared memory
// and read as a broadcast.  The best point of each region competes for a short
// list of n_cand candidates.  Every candidate takes two shifted power steps
// (x <- normalise(C x^{n-1} + sigma x), sigma = (n-1) score, the SS-HOPM step
// of Kolda & Mayo 2011, monotone for this shift); the n_refine (<= kRefine)
// best of the points reached are then refined by Riemannian Newton steps on the sphere,
// each accepted only if phi does not decrease (otherwise the power step is
// taken).  The largest refined value wins.
#pragma once
#include <cuda_bf16.h>

#include "ttm_internal.h"

namespace ttm {

namespace rot {

constexpr int kRotThreads = 128;
constexpr int kChunk = 128;       // grid points staged per step
constexpr int kMaxCand = 8;
constexpr int kRefine = 4;        // candidates refined by Newton after the power steps

// correlation maps are float or bf16 (mixed precision)
__device__ __forceinline__ float ldcorr(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ldcorr(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }

// The problems and units of one launch (RotBatch, in the kernel parameters,
// read in place: the kernels take their arguments as __grid_constant__).
struct SearchArgs {
    RotBatch b;
    UnitList list;          // optional unit list (peaks; one problem per launch)
    const float* gm;        // n_grid x K4 (SIMT search)
    const int* cell_end;    // n_grid
    int n_grid;
};

struct PolishArgs {
    RotBatch b;
    UnitList list;          // optional unit list (peaks) and strided outputs
    const float* gq;        // n_grid x 4
    int n_cand, newton, n_refine;
};

static_assert(kRotThreads == kRotTile, "one block of the SIMT kernels is one tile");

// segment of tile t: segments are in tile order, so s only moves forward
static __device__ __forceinline__ int seg_of(const RotBatch& b, uint32_t t, int s = 0) {
    while (s + 1 < b.n && t >= b.seg[s + 1].tile0) ++s;
    return s;
}

// The score sum_alpha mu_alpha C_alpha^2 is accumulated in two halves, the
// components below score_split<N>() and the rest, added at the end: the
// tensor-core search loads the two halves of a voxel's components in two
// threads, and every kernel that writes a score map sums in this same order,
// so the maps agree bit for bit.
template <int N>
__host__ __device__ constexpr int score_split() { return ((n_comp(N) + 1 + 15) / 16) * 8; }

// end of the units [.., u1) and the voxel of unit i, with an optional list
static __device__ __forceinline__ uint32_t list_end(const UnitList& l, uint32_t u1) {
    if (!l.count) return u1;
    const int c = *l.count;
    return c <= 0 ? 0u : ((uint32_t)c < u1 ? (uint32_t)c : u1);
}
static __device__ __forceinline__ size_t unit_voxel(const VoxBox& b, const UnitList& l, uint32_t i) {
    return l.idx ? (size_t)l.idx[(size_t)i * l.stride] : b.voxel(i);
}

// score = ||C||_F with C = w Corr at the interior voxels, 0 elsewhere; the
// same arithmetic as the search kernels.  Block (x segment, y, z).
template <int N, typename CT>
__global__ void __launch_bounds__(128) score_only_kernel(const CT* __restrict__ corr,
                                                         const float* __restrict__ w, int X, int Y,
                                                         size_t nvox, VoxBox box,
                                                         float* __restrict__ score) {
    constexpr int K = n_comp(N);
    constexpr Sym<N> S{};
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= X) return;
    const size_t v = ((size_t)z * Y + y) * X + x;
    const bool in = (uint32_t)(x - box.x0) < box.nx && (uint32_t)(y - box.y0) < box.ny &&
                    (uint32_t)(z - box.z0) < box.nz;
    float ss0 = 0.f, ss1 = 0.f;
    if (in) {
        const float wv = __ldg(w + v);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const float c = wv * ldcorr(corr + (size_t)k * nvox + v);
            if (k < score_split<N>()) ss0 = fmaf((float)S.mu[k], c * c, ss0);
            else ss1 = fmaf((float)S.mu[k], c * c, ss1);
        }
    }
    score[v] = sqrtf(ss0 + ss1);
}

// keep the kMaxCand largest (value, index) pairs, sorted descending
static __device__ __forceinline__ void insert_candidate(float (&tv)[kMaxCand], int (&ti)[kMaxCand],
                                                 float val, int idx) {
#pragma unroll
    for (int k = 0; k < kMaxCand; ++k) {
        if (val > tv[k]) {
            float t = tv[k]; tv[k] = val; val = t;
            int u = ti[k]; ti[k] = idx; idx = u;
        }
    }
}

static __device__ __forceinline__ void store_candidates(uint16_t* cand, size_t v, const int (&ti)[kMaxCand],
                                                 bool active) {
    uint32_t w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        uint32_t lo = active ? (uint32_t)(ti[2 * k] & 0xFFFF) : 0xFFFFu;
        uint32_t hi = active ? (uint32_t)(ti[2 * k + 1] & 0xFFFF) : 0xFFFFu;
        w[k] = lo | (hi << 16);
    }
    reinterpret_cast<uint4*>(cand)[v] = make_uint4(w[0], w[1], w[2], w[3]);
}

template <int N>
struct Geo {
    static constexpr int K = n_comp(N);
    static constexpr int K4 = (K + 3) & ~3;
};

// H = C x^{N-2} (symmetric 4x4, 10 entries in the order of HessTab pairs)
template <int N>
__device__ __forceinline__ void hess(const float (&C)[Geo<N>::K4], const float x[4], float h[10]) {
    constexpr HessTab<N> T{};
    Monomials<N - 2> mb;
    monomials<N - 2>(x, mb);
    float mw[HessTab<N>::KB];
#pragma unroll
    for (int b = 0; b < HessTab<N>::KB; ++b) mw[b] = (float)T.mult[b] * mb.v[b];
#pragma unroll
    for (int p = 0; p < 10; ++p) {
        float acc = 0.f;
#pragma unroll
        for (int b = 0; b < HessTab<N>::KB; ++b) acc = fmaf(mw[b], C[T.comp[p][b]], acc);
        h[p] = acc;
    }
}

// full 4x4 from the 10 stored entries (pairs i <= j in row order)
static __device__ __forceinline__ void unpack(const float h[10], float H[4][4]) {
    int p = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = i; j < 4; ++j) {
            H[i][j] = h[p];
            H[j][i] = h[p];
            ++p;
        }
}

static __device__ __forceinline__ void normalise4(float x[4]) {
    float n2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2] + x[3] * x[3];
    float inv = rsqrtf(n2);
#pragma unroll
    for (int i = 0; i < 4; ++i) x[i] *= inv;
}

// value and gradient pieces at x: H = C x^{N-2}, g = H x = C x^{N-1}, lam = x.g
template <int N>
__device__ __forceinline__ void eval_at(const float (&C)[Geo<N>::K4], const float x[4],
                                        float H[4][4], float g[4], float& lam) {
    float h[10];
    hess<N>(C, x, h);
    unpack(h, H);
#pragma unroll
    for (int i = 0; i < 4; ++i)
        g[i] = H[i][0] * x[0] + H[i][1] * x[1] + H[i][2] * x[2] + H[i][3] * x[3];
    lam = g[0] * x[0] + g[1] * x[1] + g[2] * x[2] + g[3] * x[3];
}

// Riemannian Newton direction on the unit sphere for maximising phi:
//   P ((N-1) H - lam I) P eta = -(g - lam x),  eta orthogonal to x,
// solved as A eta = (g - lam x) with A = -P B P + sig x x^T, which is SPD
// exactly when the tangent Hessian is negative definite.  Returns false if
// the Cholesky factorisation breaks down (not near a maximum).  Pivots are
// inverted with rsqrt, so the solve has no division.
template <int N>
__device__ __forceinline__ bool newton_dir(const float H[4][4], const float g[4], const float x[4],
                                           float lam, float sig, float eta[4]) {
    float B[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) B[i][j] = (float)(N - 1) * H[i][j] - (i == j ? lam : 0.f);
    float Bx[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) Bx[i] = B[i][0] * x[0] + B[i][1] * x[1] + B[i][2] * x[2] + B[i][3] * x[3];
    const float xBx = x[0] * Bx[0] + x[1] * Bx[1] + x[2] * Bx[2] + x[3] * Bx[3];
    // A = -B + x (Bx)^T + (Bx) x^T + (sig - x^T B x) x x^T, lower triangle only
    const float cxx = sig - xBx;
    float A[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j)
            A[i][j] = fmaf(cxx * x[i], x[j], fmaf(x[i], Bx[j], fmaf(Bx[i], x[j], -B[i][j])));
    float r[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) r[i] = g[i] - lam * x[i];
    const float tiny = 1e-9f * sig;
    float L[4][4] = {};
    float inv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float d = A[j][j];
#pragma unroll
        for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
        if (!(d > tiny)) return false;
        inv[j] = rsqrtf(d);
#pragma unroll
        for (int i = j + 1; i < 4; ++i) {
            float v = A[i][j];
#pragma unroll
            for (int k = 0; k < j; ++k) v -= L[i][k] * L[j][k];
            L[i][j] = v * inv[j];
        }
    }
    float y[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float v = r[i];
#pragma unroll
        for (int k = 0; k < i; ++k) v -= L[i][k] * y[k];
        y[i] = v * inv[i];
    }
#pragma unroll
    for (int i = 3; i >= 0; --i) {
        float v = y[i];
#pragma unroll
        for (int k = i + 1; k < 4; ++k) v -= L[k][i] * eta[k];
        eta[i] = v * inv[i];
    }
    return true;
}

// g = C x^{N-1} (the gradient of phi divided by N) and lam = x . g
template <int N>
__device__ __forceinline__ void grad_at(const float (&C)[Geo<N>::K4], const float x[4], float g[4],
                                        float& lam) {
    constexpr GradTab<N> T{};
    Monomials<N - 1> mg;
    monomials<N - 1>(x, mg);
    float mw[GradTab<N>::KG];
#pragma unroll
    for (int b = 0; b < GradTab<N>::KG; ++b) mw[b] = (float)T.mult[b] * mg.v[b];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float acc = 0.f;
#pragma unroll
        for (int b = 0; b < GradTab<N>::KG; ++b) acc = fmaf(mw[b], C[T.comp[i][b]], acc);
        g[i] = acc;
    }
    lam = g[0] * x[0] + g[1] * x[1] + g[2] * x[2] + g[3] * x[3];
}

// Two shifted power (SS-HOPM) steps x <- normalise(C x^{N-1} + sigma x) from
// x (the SS-HOPM step of Kolda & Mayo 2011, monotone for this shift); with
// want_lam, lam = phi at the point reached (one more evaluation).
template <int N>
__device__ __forceinline__ void power_steps(const float (&C)[Geo<N>::K4], float sigma, float x[4],
                                            float& lam, bool want_lam) {
    float g[4];
#pragma unroll 1
    for (int s = 0; s < 2; ++s) {
        grad_at<N>(C, x, g, lam);
#pragma unroll
        for (int i = 0; i < 4; ++i) x[i] = g[i] + sigma * x[i];
        normalise4(x);
    }
    if (want_lam) grad_at<N>(C, x, g, lam);
}

// Riemannian Newton steps on the sphere from x; a trial that lowers phi is
// rejected and replaced by a power step from the last accepted point (power
// steps with this shift never lower phi).  newton trials are evaluated; no
// direction is formed after the last one.  One evaluation site per iteration
// keeps the code small.
template <int N>
__device__ void refine(const float (&C)[Geo<N>::K4], float sigma, int newton, float x[4],
                       float& lam_out) {
    float xa[4] = {x[0], x[1], x[2], x[3]};
    float ga[4], la = -INFINITY;
    float xt[4] = {x[0], x[1], x[2], x[3]};
    bool trial_newton = false;
    const float eps = 1e-6f * sigma;
    const int iters = 1 + newton;
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
        float H[4][4], g[4], lam;
        const bool last = it + 1 == iters;
        // the last trial needs only phi: from order 6 on C x^(n-1) (4 sums)
        // is cheaper than C x^(n-2) (10 sums)
        if (N >= 6 && last && it > 0) grad_at<N>(C, xt, g, lam);
        else eval_at<N>(C, xt, H, g, lam);
        if (trial_newton && lam < la - eps) {
            if (last) break;
#pragma unroll
            for (int i = 0; i < 4; ++i) xt[i] = ga[i] + sigma * xa[i];
            normalise4(xt);
            trial_newton = false;
            continue;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            xa[i] = xt[i];
            ga[i] = g[i];
        }
        la = lam;
        if (last) break;
        float eta[4];
        if (newton_dir<N>(H, ga, xa, la, sigma, eta)) {
            const float en2 = eta[0] * eta[0] + eta[1] * eta[1] + eta[2] * eta[2] + eta[3] * eta[3];
            const float clip = en2 > 0.0625f ? 0.25f * rsqrtf(en2) : 1.f;
#pragma unroll
            for (int i = 0; i < 4; ++i) xt[i] = xa[i] + clip * eta[i];
            trial_newton = true;
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) xt[i] = ga[i] + sigma * xa[i];
            trial_newton = false;
        }
        normalise4(xt);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) x[i] = xa[i];
    lam_out = la;
}

// Score and search: C_alpha = w Corr_alpha, score = ||C||_F, phi at every grid
// point, best point of each region, the n_cand best regions -> candidate grid
// indices (0xFFFF = none).  One thread per voxel; the grid table is staged in
// shared memory and read as broadcasts.
template <int N, typename CT>
__global__ void __launch_bounds__(kRotThreads) search_simt_kernel(const __grid_constant__ SearchArgs a) {
    constexpr int K = Geo<N>::K;
    constexpr int K4 = Geo<N>::K4;
    constexpr Sym<N> S{};
    extern __shared__ __align__(16) float sm[];
    float* Mt = sm;                                   // kChunk x K4
    int* ends = reinterpret_cast<int*>(sm + kChunk * K4);

    const RotSeg& sg = a.b.seg[seg_of(a.b, blockIdx.x)];
    const CT* corr = reinterpret_cast<const CT*>(sg.corr);
    const size_t i = sg.u0 + (size_t)(blockIdx.x - sg.tile0) * kRotTile + threadIdx.x;
    const bool in_range = i < list_end(a.list, sg.u1);
    const size_t v = in_range ? unit_voxel(sg.box, a.list, (uint32_t)i) : 0;
    const float wv = in_range ? __ldg(sg.w + v) : 0.f;
    float C[K4];
#pragma unroll
    for (int k = 0; k < K4; ++k) C[k] = 0.f;
    float ss0 = 0.f, ss1 = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float c = in_range ? wv * ldcorr(corr + (size_t)k * sg.nvox + v) : 0.f;
        C[k] = c;
        if (k < score_split<N>()) ss0 = fmaf((float)S.mu[k], c * c, ss0);
        else ss1 = fmaf((float)S.mu[k], c * c, ss1);
    }
    const float score = sqrtf(ss0 + ss1);
    const bool active = in_range && score > 0.f;

    float tv[kMaxCand];
    int ti[kMaxCand];
#pragma unroll
    for (int k = 0; k < kMaxCand; ++k) { tv[k] = -INFINITY; ti[k] = 0xFFFF; }
    float cur = -INFINITY;
    int curi = 0;
    const bool any_active = __syncthreads_or(active);
    for (int g0 = 0; g0 < a.n_grid && any_active; g0 += kChunk) {
        const int gn = min(kChunk, a.n_grid - g0);
        __syncthreads();
        const float4* src = reinterpret_cast<const float4*>(a.gm + (size_t)g0 * K4);
        float4* dst = reinterpret_cast<float4*>(Mt);
        for (int e = threadIdx.x; e < gn * (K4 / 4); e += blockDim.x) dst[e] = __ldg(src + e);
        for (int e = threadIdx.x; e < gn; e += blockDim.x) ends[e] = __ldg(a.cell_end + g0 + e);
        __syncthreads();
        for (int gg = 0; gg < gn; ++gg) {
            const float4* row = reinterpret_cast<const float4*>(Mt + gg * K4);
            float phi = 0.f;
#pragma unroll
            for (int c4 = 0; c4 < K4 / 4; ++c4) {
                const float4 m = row[c4];
                phi = fmaf(m.x, C[4 * c4 + 0], phi);
                phi = fmaf(m.y, C[4 * c4 + 1], phi);
                phi = fmaf(m.z, C[4 * c4 + 2], phi);
                phi = fmaf(m.w, C[4 * c4 + 3], phi);
            }
            if (phi > cur) { cur = phi; curi = g0 + gg; }
            if (ends[gg]) {
                insert_candidate(tv, ti, cur, curi);
                cur = -INFINITY;
            }
        }
    }
    if (!in_range) return;
    sg.score[v] = score;
    store_candidates(sg.cand, i, ti, active);
}

// Refinement of the candidates and the outputs: lambda = the largest refined
// phi, q its maximiser (canonical sign), C_alpha optionally.
template <int N, typename CT>
__global__ void __launch_bounds__(kRotThreads) polish_kernel(const __grid_constant__ PolishArgs a) {
    constexpr int K = Geo<N>::K;
    constexpr int K4 = Geo<N>::K4;
    const RotSeg& sg = a.b.seg[seg_of(a.b, blockIdx.x)];
    const CT* corr = reinterpret_cast<const CT*>(sg.corr);
    const size_t i = sg.u0 + (size_t)(blockIdx.x - sg.tile0) * kRotTile + threadIdx.x;
    if (i >= list_end(a.list, sg.u1)) return;
    const size_t v = unit_voxel(sg.box, a.list, (uint32_t)i);
    const float wv = __ldg(sg.w + v);
    float C[K4];
#pragma unroll
    for (int k = 0; k < K4; ++k) C[k] = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float c = wv * ldcorr(corr + (size_t)k * sg.nvox + v);
        C[k] = c;
        if (sg.comp_out) sg.comp_out[(size_t)k * sg.nvox + v] = c;
    }
    const float score = __ldg(sg.score + v);
    const uint4 cr = __ldg(reinterpret_cast<const uint4*>(sg.cand) + i);
    const uint32_t cw[4] = {cr.x, cr.y, cr.z, cr.w};
    float best_l = 0.f;
    float best_q[4] = {1.f, 0.f, 0.f, 0.f};
    if (score > 0.f && (cw[0] & 0xFFFFu) != 0xFFFFu) {
        const float sigma = (float)(N - 1) * score;
        best_l = -INFINITY;
        // phase 1: two power steps from every candidate; the kRefine best
        // (by phi at the point reached) are kept, sorted descending.  When
        // every candidate is refined the ranking only orders the refinement:
        // the candidates keep the search's order and phi is not evaluated
        const bool rank = a.n_cand > a.n_refine;
        float kl[kRefine], kx[kRefine][4];
#pragma unroll
        for (int s = 0; s < kRefine; ++s) {
            kl[s] = -INFINITY;
#pragma unroll
            for (int i = 0; i < 4; ++i) kx[s][i] = 0.f;
        }
#pragma unroll 1
        for (int k = 0; k < a.n_cand && k < kMaxCand; ++k) {
            const int gi = (int)((cw[k >> 1] >> (16 * (k & 1))) & 0xFFFFu);
            if (gi == 0xFFFF) break;
            float x[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) x[i] = __ldg(a.gq + 4 * gi + i);
            float l;
            power_steps<N>(C, sigma, x, l, rank);
            if (!rank) l = -(float)k;
#pragma unroll
            for (int s = 0; s < kRefine; ++s) {
                const bool up = l > kl[s];
                const float tl = kl[s];
                kl[s] = up ? l : kl[s];
                l = up ? tl : l;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float tx = kx[s][i];
                    kx[s][i] = up ? x[i] : kx[s][i];
                    x[i] = up ? tx : x[i];
                }
            }
        }
        // phase 2: Newton refinement of the n_refine best kept points
#pragma unroll 1
        for (int s = 0; s < kRefine; ++s) {
            if (s >= a.n_refine) break;
            // the kept point s, picked with compile-time indices (registers,
            // no local memory)
            float ls = -INFINITY, x[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int j = 0; j < kRefine; ++j) {
                const bool pick = j == s;
                ls = pick ? kl[j] : ls;
#pragma unroll
                for (int i = 0; i < 4; ++i) x[i] = pick ? kx[j][i] : x[i];
            }
            if (!(ls > -INFINITY)) break;
            float l;
            refine<N>(C, sigma, a.newton, x, l);
            if (l > best_l) {
                best_l = l;
#pragma unroll
                for (int i = 0; i < 4; ++i) best_q[i] = x[i];
            }
        }
        // canonical representative of {q, -q}: first non-zero component positive
        float sgn = 1.f;
        if (best_q[0] != 0.f) sgn = best_q[0] < 0.f ? -1.f : 1.f;
        else if (best_q[1] != 0.f) sgn = best_q[1] < 0.f ? -1.f : 1.f;
        else if (best_q[2] != 0.f) sgn = best_q[2] < 0.f ? -1.f : 1.f;
        else sgn = best_q[3] < 0.f ? -1.f : 1.f;
#pragma unroll
        for (int i = 0; i < 4; ++i) best_q[i] *= sgn;
    }
    if (a.list.out_stride > 0) {
        float* qo = sg.quat + i * (size_t)a.list.out_stride;
#pragma unroll
        for (int k = 0; k < 4; ++k) qo[k] = best_q[k];
        if (sg.lambda) sg.lambda[i * (size_t)a.list.out_stride] = best_l;
        return;
    }
    reinterpret_cast<float4*>(sg.quat)[v] = make_float4(best_q[0], best_q[1], best_q[2], best_q[3]);
    if (sg.lambda) sg.lambda[v] = best_l;
}

// search_done: run only the refinement; search_only: run only the SIMT search
template <int N, typename CT>
ttm_status launch_n_t(const SearchArgs& s, const PolishArgs& p, bool search_done, bool search_only,
                      cudaStream_t st, long long* cnt) {
    if (s.b.ntiles == 0) return TTM_OK;
    const unsigned blocks = s.b.ntiles;
    if (!search_done) {
        const size_t smem = (size_t)kChunk * Geo<N>::K4 * sizeof(float) + kChunk * sizeof(int);
        TTM_CUDA_TRY(cudaFuncSetAttribute(search_simt_kernel<N, CT>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        search_simt_kernel<N, CT><<<blocks, kRotThreads, smem, st>>>(s);
        TTM_TRY(after_launch(cnt));
    }
    if (search_only) return TTM_OK;
    polish_kernel<N, CT><<<blocks, kRotThreads, 0, st>>>(p);
    return after_launch(cnt);
}

template <int N>
ttm_status launch_n(const SearchArgs& s, const PolishArgs& p, bool search_done, bool search_only,
                    bool bf16, cudaStream_t st, long long* cnt) {
    return bf16 ? launch_n_t<N, __nv_bfloat16>(s, p, search_done, search_only, st, cnt)
                : launch_n_t<N, float>(s, p, search_done, search_only, st, cnt);
}

}  // namespace rot

template <int N>
ttm_status launch_rotation_n(const rot::SearchArgs& s, const rot::PolishArgs& p, bool search_done,
                             bool search_only, bool bf16, cudaStream_t st, long long* cnt);

// tensor-core grid search for orders 4 and 6 with the default 2048-point grid
// in 128 regions (k_search_tc.cu); returns TTM_ERR_UNSUPPORTED otherwise
bool search_tc_supported(int n_order, int n_grid, int n_cells);
ttm_status launch_search_tc(int n_order, const rot::SearchArgs& s, const uint16_t* grid_fp16,
                            int* status, bool bf16, cudaStream_t st, long long* cnt);

}  // namespace ttm
