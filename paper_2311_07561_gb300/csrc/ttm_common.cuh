// Shared definitions of the CUDA path: status plumbing, launch accounting and
// compile-time tables of the symmetric tensors S^n(R^4) (Sec. 3.1 of the
// paper: a symmetric tensor of order n in dimension 4 has C(n+3, n)
// independent components).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "ttm.h"

namespace ttm {

// --------------------------------------------------------------------------
// error plumbing
// --------------------------------------------------------------------------

#define TTM_CUDA_TRY(expr)                                   \
    do {                                                     \
        cudaError_t _e = (expr);                             \
        if (_e != cudaSuccess) {                             \
            ::ttm::note_cuda_error(_e, #expr, __FILE__, __LINE__); \
            return TTM_ERR_CUDA;                             \
        }                                                    \
    } while (0)

#define TTM_TRY(expr)                                        \
    do {                                                     \
        ttm_status _s = (expr);                              \
        if (_s != TTM_OK) return _s;                         \
    } while (0)

void note_cuda_error(cudaError_t e, const char* what, const char* file, int line);

// Checks the launch that was just queued; counts it.
ttm_status after_launch(long long* counter);

// --------------------------------------------------------------------------
// bounded waits
// --------------------------------------------------------------------------

// Polls phase `phase` of the shared-memory mbarrier at `bar` at most `limit`
// times (mbarrier.try_wait, which itself suspends for a while between
// polls); false when the phase never completed.  Every device-side wait of
// the tensor-core kernels goes through this loop, so none can hang: a wait
// that runs out makes the kernel record TTM_ERR_TIMEOUT and return.
// The kernels' limit: 2^18 polls, about one second at the ~3.7 us a poll
// that does not complete takes on GB300 (measured by ttm_probe_bounded_wait),
// far beyond any MMA or bulk-copy latency.
constexpr long kMbarWaitPolls = 1L << 18;

#ifdef __CUDACC__
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t phase, long limit) {
    for (long it = 0; it < limit; ++it) {
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
#endif

// --------------------------------------------------------------------------
// symmetric tensor tables
// --------------------------------------------------------------------------

__host__ __device__ constexpr int binom(int n, int k) {
    long long r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return (int)r;
}

// Number of independent components of S^n(R^4).
__host__ __device__ constexpr int n_comp(int n) { return n < 0 ? 0 : binom(n + 3, 3); }

__host__ __device__ constexpr int factorial(int n) {
    int r = 1;
    for (int i = 2; i <= n; ++i) r *= i;
    return r;
}

// Exponent vectors of the components of S^N(R^4), in the lexicographic order
// of their sorted index tuples i1 <= ... <= iN (the component order of the C
// ABI), with the multinomial weight mu = N! / (e0! e1! e2! e3!) of each (the
// number of full index tuples that sort to it).
template <int N>
struct Sym {
    static constexpr int K = n_comp(N);
    int e[K > 0 ? K : 1][4];
    int mu[K > 0 ? K : 1];

    __host__ __device__ constexpr Sym() : e{}, mu{} {
        int t[N > 0 ? N : 1] = {};
        for (int k = 0; k < K; ++k) {
            int ex[4] = {0, 0, 0, 0};
            for (int p = 0; p < N; ++p) ex[t[p]] += 1;
            for (int i = 0; i < 4; ++i) e[k][i] = ex[i];
            mu[k] = factorial(N) / (factorial(ex[0]) * factorial(ex[1]) * factorial(ex[2]) *
                                    factorial(ex[3]));
            // next non-decreasing tuple: bump the rightmost entry below 3 and
            // copy it to the right
            int p = N - 1;
            while (p >= 0 && t[p] == 3) --p;
            if (p < 0) break;
            t[p] += 1;
            for (int q = p + 1; q < N; ++q) t[q] = t[p];
        }
    }

    // Position of the component with exponents (a, b, c, d), or -1.
    __host__ __device__ constexpr int find(int a, int b, int c, int d) const {
        for (int k = 0; k < K; ++k)
            if (e[k][0] == a && e[k][1] == b && e[k][2] == c && e[k][3] == d) return k;
        return -1;
    }
};

// Table for the Hessian-like matrix H = A x^{N-2} of a symmetric tensor A of
// order N (Sec. 3.1: (A x^k) contracts k indices with x).  Entry (i, j) is
//   H_ij = sum_beta mult(beta) A_{sorted(i, j, beta)} x^beta,
// the sum running over the components beta of S^{N-2}(R^4).  For each of the
// 10 pairs i <= j and each beta the table stores the component index of A
// and the weight mult(beta).
template <int N>
struct HessTab {
    static constexpr int KB = n_comp(N - 2);
    int comp[10][KB > 0 ? KB : 1];
    int mult[KB > 0 ? KB : 1];
    int pi[10], pj[10];

    __host__ __device__ constexpr HessTab() : comp{}, mult{}, pi{}, pj{} {
        constexpr Sym<N> A{};
        constexpr Sym<N - 2> B{};
        int p = 0;
        for (int i = 0; i < 4; ++i)
            for (int j = i; j < 4; ++j) {
                pi[p] = i;
                pj[p] = j;
                for (int b = 0; b < KB; ++b) {
                    int ex[4] = {B.e[b][0], B.e[b][1], B.e[b][2], B.e[b][3]};
                    ex[i] += 1;
                    ex[j] += 1;
                    comp[p][b] = A.find(ex[0], ex[1], ex[2], ex[3]);
                }
                ++p;
            }
        for (int b = 0; b < KB; ++b) mult[b] = B.mu[b];
    }
};

// Table for the vector g = A x^{N-1} of a symmetric tensor A of order N
// (Sec. 3.1): g_i = sum_gamma mult(gamma) A_{sorted(i, gamma)} x^gamma, the sum
// over the components gamma of S^{N-1}(R^4) with their multinomial weights.
template <int N>
struct GradTab {
    static constexpr int KG = n_comp(N - 1);
    int comp[4][KG > 0 ? KG : 1];
    int mult[KG > 0 ? KG : 1];

    __host__ __device__ constexpr GradTab() : comp{}, mult{} {
        constexpr Sym<N> A{};
        constexpr Sym<N - 1> G{};
        for (int i = 0; i < 4; ++i)
            for (int g = 0; g < KG; ++g) {
                int ex[4] = {G.e[g][0], G.e[g][1], G.e[g][2], G.e[g][3]};
                ex[i] += 1;
                comp[i][g] = A.find(ex[0], ex[1], ex[2], ex[3]);
            }
        for (int g = 0; g < KG; ++g) mult[g] = G.mu[g];
    }
};

// Monomials x^beta for every component beta of S^M(R^4), computed from the
// degree-(M-1) monomials by one multiplication each.
template <int M>
struct MonoTab {
    static constexpr int KM = n_comp(M);
    static constexpr int KP = n_comp(M - 1);
    int parent[KM > 0 ? KM : 1];   // index among degree M-1 monomials
    int var[KM > 0 ? KM : 1];      // variable multiplied in
    __host__ __device__ constexpr MonoTab() : parent{}, var{} {
        constexpr Sym<M> S{};
        constexpr Sym<M - 1> P{};
        for (int k = 0; k < KM; ++k) {
            int i = 0;
            while (S.e[k][i] == 0) ++i;      // lowest variable present
            int ex[4] = {S.e[k][0], S.e[k][1], S.e[k][2], S.e[k][3]};
            ex[i] -= 1;
            parent[k] = P.find(ex[0], ex[1], ex[2], ex[3]);
            var[k] = i;
        }
    }
};

template <int M>
struct Monomials {
    float v[n_comp(M) > 0 ? n_comp(M) : 1];
};

template <int M>
__device__ __forceinline__ void monomials(const float x[4], Monomials<M>& out) {
    if constexpr (M == 0) {
        out.v[0] = 1.0f;
    } else {
        Monomials<M - 1> prev;
        monomials<M - 1>(x, prev);
        constexpr MonoTab<M> T{};
#pragma unroll
        for (int k = 0; k < n_comp(M); ++k) out.v[k] = prev.v[T.parent[k]] * x[T.var[k]];
    }
}

// Interior range of a volume axis of length n for box edge s: [c, n - s + c].
__host__ __device__ inline bool interior(int v, int n, int s) {
    int c = s / 2;
    return v >= c && v <= n - s + c;
}

}  // namespace ttm
