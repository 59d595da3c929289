// Two-level line FFTs for the long lines of the correlation path.
//
// A line of length L = L1 L2 is transformed with one shared-memory exchange:
// with n = n1 + L1 n2 and k = k2 + L2 k1,
//   X[k2 + L2 k1] = sum_n1 W_L^(n1 k2) W_L1^(n1 k1) sum_n2 x[n1 + L1 n2] W_L2^(n2 k2),
// so thread n1 loads its L2 samples x[n1 + L1 n2] straight from global memory
// into registers, transforms them (DFT of length L2 in registers), multiplies
// by W_L^(n1 k2) and writes them to shared memory; after one barrier thread k2
// reads the L1 values of its column k2, transforms them (DFT of length L1 in
// registers) and stores X[k2 + L2 k1] straight to global memory.  Each point
// crosses shared memory once (a write and a read) instead of once per
// Stockham stage, and the layouts below are free of bank conflicts.
//
// The register DFTs are mixed-radix Cooley-Tukey splits N = P Q down to the
// radices of dft_small (2, 3, 4, 5, 8, 16); their internal twiddles are
// compile-time constants from a constexpr table (cos and sin of 2 pi m / N
// by Taylor series in double precision, rounded to float).  The twiddles
// W_L^(n1 k2) come from the FP64-computed table of the pass.
#pragma once

namespace ttm {
namespace fftk {

// ---- compile-time cos / sin of 2 pi m / N --------------------------------
constexpr double kTwoPi = 6.283185307179586476925287;

constexpr double taylor_sin(double x) {
    double term = x, sum = x;
    for (int k = 1; k < 16; ++k) {
        term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
        sum += term;
    }
    return sum;
}

constexpr double taylor_cos(double x) {
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 16; ++k) {
        term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
        sum += term;
    }
    return sum;
}

// angle 2 pi m / N brought into (-pi, pi] with exact integer arithmetic
constexpr double angle_2pi(int m, int N) {
    m %= N;
    if (m < 0) m += N;
    if (2 * m > N) m -= N;
    return kTwoPi * (double)m / (double)N;
}

template <int N>
struct TwTable {
    float c[N], s[N];
    constexpr TwTable() : c(), s() {
        for (int m = 0; m < N; ++m) {
            c[m] = (float)taylor_cos(angle_2pi(m, N));
            s[m] = (float)taylor_sin(angle_2pi(m, N));
        }
    }
};

// exp(SIGN 2 pi i m / N) for a compile-time m after unrolling
template <int N, int SIGN>
__device__ __forceinline__ float2 tw_const(int m) {
    constexpr TwTable<N> T{};
    const int r = ((m % N) + N) % N;
    return make_float2(T.c[r], SIGN < 0 ? -T.s[r] : T.s[r]);
}

// a * exp(SIGN 2 pi i m / N) for a compile-time m: the multiplications by
// +-1 and +-i are swaps and sign changes
template <int N, int SIGN>
__device__ __forceinline__ float2 mul_tw(float2 a, int m) {
    const int r = ((m % N) + N) % N;
    if (r == 0) return a;
    if (2 * r == N) return make_float2(-a.x, -a.y);
    if (4 * r == N) return mul_mi<SIGN>(a);
    if (4 * r == 3 * N) return mul_mi<-SIGN>(a);
    return cmul(a, tw_const<N, SIGN>(r));
}

// ---- register DFTs of compile-time length ---------------------------------
__host__ __device__ constexpr bool base_radix(int n) {
    return n == 2 || n == 3 || n == 4 || n == 5 || n == 8 || n == 16;
}
// first factor of a split N = P Q: the largest base radix dividing N
__host__ __device__ constexpr int split_p(int n) {
    return n % 16 == 0 ? 16 : n % 8 == 0 ? 8 : n % 5 == 0 ? 5 : n % 4 == 0 ? 4 : n % 3 == 0 ? 3 : 2;
}

template <int N, int SIGN>
__device__ __forceinline__ void dft_reg(float2 (&v)[N]);

// N = P Q: for each q the P samples v[Q p + q] are transformed, multiplied
// by W_N^(q k1), and for each k1 the Q values are transformed into
// X[k1 + P k2]
template <int N, int P, int SIGN>
__device__ __forceinline__ void dft_split(float2 (&v)[N]) {
    constexpr int Q = N / P;
    float2 t[N];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        float2 a[P];
#pragma unroll
        for (int p = 0; p < P; ++p) a[p] = v[Q * p + q];
        dft_reg<P, SIGN>(a);
#pragma unroll
        for (int k1 = 0; k1 < P; ++k1)
            t[k1 * Q + q] = mul_tw<N, SIGN>(a[k1], q * k1);
    }
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) {
        float2 b[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) b[q] = t[k1 * Q + q];
        dft_reg<Q, SIGN>(b);
#pragma unroll
        for (int k2 = 0; k2 < Q; ++k2) v[k1 + P * k2] = b[k2];
    }
}

template <int N, int SIGN>
__device__ __forceinline__ void dft_reg(float2 (&v)[N]) {
    if constexpr (N == 1) {
        return;
    } else if constexpr (base_radix(N)) {
        dft_small<N, SIGN>(v);
    } else {
        dft_split<N, split_p(N), SIGN>(v);
    }
}

// ---- line lengths that take the two-level passes ---------------------------
// L = L1 L2 with L1 threads per line in the first step (16 up to 480, 32
// from 512): every compiled length from 128 up
template <int L> struct TwoLevel { static constexpr int L1 = 0, L2 = 0; };
#define TTM_TWO_LEVEL(L_, L1_) \
    template <> struct TwoLevel<L_> { static constexpr int L1 = L1_, L2 = L_ / L1_; };
TTM_TWO_LEVEL(128, 16) TTM_TWO_LEVEL(144, 16) TTM_TWO_LEVEL(160, 16) TTM_TWO_LEVEL(192, 16)
TTM_TWO_LEVEL(240, 16) TTM_TWO_LEVEL(256, 16) TTM_TWO_LEVEL(288, 16) TTM_TWO_LEVEL(320, 16)
TTM_TWO_LEVEL(384, 16) TTM_TWO_LEVEL(480, 16) TTM_TWO_LEVEL(512, 32) TTM_TWO_LEVEL(576, 32)
TTM_TWO_LEVEL(640, 32) TTM_TWO_LEVEL(768, 32) TTM_TWO_LEVEL(960, 32) TTM_TWO_LEVEL(1024, 32)
#undef TTM_TWO_LEVEL
// taken where the Stockham form needs three or more shared-memory stages
// (at 128 and 256 its two radix-16 stages measured as fast or faster)
template <int L> constexpr bool two_level() { return TwoLevel<L>::L1 > 0 && n_stages(L) >= 3; }

// resident CTAs per SM the register budget is sized for: two for lines whose
// second factor is at most 16 (their register DFTs are small), else one
template <int L2> constexpr int two_min_blocks() { return L2 <= 16 ? 2 : 1; }
// the column pass also with bf16 samples up to L2 = 30: its register DFTs
// and the prefetched bf16 pairs fit 128 registers (FP32 samples, twice the
// prefetch registers, and 32-point DFTs spill)
template <int L2, typename PS> constexpr int cols_min_blocks() {
    return L2 <= 16 || (sizeof(PS) == 4 && L2 <= 30) ? 2 : 1;
}

constexpr int kTwoThreads = 256;

// exchange buffer bytes of the column passes: L2 rows of (L1 + 1) x TB values
template <int L1, int L2>
constexpr size_t two_cols_smem() { return (size_t)L2 * (L1 + 1) * (kTwoThreads / L1) * sizeof(float2); }

// ---- column pass: lines of length L1 L2, element stride B ---------------
// Tile = TB = 256 / L1 consecutive columns of one plane (ColsMap); persistent
// CTAs, the raw samples of the next tile are loaded into registers while the
// current one is transformed.  Line samples lo..hi are stored.
template <int L1, int L2, int SIGN, typename PS>
__global__ void __launch_bounds__(kTwoThreads, cols_min_blocks<L2, PS>()) cols2_t(PS* __restrict__ data, int B,
                                                          const float2* __restrict__ tw,
                                                          ColsMap mp, int ntb, size_t ntiles) {
    constexpr int L = L1 * L2;
    constexpr int TB = kTwoThreads / L1;
    constexpr int ZP = L1 + 1;
    extern __shared__ float2 zx[];                    // [k2][n1 (padded)][column]
    const int t = threadIdx.x;
    const int n1 = t / TB, ca = t % TB;
    PS raw[L2];
    auto load = [&](size_t tile) {
        const size_t plane = tile / (size_t)ntb;
        const int b = (int)(tile - plane * (size_t)ntb) * TB + ca;
        const size_t base = cols_plane_base(mp, (size_t)mp.p0 + plane, L, B);
        if (b < B) {
#pragma unroll
            for (int n2 = 0; n2 < L2; ++n2) raw[n2] = data[base + (size_t)(n1 + L1 * n2) * B + b];
        }
    };
    size_t tile = blockIdx.x;
    if (tile >= ntiles) return;
    load(tile);
    for (; tile < ntiles; tile += gridDim.x) {
        const size_t plane = tile / (size_t)ntb;
        const int b0 = (int)(tile - plane * (size_t)ntb) * TB;
        const size_t base = cols_plane_base(mp, (size_t)mp.p0 + plane, L, B);
        float2 v[L2];
        const bool in_a = b0 + ca < B;
#pragma unroll
        for (int n2 = 0; n2 < L2; ++n2) v[n2] = in_a ? ldc(&raw[n2]) : make_float2(0.f, 0.f);
        if (tile + gridDim.x < ntiles) load(tile + gridDim.x);
        dft_reg<L2, SIGN>(v);
#pragma unroll
        for (int k2 = 1; k2 < L2; ++k2) {
            float2 w = __ldg(tw + n1 * k2);            // n1 k2 < L
            if (SIGN > 0) w.y = -w.y;
            v[k2] = cmul(v[k2], w);
        }
        __syncthreads();                               // the previous tile's reads are done
#pragma unroll
        for (int k2 = 0; k2 < L2; ++k2) zx[(k2 * ZP + n1) * TB + ca] = v[k2];
        __syncthreads();
        for (int it = t; it < L2 * TB; it += kTwoThreads) {
            const int k2 = it / TB, col = it % TB;
            float2 u[L1];
#pragma unroll
            for (int m = 0; m < L1; ++m) u[m] = zx[(k2 * ZP + m) * TB + col];
            dft_reg<L1, SIGN>(u);
            const int b = b0 + col;
            if (b < B) {
#pragma unroll
                for (int k1 = 0; k1 < L1; ++k1) {
                    const int l = k2 + L2 * k1;
                    if (l >= mp.lo && l <= mp.hi) stc(data + base + (size_t)l * B + b, u[k1]);
                }
            }
        }
    }
}

// ---- z lines of F(f) conj(T_k) for all K components, inverse ----------------
// One tile of TB columns per CTA: the image samples of this thread stay in
// registers, the next component's samples are fetched while the current
// product is transformed; z samples lo..hi of every product are stored.
// With FP32 template spectra the fetch goes to registers; with bf16 ones it
// is a cp.async copy into a staging buffer (each thread its own slots), which
// frees those registers for a second CTA per SM.

// 4-byte asynchronous copy global -> shared, its commit and wait
__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// CTAs per SM the fused multiply's registers are sized for, and its shared
// memory: the exchange buffer, plus the staging buffer for bf16 samples
template <typename TS> constexpr int mul_min_blocks(int l2) {
    return sizeof(TS) == 4 ? 2 : (l2 <= 16 ? 2 : 1);
}
template <int L1, int L2, typename TS> constexpr size_t mul2_smem() {
    return two_cols_smem<L1, L2>() + (sizeof(TS) == 4 ? (size_t)L2 * kTwoThreads * 4 : 0);
}

template <int L1, int L2, typename TS, typename PS>
__global__ void __launch_bounds__(kTwoThreads, mul_min_blocks<TS>(L2)) cols_mul2_t(const float2* __restrict__ spec,
                                                              const TS* __restrict__ tspec,
                                                              PS* __restrict__ out, int B, int K,
                                                              const float2* __restrict__ tw,
                                                              int lo, int hi) {
    constexpr int L = L1 * L2;
    constexpr int TB = kTwoThreads / L1;
    constexpr int ZP = L1 + 1;
    constexpr bool kAsync = sizeof(TS) == 4;
    extern __shared__ float2 zx[];
    TS* stg = reinterpret_cast<TS*>(zx + L2 * ZP * TB);      // [n2][thread] (async form)
    const int t = threadIdx.x;
    const int n1 = t / TB, ca = t % TB;
    const int b0 = blockIdx.x * TB;
    const size_t plane = (size_t)L * B;
    const bool in_a = b0 + ca < B;
    const size_t e0 = (size_t)n1 * B + b0 + ca;
    float2 fi[L2];
    TS tr[kAsync ? 1 : L2];
    auto stage = [&](int k) {
        if (!in_a) return;
        const TS* ts = tspec + (size_t)k * plane + e0;
#pragma unroll
        for (int n2 = 0; n2 < L2; ++n2)
            cp_async4((uint32_t)__cvta_generic_to_shared(stg + n2 * kTwoThreads + t), ts + (size_t)n2 * L1 * B);
        cp_async_commit();
    };
#pragma unroll
    for (int n2 = 0; n2 < L2; ++n2) {
        const size_t e = e0 + (size_t)n2 * L1 * B;
        fi[n2] = in_a ? spec[e] : make_float2(0.f, 0.f);
        if constexpr (!kAsync) { if (in_a && K > 0) tr[n2] = tspec[e]; }
    }
    if constexpr (kAsync) { if (K > 0) stage(0); }
    for (int k = 0; k < K; ++k) {
        float2 v[L2];
        if constexpr (kAsync) {
            cp_async_wait_all();
#pragma unroll
            for (int n2 = 0; n2 < L2; ++n2)
                v[n2] = in_a ? cmulc(fi[n2], ldc(stg + n2 * kTwoThreads + t)) : make_float2(0.f, 0.f);
            if (k + 1 < K) stage(k + 1);
        } else {
#pragma unroll
            for (int n2 = 0; n2 < L2; ++n2) v[n2] = in_a ? cmulc(fi[n2], ldc(&tr[n2])) : make_float2(0.f, 0.f);
            if (in_a && k + 1 < K) {
                const TS* ts = tspec + (size_t)(k + 1) * plane;
#pragma unroll
                for (int n2 = 0; n2 < L2; ++n2) tr[n2] = ts[(size_t)(n1 + L1 * n2) * B + b0 + ca];
            }
        }
        dft_reg<L2, +1>(v);
#pragma unroll
        for (int k2 = 1; k2 < L2; ++k2) {
            float2 w = __ldg(tw + n1 * k2);
            w.y = -w.y;
            v[k2] = cmul(v[k2], w);
        }
        __syncthreads();
#pragma unroll
        for (int k2 = 0; k2 < L2; ++k2) zx[(k2 * ZP + n1) * TB + ca] = v[k2];
        __syncthreads();
        PS* o = out + (size_t)k * plane;
        for (int it = t; it < L2 * TB; it += kTwoThreads) {
            const int k2 = it / TB, col = it % TB;
            float2 u[L1];
#pragma unroll
            for (int m = 0; m < L1; ++m) u[m] = zx[(k2 * ZP + m) * TB + col];
            dft_reg<L1, +1>(u);
            const int b = b0 + col;
            if (b < B) {
#pragma unroll
                for (int k1 = 0; k1 < L1; ++k1) {
                    const int l = k2 + L2 * k1;
                    if (l >= lo && l <= hi) stc(o + (size_t)l * B + b, u[k1]);
                }
            }
        }
    }
    if constexpr (kAsync) cp_async_wait_all();
}

// ---- half-spectrum rows -> real x lines, two-level ------------------------
// A tile is NR = 256 / L1 kept rows (z in keep.z0..z1, y in keep.y0..y1 of
// every batch item, in that order); thread (row, n1) loads its L2 samples of
// the Hermitian extension X[L - x] = conj X[x] straight from global memory;
// the next tile's samples are loaded while the current one is transformed.
// The real parts of the kept samples x0..x1 go to the X x Y x Z maps.
template <int L1, int L2>
constexpr size_t two_rows_smem() { return (size_t)(kTwoThreads / L1) * L2 * (L1 + 1) * sizeof(float2); }

template <int L1, int L2, typename PS, typename RT>
__global__ void __launch_bounds__(kTwoThreads, two_min_blocks<L2>()) rows_c2r2_t(const PS* __restrict__ in, int X,
                                                              int Y, int Z, FftGeom g,
                                                              RT* __restrict__ out, int n_batch,
                                                              const float2* __restrict__ tw,
                                                              FftKeep keep) {
    constexpr int L = L1 * L2;
    constexpr int XH = L / 2 + 1;
    constexpr int NR = kTwoThreads / L1;
    constexpr int ZP = L1 + 1;
    extern __shared__ float2 zx[];                    // [row][k2][n1 (padded)]
    const int t = threadIdx.x;
    const int ra = t / L1, n1 = t % L1;
    const int ny = keep.y1 - keep.y0 + 1, nz = keep.z1 - keep.z0 + 1;
    const size_t nrows = (size_t)n_batch * nz * ny;
    const size_t ntiles = (nrows + NR - 1) / NR;
    // row q of the kept rows: its half-spectrum row and its output offset
    auto row_of = [&](size_t q, size_t& src_row, long long& dst) {
        const size_t per_item = (size_t)nz * ny;
        const size_t item = q / per_item;
        const size_t r = q - item * per_item;
        const int z = keep.z0 + (int)(r / (size_t)ny);
        const int y = keep.y0 + (int)(r % (size_t)ny);
        src_row = (item * (size_t)g.Zp + (size_t)z) * (size_t)g.Yp + (size_t)y;
        dst = (y < Y && z < Z) ? (long long)(item * ((size_t)X * Y * Z) + ((size_t)z * Y + y) * X)
                               : -1;
    };
    PS raw[L2];
    auto load = [&](size_t tile) {
        const size_t q = tile * NR + ra;
        if (q < nrows) {
            size_t src;
            long long dst;
            row_of(q, src, dst);
            const PS* rowp = in + src * XH;
#pragma unroll
            for (int n2 = 0; n2 < L2; ++n2) {
                const int n = n1 + L1 * n2;
                raw[n2] = rowp[n < XH ? n : L - n];
            }
        }
    };
    size_t tile = blockIdx.x;
    if (tile >= ntiles) return;
    load(tile);
    const int xk0 = keep.x0, xk1 = min(keep.x1, X - 1);
    for (; tile < ntiles; tile += gridDim.x) {
        float2 v[L2];
        const bool in_a = tile * NR + ra < nrows;
#pragma unroll
        for (int n2 = 0; n2 < L2; ++n2) {
            const int n = n1 + L1 * n2;
            float2 c = in_a ? ldc(&raw[n2]) : make_float2(0.f, 0.f);
            if (n >= XH) c.y = -c.y;                   // conj X[L - n]
            v[n2] = c;
        }
        if (tile + gridDim.x < ntiles) load(tile + gridDim.x);
        dft_reg<L2, +1>(v);
#pragma unroll
        for (int k2 = 1; k2 < L2; ++k2) {
            float2 w = __ldg(tw + n1 * k2);
            w.y = -w.y;
            v[k2] = cmul(v[k2], w);
        }
        __syncthreads();
#pragma unroll
        for (int k2 = 0; k2 < L2; ++k2) zx[(ra * L2 + k2) * ZP + n1] = v[k2];
        __syncthreads();
        for (int it = t; it < NR * L2; it += kTwoThreads) {
            const int rb = it / L2, k2 = it % L2;
            const size_t q = tile * NR + rb;
            if (q >= nrows) continue;
            size_t src;
            long long dst;
            row_of(q, src, dst);
            float2 u[L1];
#pragma unroll
            for (int m = 0; m < L1; ++m) u[m] = zx[(rb * L2 + k2) * ZP + m];
            dft_reg<L1, +1>(u);
            if (dst >= 0) {
#pragma unroll
                for (int k1 = 0; k1 < L1; ++k1) {
                    const int x = k2 + L2 * k1;
                    if (x >= xk0 && x <= xk1) str(out + dst + x, u[k1].x);
                }
            }
        }
    }
}

// ---- half-spectrum rows -> real x lines through a half-length transform -----
// A real line y[n] = sum_k X[k] W_L^(-n k) of even length L = 2M is the
// complex transform of length M of
//   Z[k] = X[k] + conj X[M-k] + i (X[k] - conj X[M-k]) W_L^(-k),   k < M,
// read as z[m] = y[2m] + i y[2m+1]: half the transform work of the full-length
// pass, and the outputs leave in pairs.  M = L1 L2 takes the two-level form
// (thread (row, n1) holds Z[n1 + L1 n2]; the twiddles of length M are
// W_M^j = W_L^(2j) from the pass's table).  The samples X[k] of the next tile
// are loaded into registers while the current one is transformed; X[M-k]
// (another thread's X[k'] of the same row) is read when needed.
template <int L> constexpr bool c2r_half() { return L >= 256 && TwoLevel<L / 2>::L1 > 0; }

// split of the half length M = L1 L2 in the row pass: the column passes' split,
// except 480 = 32 x 15 (register DFTs of 15 and 32 points instead of 30 and 16
// leave room for two CTAs per SM)
template <int M> struct RowSplit { static constexpr int L1 = TwoLevel<M>::L1, L2 = TwoLevel<M>::L2; };
template <> struct RowSplit<480> { static constexpr int L1 = 32, L2 = 15; };

// split of the fused multiply's z lines (the column passes' split by default)
template <int L> struct MulSplit { static constexpr int L1 = TwoLevel<L>::L1, L2 = TwoLevel<L>::L2; };

// row groups per tile of the half-length row pass: two when one group's
// second-step items (NR rows x L2) would leave threads idle and the samples
// are bf16 pairs (two groups of FP32 samples do not fit the registers)
template <int L1, int L2, typename PS> constexpr int c2r_groups() {
    return sizeof(PS) == 4 && (kTwoThreads / L1) * L2 < kTwoThreads ? 2 : 1;
}
template <int L1, int L2, typename PS> constexpr size_t c2r_half_smem() {
    return (size_t)c2r_groups<L1, L2, PS>() * two_rows_smem<L1, L2>();
}

// the sample of lane src of a row's L1 lanes (a row is one warp or half of one)
template <int W>
__device__ __forceinline__ float2 shfl_row(float2 v, int src) {
    return make_float2(__shfl_sync(0xffffffffu, v.x, src, W), __shfl_sync(0xffffffffu, v.y, src, W));
}
template <int W>
__device__ __forceinline__ __nv_bfloat162 shfl_row(__nv_bfloat162 v, int src) {
    unsigned u;
    memcpy(&u, &v, sizeof(u));
    u = __shfl_sync(0xffffffffu, u, src, W);
    memcpy(&v, &u, sizeof(u));
    return v;
}

// two adjacent real outputs in one store (p aligned to two elements)
__device__ __forceinline__ void str2(float* p, float a, float b) {
    *reinterpret_cast<float2*>(p) = make_float2(a, b);
}
__device__ __forceinline__ void str2(__nv_bfloat16* p, float a, float b) {
    *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(a, b);
}

// A tile is NG groups of NR rows.  Thread (row, n1) holds X[n1 + L1 n2] of
// its row; X[M - k] of its sample k is sample L2 - 1 - n2 of lane L1 - n1 of
// the same row (sample L2 - n2 of lane 0, or X[M], for lane 0), read by a
// shuffle.  The outputs z[m] = (y[2m], y[2m + 1]) are stored as pairs.
template <int L1, int L2, typename PS, typename RT>
__global__ void __launch_bounds__(kTwoThreads, two_min_blocks<L2>()) rows_c2r_half_t(
    const PS* __restrict__ in, int X, int Y, int Z, FftGeom g, RT* __restrict__ out, int n_batch,
    const float2* __restrict__ tw, FftKeep keep) {
    constexpr int M = L1 * L2;
    constexpr int XH = M + 1;
    constexpr int NR = kTwoThreads / L1;
    constexpr int NG = c2r_groups<L1, L2, PS>();
    constexpr int ZP = L1 + 1;
    static_assert(L1 == 16 || L1 == 32, "a row is one warp or half of one");
    extern __shared__ float2 zx[];                    // [group row][k2][n1 (padded)]
    const int t = threadIdx.x;
    const int ra = t / L1, n1 = t % L1;
    const int partner = (L1 - n1) & (L1 - 1);
    const int ny = keep.y1 - keep.y0 + 1, nz = keep.z1 - keep.z0 + 1;
    const size_t nrows = (size_t)n_batch * nz * ny;
    const size_t ntiles = (nrows + NG * NR - 1) / (NG * NR);
    auto row_of = [&](size_t q, size_t& src_row, long long& dst) {
        const size_t per_item = (size_t)nz * ny;
        const size_t item = q / per_item;
        const size_t r = q - item * per_item;
        const int z = keep.z0 + (int)(r / (size_t)ny);
        const int y = keep.y0 + (int)(r % (size_t)ny);
        src_row = (item * (size_t)g.Zp + (size_t)z) * (size_t)g.Yp + (size_t)y;
        dst = (y < Y && z < Z) ? (long long)(item * ((size_t)X * Y * Z) + ((size_t)z * Y + y) * X)
                               : -1;
    };
    PS raw[NG][L2];
    PS xm[NG];                                        // X[M] of the row
#pragma unroll
    for (int h = 0; h < NG; ++h) {
        memset(&xm[h], 0, sizeof(PS));
#pragma unroll
        for (int n2 = 0; n2 < L2; ++n2) memset(&raw[h][n2], 0, sizeof(PS));
    }
    auto load = [&](size_t tile) {
#pragma unroll
        for (int h = 0; h < NG; ++h) {
            const size_t q = (tile * NG + h) * NR + ra;
            if (q < nrows) {
                size_t src;
                long long dst;
                row_of(q, src, dst);
                const PS* rowp = in + src * XH;
#pragma unroll
                for (int n2 = 0; n2 < L2; ++n2) raw[h][n2] = rowp[n1 + L1 * n2];
                xm[h] = rowp[M];
            }
        }
    };
    size_t tile = blockIdx.x;
    if (tile >= ntiles) return;
    load(tile);
    const int xk0 = keep.x0, xk1 = min(keep.x1, X - 1);
    for (; tile < ntiles; tile += gridDim.x) {
        __syncthreads();                               // the previous tile's reads are done
#pragma unroll
        for (int h = 0; h < NG; ++h) {
            const bool in_a = (tile * NG + h) * NR + ra < nrows;
            float2 v[L2];
#pragma unroll
            for (int n2 = 0; n2 < L2; ++n2) {
                const int k = n1 + L1 * n2;
                PS mb = shfl_row<L1>(raw[h][L2 - 1 - n2], partner);
                if (n1 == 0) mb = n2 == 0 ? xm[h] : raw[h][(L2 - n2) % L2];
                float2 zk = make_float2(0.f, 0.f);
                if (in_a) {
                    const float2 a = ldc(&raw[h][n2]);
                    float2 b = ldc(&mb);
                    b.y = -b.y;                        // conj X[M - k]
                    float2 w = __ldg(tw + k);
                    w.y = -w.y;                        // W_L^(-k)
                    const float2 d = cmul(csub(a, b), w);
                    zk = make_float2(a.x + b.x - d.y, a.y + b.y + d.x);   // (a + b) + i d
                }
                v[n2] = zk;
            }
            dft_reg<L2, +1>(v);
#pragma unroll
            for (int k2 = 1; k2 < L2; ++k2) {
                float2 w = __ldg(tw + 2 * n1 * k2);    // W_M^(n1 k2) = W_L^(2 n1 k2)
                w.y = -w.y;
                v[k2] = cmul(v[k2], w);
            }
#pragma unroll
            for (int k2 = 0; k2 < L2; ++k2) zx[((h * NR + ra) * L2 + k2) * ZP + n1] = v[k2];
        }
        if (tile + gridDim.x < ntiles) load(tile + gridDim.x);
        __syncthreads();
        for (int it = t; it < NG * NR * L2; it += kTwoThreads) {
            const int rb = it / L2, k2 = it % L2;
            const size_t q = tile * NG * NR + rb;
            if (q >= nrows) continue;
            size_t src;
            long long dst;
            row_of(q, src, dst);
            float2 u[L1];
#pragma unroll
            for (int m = 0; m < L1; ++m) u[m] = zx[(rb * L2 + k2) * ZP + m];
            dft_reg<L1, +1>(u);
            if (dst >= 0) {
                RT* o = out + dst;
                const bool pair_ok = (reinterpret_cast<uintptr_t>(o) & (2 * sizeof(RT) - 1)) == 0;
#pragma unroll
                for (int k1 = 0; k1 < L1; ++k1) {
                    const int x = 2 * (k2 + L2 * k1);   // z[m] = (y[2m], y[2m+1])
                    if (pair_ok && x >= xk0 && x + 1 <= xk1) {
                        str2(o + x, u[k1].x, u[k1].y);
                    } else {
                        if (x >= xk0 && x <= xk1) str(o + x, u[k1].x);
                        if (x + 1 >= xk0 && x + 1 <= xk1) str(o + x + 1, u[k1].y);
                    }
                }
            }
        }
    }
}

// ---- real x lines -> half-spectrum rows through a half-length transform ------
// The forward counterpart: z[m] = x[2m] + i x[2m+1] (m < M, L = 2M), Z = the
// complex transform of length M (two-level, RowSplit), then
//   X[k] = (Z[k] + conj Z[M-k]) / 2 - i W_L^k (Z[k] - conj Z[M-k]) / 2,  k = 0..M
// (Z[M] = Z[0]) through a second exchange in shared memory.  Every row of the
// padded box is written (rows beyond the data are zero).  mode 0 transforms
// f, mode 1 (f - mean), mode 2 (f - mean)^2 and adds sum (f - mean)^4 into
// moments[2], mean = moments[0] / (X Y Z), as the Stockham pass does.
template <int L> constexpr bool r2c_half() { return L >= 256 && TwoLevel<L / 2>::L1 > 0; }

template <int L1, int L2>
__global__ void __launch_bounds__(kTwoThreads, two_min_blocks<L2>()) rows_r2c_half_t(
    const float* __restrict__ f, int X, int Y, int Z, FftGeom g, float2* __restrict__ out,
    const float2* __restrict__ tw, int mode, double* __restrict__ moments) {
    constexpr int M = L1 * L2;
    constexpr int XH = M + 1;
    constexpr int NR = kTwoThreads / L1;
    constexpr int ZP = L1 + 1;
    extern __shared__ float2 zx[];                    // exchange, then the rows' Z
    __shared__ double part[kTwoThreads / 32];
    const int t = threadIdx.x;
    const int ra = t / L1, n1 = t % L1;
    const size_t nrows = (size_t)g.Yp * g.Zp;
    const size_t ntiles = (nrows + NR - 1) / NR;
    const float mean = mode ? (float)(moments[0] / ((double)X * Y * Z)) : 0.f;
    // input offset of row q of the padded box, -1 for a zero row
    auto src_of = [&](size_t q) -> long long {
        if (q >= nrows) return -1;
        const int y = (int)(q % (size_t)g.Yp), z = (int)(q / (size_t)g.Yp);
        return (y < Y && z < Z) ? (long long)(((size_t)z * Y + y) * X) : -1;
    };
    float q4 = 0.f;                                   // mode 2: this thread's sum of (f - mean)^4
    for (size_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long sa = src_of(tile * NR + ra);
        float2 v[L2];
#pragma unroll
        for (int n2 = 0; n2 < L2; ++n2) {
            const int x = 2 * (n1 + L1 * n2);
            float a = 0.f, b = 0.f;
            if (sa >= 0) {
                if (x < X) a = __ldg(f + sa + x) - mean;
                if (x + 1 < X) b = __ldg(f + sa + x + 1) - mean;
                if (mode == 2) {
                    a *= a;
                    b *= b;
                    q4 = fmaf(a, a, fmaf(b, b, q4));
                }
            }
            v[n2] = make_float2(a, b);
        }
        dft_reg<L2, -1>(v);
#pragma unroll
        for (int k2 = 1; k2 < L2; ++k2) v[k2] = cmul(v[k2], __ldg(tw + 2 * n1 * k2));   // W_M^(n1 k2)
        __syncthreads();                              // the previous tile's rows are stored
#pragma unroll
        for (int k2 = 0; k2 < L2; ++k2) zx[(ra * L2 + k2) * ZP + n1] = v[k2];
        __syncthreads();
        // step B: NI items per thread, kept in registers until the exchange
        // buffer is free
        constexpr int NI = (NR * L2 + kTwoThreads - 1) / kTwoThreads;
        static_assert(NI <= 2, "at most two step-B items per thread");
        float2 zk[NI][L1];
#pragma unroll
        for (int i = 0; i < NI; ++i) {
            const int it = t + i * kTwoThreads;
            if (it < NR * L2) {
                const int rb = it / L2, k2 = it % L2;
#pragma unroll
                for (int m = 0; m < L1; ++m) zk[i][m] = zx[(rb * L2 + k2) * ZP + m];
                dft_reg<L1, -1>(zk[i]);
            }
        }
        __syncthreads();                              // the exchange buffer is free
#pragma unroll
        for (int i = 0; i < NI; ++i) {
            const int it = t + i * kTwoThreads;
            if (it < NR * L2) {
                const int rb = it / L2, k2 = it % L2;
#pragma unroll
                for (int k1 = 0; k1 < L1; ++k1) zx[rb * M + k2 + L2 * k1] = zk[i][k1];
            }
        }
        __syncthreads();
        for (int it = t; it < NR * XH; it += kTwoThreads) {
            const int rb = it / XH, k = it % XH;
            const size_t q = tile * NR + rb;
            if (q >= nrows) continue;
            const float2 a = zx[rb * M + (k == M ? 0 : k)];
            float2 b = zx[rb * M + (k == 0 ? 0 : M - k)];
            b.y = -b.y;                               // conj Z[M - k]
            const float2 e = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y + b.y));
            const float2 d = cmul(make_float2(0.5f * (a.x - b.x), 0.5f * (a.y - b.y)), __ldg(tw + k));
            out[q * XH + k] = make_float2(e.x + d.y, e.y - d.x);      // e - i d
        }
    }
    if (mode == 2) {
        double d = q4;
        for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
        if ((t & 31) == 0) part[t >> 5] = d;
        __syncthreads();
        if (t == 0) {
            double s4 = 0.0;
            for (int k = 0; k < kTwoThreads / 32; ++k) s4 += part[k];
            if (s4 != 0.0) atomicAdd(moments + 2, s4);
        }
    }
}

}  // namespace fftk
}  // namespace ttm
