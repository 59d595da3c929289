// Direct correlation on the 5th-generation tensor cores (implicit GEMM) for
// small templates (Sec. 2 cross-correlation, Sec. 3.2):
//
//   Corr_alpha(x) = sum_t f(x + o_t) T_alpha(t),   t over the mask voxels (taps),
//
// written as D[v, alpha] = sum_t A[v, t] B[t, alpha] with A the im2col matrix
// of a tile of 128 interior voxels (A[v, t] = f at voxel v shifted by tap t)
// and B the template components of every tap.  tcgen05.mma kind::f16: FP16
// operands, FP32 accumulation in tensor memory; M = 128 voxels, N = K padded
// to a multiple of 16 (48 for K = 35, 96 for K = 84), 16 taps per MMA.
//
// Conditioning for FP16: A holds (f - mean(f)) / std(f) (every component sums
// to zero over the mask, Sec. 3.2, so a constant shift of f changes no
// correlation) and B holds T / max|T|; the epilogue multiplies by
// std(f) max|T|.
//
// One persistent CTA of 256 threads per SM.  B (all taps, UMMA K-major
// core-matrix layout) and the taps' volume offsets stay in shared memory.  Per
// tile the CTA builds A 32 taps at a time into one of two buffers (thread
// t and t + 128 = voxel t, 16 taps each), and thread 0 issues two MMAs per
// buffer, committed to that buffer's mbarrier; a buffer is rebuilt only after
// its MMAs have completed.  Waits are bounded: on expiry the kernel records
// TTM_ERR_TIMEOUT, waits once more for its MMAs, frees its tensor memory and
// exits.
#include <cuda_fp16.h>

#include <cmath>

#include "ttm_internal.h"

namespace ttm {

namespace {

constexpr int kThreads = 256;
constexpr int kStageTaps = 32;                      // taps per A buffer (two MMAs)
constexpr uint32_t kABytes = 128 * kStageTaps * 2;  // 8 KB

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase) {
    return mbar_wait_bounded(bar, phase, kMbarWaitPolls);
}

__device__ __forceinline__ void tmem_ld8(uint32_t addr, uint32_t (&r)[8]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7])
        : "r"(addr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

struct DirectTcArgs {
    const float* f;
    float* corr;               // K x nvox
    size_t nvox;
    VoxBox box;                // interior voxels: the units of the GEMM's M dimension
    int X, Y;
    const uint4* btab;         // n_taps_pad x NP FP16 in the kernel's shared-memory layout
    const int* tap_dxyz;       // per tap: (dx + 64) | (dy + 64) << 8 | (dz + 64) << 16
    int n_taps_pad;            // multiple of kStageTaps
    int K;
    float t_scale;             // max |T| (B holds T / max |T|)
    const double* moments;     // sum f, sum f^2 over the volume
    int* status;
};

template <int NP>
__global__ void __launch_bounds__(kThreads, 1) direct_tc_kernel(DirectTcArgs a) {
    constexpr int kCols = NP <= 32 ? 32 : (NP <= 64 ? 64 : 128);   // TMEM columns
    // kind::f16 instruction descriptor: D FP32, A and B FP16, K-major, M = 128, N = NP
    constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(NP >> 3) << 17) | ((128u >> 4) << 24);
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ uint32_t tmem_base_s;
    __shared__ float stat_s[2];
    const int t = threadIdx.x;
    const int warp = t >> 5;
    const int ntp = a.n_taps_pad;
    const uint32_t b_bytes = (uint32_t)ntp * NP * 2;
    unsigned char* Bs = sm;
    unsigned char* As = sm + b_bytes;                                  // two buffers
    int* offs = reinterpret_cast<int*>(sm + b_bytes + 2 * kABytes);    // volume offset per tap

    {
        uint4* dst = reinterpret_cast<uint4*>(Bs);
        for (int e = t; e < (int)(b_bytes / 16); e += kThreads) dst[e] = __ldg(a.btab + e);
        for (int e = t; e < ntp; e += kThreads) {
            const int p = __ldg(a.tap_dxyz + e);
            const int dx = (p & 255) - 64, dy = ((p >> 8) & 255) - 64, dz = ((p >> 16) & 255) - 64;
            offs[e] = (dz * a.Y + dy) * a.X + dx;
        }
    }
    if (t == 0) {
        const double n = (double)a.nvox;
        const double mean = a.moments[0] / n;
        const double var = fmax(a.moments[1] / n - mean * mean, 0.0);
        const double sd = var > 0.0 ? sqrt(var) : 1.0;
        stat_s[0] = (float)mean;
        stat_s[1] = (float)(1.0 / sd);
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&bars[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&bars[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         smem_u32(&tmem_base_s)), "n"(kCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_base_s;
    const float mean = stat_s[0], inv_sd = stat_s[1];
    const float out_scale = a.t_scale / inv_sd;
    const uint32_t bar[2] = {smem_u32(&bars[0]), smem_u32(&bars[1])};
    const uint32_t a_base = smem_u32(As), b_base = smem_u32(Bs);
    uint32_t phase[2] = {0u, 0u};
    int pending[2] = {0, 0};           // MMA groups committed to bar[b] and not yet waited on
    bool ok = true;

    const int lane_t = t & 127;        // voxel of the tile = TMEM lane
    const int half = t >> 7;           // taps half * 16 .. + 15 of a stage; output columns
    const size_t units = a.box.count();
    const size_t ntiles = (units + 127) / 128;
    const int nstages = ntp / kStageTaps;
    for (size_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const size_t i = tile * 128 + lane_t;
        const bool in_range = i < units;
        const long long v = in_range ? (long long)a.box.voxel((uint32_t)i) : 0;
        for (int sidx = 0; sidx < nstages; ++sidx) {
            const int b = sidx & 1;
            // the buffer's previous MMAs must be done before it is rebuilt
            if (pending[b]) {
                const bool got = mbar_wait(bar[b], phase[b]);
                if (!__syncthreads_and(got)) { ok = false; break; }
                phase[b] ^= 1u;
                pending[b] = 0;
            }
            // 16 taps of voxel lane_t: two core-matrix rows (8 FP16 each)
            const int tap0 = sidx * kStageTaps + half * 16;
            float x[16];
#pragma unroll
            for (int e = 0; e < 16; ++e)
                x[e] = in_range ? __ldg(a.f + v + offs[tap0 + e]) : mean;
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                uint32_t w[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const __half2 h = __floats2half2_rn((x[8 * r + 2 * q] - mean) * inv_sd,
                                                        (x[8 * r + 2 * q + 1] - mean) * inv_sd);
                    w[q] = *reinterpret_cast<const uint32_t*>(&h);
                }
                const int kc = half * 2 + r;                      // core-matrix column (8 taps)
                *reinterpret_cast<uint4*>(As + (uint32_t)b * kABytes +
                                          ((kc * 16 + (lane_t >> 3)) * 8 + (lane_t & 7)) * 16) =
                    make_uint4(w[0], w[1], w[2], w[3]);
            }
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncthreads();
            if (t == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
                for (int s2 = 0; s2 < 2; ++s2) {
                    const uint64_t ad = smem_desc(a_base + (uint32_t)b * kABytes +
                                                      (uint32_t)(2 * s2) * 16 * 128,
                                                  16 * 128, 128);
                    const int kc0 = (sidx * kStageTaps) / 8 + 2 * s2;
                    const uint64_t bd = smem_desc(b_base + (uint32_t)kc0 * (NP / 8) * 128,
                                                  (NP / 8) * 128, 128);
                    const int acc = (sidx > 0 || s2 > 0) ? 1 : 0;
                    asm volatile(
                        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                        "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc) : "memory");
                }
                asm volatile(
                    "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                    ::"r"(bar[b]) : "memory");
            }
            pending[b] = 1;
        }
        if (!ok) break;
        // the last MMAs of the tile: both buffers' commits
        bool got = true;
        for (int b = 0; b < 2; ++b)
            if (pending[b] && mbar_wait(bar[b], phase[b])) {
                phase[b] ^= 1u;
                pending[b] = 0;
            } else if (pending[b]) {
                got = false;
            }
        if (!__syncthreads_and(got)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        // epilogue: this thread's voxel, columns half * NP/2 .. ; lanes of warp w: 32 (w % 4)
        const uint32_t lane_addr = tmem + ((uint32_t)((warp & 3) * 32) << 16);
#pragma unroll
        for (int c0 = 0; c0 < NP / 2; c0 += 8) {
            uint32_t r[8];
            tmem_ld8(lane_addr + (uint32_t)(half * (NP / 2) + c0), r);
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int k = half * (NP / 2) + c0 + e;
                if (in_range && k < a.K) a.corr[(size_t)k * a.nvox + v] = __uint_as_float(r[e]) * out_scale;
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();     // TMEM and the A buffers are reused by the next tile
    }
    if (!ok) {
        if (t == 0) atomicExch(a.status, TTM_ERR_TIMEOUT);
        // MMAs still in flight complete before the tensor memory is released
        for (int b = 0; b < 2; ++b)
            if (pending[b]) mbar_wait(bar[b], phase[b]);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "n"(kCols)
                     : "memory");
}

}  // namespace

int direct_tc_columns(int K) { return ((K + 15) / 16) * 16; }

size_t direct_tc_smem(int K, int n_taps) {
    const int np = direct_tc_columns(K);
    const int ntp = ((n_taps + kStageTaps - 1) / kStageTaps) * kStageTaps;
    return (size_t)ntp * np * 2 + 2 * kABytes + (size_t)ntp * 4;
}

bool direct_tc_supported(int K, int n_taps) {
    const int np = direct_tc_columns(K);
    return (np == 48 || np == 96) && direct_tc_smem(K, n_taps) <= 200 * 1024;
}

// FP16 table of T / max|T| in the kernel's layout: element (t, n) of the
// n_taps_pad x NP matrix at core matrix (t / 8, n / 8), row n % 8, column t % 8,
// core matrices ordered tap-block-major; zero for padded taps and columns.
void build_direct_tc_table(const std::vector<float>& taps, int n_taps, int K,
                           std::vector<uint16_t>& out, float* t_scale) {
    const int np = direct_tc_columns(K);
    const int ntp = ((n_taps + kStageTaps - 1) / kStageTaps) * kStageTaps;
    float mx = 0.f;
    for (float v : taps) mx = std::fmax(mx, std::fabs(v));
    if (!(mx > 0.f)) mx = 1.f;
    *t_scale = mx;
    out.assign((size_t)ntp * np, 0);
    for (int t = 0; t < n_taps; ++t)
        for (int n = 0; n < K; ++n) {
            const __half h = __float2half_rn(taps[(size_t)t * K + n] / mx);
            const size_t idx = (((size_t)(t / 8) * (np / 8) + n / 8) * 8 + n % 8) * 8 + t % 8;
            out[idx] = __half_as_ushort(h);
        }
}

ttm_status launch_direct_tc(const float* f, int X, int Y, int Z, const TemplateData& T, int K,
                            const double* d_moments, float* corr, int* status, cudaStream_t st,
                            long long* cnt) {
    if (!T.d_tc_tab || !direct_tc_supported(K, T.n_taps)) return TTM_ERR_UNSUPPORTED;
    const VoxBox box = interior_box(X, Y, Z, T.desc.s);
    const size_t units = box.count();
    if (units == 0) return TTM_OK;
    if (units > 0xFFFFFFFFull) return TTM_ERR_UNSUPPORTED;
    DirectTcArgs a;
    a.f = f; a.corr = corr; a.nvox = (size_t)X * Y * Z; a.box = box; a.X = X; a.Y = Y;
    a.btab = reinterpret_cast<const uint4*>(T.d_tc_tab);
    a.tap_dxyz = T.d_tap_dxyz;
    a.n_taps_pad = ((T.n_taps + kStageTaps - 1) / kStageTaps) * kStageTaps;
    a.K = K;
    a.t_scale = T.tc_scale;
    a.moments = d_moments;
    a.status = status;
    const size_t smem = direct_tc_smem(K, T.n_taps);
    int dev = 0, sms = 0;
    TTM_CUDA_TRY(cudaGetDevice(&dev));
    TTM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const size_t ntiles = (units + 127) / 128;
    const unsigned grid = (unsigned)(ntiles < (size_t)sms ? ntiles : (size_t)sms);
    if (direct_tc_columns(K) == 48) {
        TTM_CUDA_TRY(cudaFuncSetAttribute(direct_tc_kernel<48>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        direct_tc_kernel<48><<<grid, kThreads, smem, st>>>(a);
    } else {
        TTM_CUDA_TRY(cudaFuncSetAttribute(direct_tc_kernel<96>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        direct_tc_kernel<96><<<grid, kThreads, smem, st>>>(a);
    }
    return after_launch(cnt);
}

}  // namespace ttm
