// Tensor-core grid search of the per-voxel rotation for tensor orders 4 and 6
// (Sec. 3.3-3.4 of the paper: the rotation is the maximiser of
// phi(Q) = C_n(x) . Q^(n) on the unit sphere).
//
// phi at the 2048 grid points of every voxel is one dense contraction,
//   Phi[v, g] = sum_alpha Cn[v, alpha] M[g, alpha],  M[g, alpha] = mu_alpha q_g^alpha,
// with Cn = C / ||C||_F (a positive per-voxel scale changes no ranking).  It runs
// on the 5th-generation tensor cores: tcgen05.mma kind::f16 (FP16 operands,
// FP32 accumulation) with M = 128 voxels, N = 256 grid points and K = KP (the
// K components, a constant column that adds +1 to phi, zero padding to a
// multiple of 16: 48 for order 4, 96 for order 6), D in tensor memory.
//
// One persistent CTA per SM of 256 threads; a tile is 128 consecutive voxels
// of the interior box (threads t and t + 128 = voxel t of the tile = TMEM lane
// t; each reads 128 of a chunk's 256 columns).  (512 threads in four column
// groups measured no faster and leave less room for the refinement kernel
// that runs beside the search.)  The FP16
// grid table (2048 x KP, K-major core-matrix layout without swizzle, stored
// chunk by chunk of 256 points) is either copied into shared memory once per
// CTA (order 4: 192 KB) or streamed chunk by chunk with bulk copies into two
// shared-memory buffers (order 6: 48 KB per chunk, from L2).  Per tile: every
// thread writes its voxel's normalised components as one FP16 row of A; thread
// 0 issues the MMAs of one 256-point chunk into one half of a 512-column TMEM
// accumulator while all threads read the other half (the previous chunk) with
// tcgen05.ld and keep, per grid region of 16 consecutive points, the best
// point, and the 8 best regions.  Waits on the mbarriers are bounded: on
// expiry the kernel records TTM_ERR_TIMEOUT, waits once more for its MMAs and
// copies in flight, frees its TMEM and exits.
#include <climits>

#include <cuda_fp16.h>

#include "k_rotation.cuh"

namespace ttm {

namespace {

constexpr int kThreads = 256;    // warps w and w + 4 read the same TMEM lanes
constexpr int kGroups = kThreads / 128;    // column groups of a chunk (one per 4 warps)
constexpr int kChunkN = 256;         // grid points per MMA
constexpr uint32_t kMergeBytes = (kGroups - 1) * 128 * 8 * 4;  // top-8 keys of groups 1..

// Shapes for K tensor components and G grid points (1024 or 2048): padded
// K, shared-memory sizes, and whether the grid table is resident or streamed.
template <int K, int G>
struct TcShape {
    static constexpr int kChunks = G / kChunkN;
    static constexpr int KP = ((K + 1 + 15) / 16) * 16;          // + constant column
    static constexpr int KC = KP / 8;                            // core-matrix columns along K
    static constexpr uint32_t ABytes = (uint32_t)KC * 16 * 128;
    static constexpr uint32_t ChunkBytes = (uint32_t)KC * (kChunkN / 8) * 128;
    static constexpr bool Stream = (uint64_t)ChunkBytes * kChunks > 200u * 1024u;
    static constexpr uint32_t BBytes = Stream ? 2 * ChunkBytes : ChunkBytes * kChunks;
    static constexpr uint32_t Smem = BBytes + ABytes + kMergeBytes;
    static_assert(Smem <= 227u * 1024u, "shared memory");
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: K-major, no swizzle; lbo = byte distance of
// core matrices adjacent along K, sbo = along M/N
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// kind::f16 instruction descriptor: D FP32, A and B FP16, both K-major, M = 128, N = 256
constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(kChunkN >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase) {
    return mbar_wait_bounded(bar, phase, kMbarWaitPolls);
}

// MMAs of one 256-point chunk whose B block (KP/8 x 32 core matrices, K-block
// major) starts at b_chunk; A is 128 x KP (KP/8 x 16 core matrices)
template <int KP>
__device__ __forceinline__ void issue_chunk(uint32_t tmem_d, uint32_t a_base, uint32_t b_chunk,
                                           uint32_t bar) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
    for (int s = 0; s < KP / 16; ++s) {
        const uint64_t ad = smem_desc(a_base + (uint32_t)(2 * s) * 16 * 128, 16 * 128, 128);
        const uint64_t bd = smem_desc(b_chunk + (uint32_t)(2 * s) * (kChunkN / 8) * 128,
                                      (kChunkN / 8) * 128, 128);
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
            "l"(ad), "l"(bd), "r"(kIdesc), "r"(s) : "memory");
    }
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
        : "memory");
}

// (c ? a : b) bit by bit: one LOP3 whose b operand is an immediate
template <int B>
__device__ __forceinline__ int select_bits(int a, int c) {
    int d;
    asm("lop3.b32 %0, %1, %2, %3, 0xE4;" : "=r"(d) : "r"(a), "n"(B), "r"(c));
    return d;
}

// key[j] = (r[j] & ~2047) | (15 - j % 16) for j = J..M-1 (compile-time j)
template <int J, int M>
__device__ __forceinline__ void pack_keys(int (&key)[M], const uint32_t (&r)[M], int mask) {
    if constexpr (J < M) {
        key[J] = select_bits<15 - (J & 15)>((int)r[J], mask);
        pack_keys<J + 1, M>(key, r, mask);
    }
}

// compare-exchange for a descending order
__device__ __forceinline__ void cx(int& hi, int& lo) {
    const int a = max(hi, lo);
    lo = min(hi, lo);
    hi = a;
}

// top (8, descending) := the 8 largest of top and n (4, descending): the
// element-wise max of top and reversed n is bitonic, then three half-cleaner
// stages sort it
__device__ __forceinline__ void merge4(int (&top)[8], int (&n)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) top[4 + i] = max(top[4 + i], n[3 - i]);
#pragma unroll
    for (int i = 0; i < 4; ++i) cx(top[i], top[i + 4]);
#pragma unroll
    for (int i = 0; i < 8; i += 4) { cx(top[i], top[i + 2]); cx(top[i + 1], top[i + 3]); }
#pragma unroll
    for (int i = 0; i < 8; i += 2) cx(top[i], top[i + 1]);
}

// the same for two lists of 8
__device__ __forceinline__ void merge8(int (&top)[8], const int (&n)[8]) {
#pragma unroll
    for (int i = 0; i < 8; ++i) top[i] = max(top[i], n[7 - i]);
#pragma unroll
    for (int i = 0; i < 4; ++i) cx(top[i], top[i + 4]);
#pragma unroll
    for (int i = 0; i < 8; i += 4) { cx(top[i], top[i + 2]); cx(top[i + 1], top[i + 3]); }
#pragma unroll
    for (int i = 0; i < 8; i += 2) cx(top[i], top[i + 1]);
}

// one thread: arm the barrier for `bytes` and start a bulk copy global -> shared
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
        ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// 32 TMEM columns of this warp's 32 lanes into r; the copy completes at
// tmem_wait32, which names r as modified so nothing reads r before it
__device__ __forceinline__ void tmem_ld32(uint32_t addr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
          "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
          "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]),
          "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
          "=r"(r[30]), "=r"(r[31])
        : "r"(addr)
        : "memory");
}

__device__ __forceinline__ void tmem_wait32(uint32_t (&r)[32]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;\n"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                   "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                   "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]),
                   "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]),
                   "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]),
                   "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}

// 32 columns = 2 regions of 16 -> their best keys n0, n1.  phi + 1 >= 0
// (|phi| <= 1 for unit-norm C), so its float bits order like the values; the
// low 11 bits become the code 2047 - g of the grid index g: first only the
// position in the region (15 - j, one LOP3 per value), the region part (low0 =
// 2047 - grid index of column 0) is added to each region's maximum
__device__ __forceinline__ void region_max32(const uint32_t (&r)[32], int low0, int& n0, int& n1) {
    int key[32];
    pack_keys<0, 32>(key, r, ~2047);
    int nk[2];
#pragma unroll
    for (int q2 = 0; q2 < 2; ++q2) {
        // three-input integer maxima, 16 -> 6 -> 2 -> 1
        const int* k16 = key + 16 * q2;
        const int m0 = __vimax3_s32(k16[0], k16[1], k16[2]);
        const int m1 = __vimax3_s32(k16[3], k16[4], k16[5]);
        const int m2 = __vimax3_s32(k16[6], k16[7], k16[8]);
        const int m3 = __vimax3_s32(k16[9], k16[10], k16[11]);
        const int m4 = __vimax3_s32(k16[12], k16[13], k16[14]);
        const int a0 = __vimax3_s32(m0, m1, m2);
        const int a1 = __vimax3_s32(m3, m4, k16[15]);
        nk[q2] = max(a0, a1) + (low0 - 16 * q2 - 15);
    }
    n0 = nk[0];
    n1 = nk[1];
}

// Half G (0 or 1) of the KP columns of a voxel's A row: columns
// G KP/2 .. (G+1) KP/2 - 1 of [w Corr_0 .. w Corr_{K-1}, 1, 0 ...].
// The raw components of half G of a voxel's A row (all loads issued at
// once, used a tile later: the next tile's loads are in flight while this
// tile's epilogue runs)
template <int N, int G, int KP, typename CT>
__device__ __forceinline__ void a_half_fetch(const CT* __restrict__ corr, size_t nvox, size_t v,
                                             bool in_range, CT (&raw)[KP / 2]) {
    constexpr int K = n_comp(N);
    constexpr int KH = KP / 2;
#pragma unroll
    for (int j = 0; j < KH; ++j) {
        constexpr int k0 = G * KH;
        raw[j] = (in_range && k0 + j < K) ? __ldg(corr + (size_t)(k0 + j) * nvox + v) : CT(0.f);
    }
}

// C = w * the fetched components (zero beyond K); returns the half of
// sum mu_k C_k^2 they carry
template <int N, int G, int KP, typename CT>
__device__ __forceinline__ float a_half_finish(const CT (&raw)[KP / 2], float wv,
                                               float (&C)[KP / 2]) {
    constexpr int K = n_comp(N);
    constexpr int KH = KP / 2;
    constexpr Sym<N> S{};
    float ss = 0.f;
#pragma unroll
    for (int j = 0; j < KH; ++j) {
        constexpr int k0 = G * KH;
        C[j] = 0.f;
        if (k0 + j < K) {
            C[j] = (float)raw[j] * wv;
            ss = fmaf((float)S.mu[k0 + j], C[j] * C[j], ss);
        }
    }
    return ss;
}

// The FP16 columns of half G of the row, normalised by 1/score, into the
// K-major core-matrix layout of A (column K is the constant 1 that adds +1
// to every phi, see below)
template <int N, int G, int KP>
__device__ __forceinline__ void a_half_store(const float (&C)[KP / 2], float inv,
                                             unsigned char* As, int lane_t) {
    constexpr int K = n_comp(N);
    constexpr int KH = KP / 2;
#pragma unroll
    for (int kc = 0; kc < KH / 8; ++kc) {
        __half h[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int j = kc * 8 + e;
            const int k = G * KH + j;
            h[e] = __float2half_rn(k < K ? C[j] * inv : (k == K ? 1.f : 0.f));
        }
        uint4 pk;
        pk.x = (uint32_t)__half_as_ushort(h[0]) | ((uint32_t)__half_as_ushort(h[1]) << 16);
        pk.y = (uint32_t)__half_as_ushort(h[2]) | ((uint32_t)__half_as_ushort(h[3]) << 16);
        pk.z = (uint32_t)__half_as_ushort(h[4]) | ((uint32_t)__half_as_ushort(h[5]) << 16);
        pk.w = (uint32_t)__half_as_ushort(h[6]) | ((uint32_t)__half_as_ushort(h[7]) << 16);
        const int kcg = G * (KH / 8) + kc;
        *reinterpret_cast<uint4*>(As + ((kcg * 16 + (lane_t >> 3)) * 8 + (lane_t & 7)) * 16) = pk;
    }
}

// 168 registers: the next tile's components stay in registers through the
// epilogue, and one CTA of this kernel (256 threads) still leaves room for a
// CTA of the refinement kernel (128 threads x 168) on the same SM
template <typename CT, int N, int G>
__global__ void __maxnreg__(168) search_tc_kernel(const __grid_constant__ rot::SearchArgs a,
                                                                const uint4* __restrict__ gtab,
                                                                int* status) {
    using Sh = TcShape<n_comp(N), G>;
    constexpr int kChunks = Sh::kChunks;
    constexpr int K = n_comp(N);
    constexpr int KP = Sh::KP;
    constexpr bool kStream = Sh::Stream;
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t bars[2];     // MMA completion, one per TMEM half
    __shared__ __align__(8) uint64_t lbars[2];    // grid-chunk copies (streamed table)
    __shared__ __align__(8) uint64_t ebars[2];    // TMEM half read by every warp (count: warps)
    __shared__ uint32_t tmem_base_s;
    constexpr Sym<N> S{};
    const int t = threadIdx.x;
    const int warp = t >> 5;
    unsigned char* Bs = sm;
    unsigned char* As = sm + Sh::BBytes;
    int* merge = reinterpret_cast<int*>(sm + Sh::BBytes + Sh::ABytes);   // [8][128]

    if constexpr (!kStream) {   // grid table, once per CTA
        uint4* dst = reinterpret_cast<uint4*>(Bs);
        for (int e = t; e < (int)(Sh::BBytes / 16); e += kThreads) dst[e] = __ldg(gtab + e);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;\n" ::"r"(
                         smem_u32(&tmem_base_s)) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (t == 0) {
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&bars[b])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&lbars[b])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&ebars[b])),
                         "n"(kThreads / 32) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_base_s;
    const uint32_t a_base = smem_u32(As), b_base = smem_u32(Bs);
    const uint32_t bar0 = smem_u32(&bars[0]), bar1 = smem_u32(&bars[1]);
    const uint32_t lbar0 = smem_u32(&lbars[0]), lbar1 = smem_u32(&lbars[1]);
    // barrier phases and flags as bit masks (bit h for TMEM half / buffer h),
    // so that they stay in registers
    uint32_t phase = 0u;             // MMA barriers
    uint32_t lphase = 0u;            // thread 0: copy barriers
    const uint32_t ebar0 = smem_u32(&ebars[0]), ebar1 = smem_u32(&ebars[1]);
    uint32_t ephase = 0u;            // thread 0: TMEM-half barriers
    uint32_t half_used = 0u;         // thread 0: an epilogue of this half is still to be waited for
    uint32_t mma_pending = 0u;       // thread 0: MMAs committed to bars[h] and not yet seen done
    uint32_t loads_pending = 0u;     // thread 0: copies issued and not yet waited on
    bool ok = true;

    // tiles of the launch (with a unit list, one problem: the listed units)
    size_t ntiles = a.b.ntiles;
    if (a.list.count) {
        const uint32_t uend = rot::list_end(a.list, a.b.seg[0].u1);
        ntiles = ((uend > a.b.seg[0].u0 ? uend - a.b.seg[0].u0 : 0) + 127) / 128;
    }
    const unsigned char* gsrc = reinterpret_cast<const unsigned char*>(gtab);
    // streamed table: chunk q (counted over the whole CTA) goes to buffer q & 1;
    // the copy of chunk q + 2 starts once the MMAs of chunk q have completed
    if (kStream && t == 0) {
        for (int q = 0; q < 2; ++q) {
            bulk_load(b_base + (uint32_t)q * Sh::ChunkBytes, gsrc + (size_t)q * Sh::ChunkBytes,
                      Sh::ChunkBytes, ((q) ? lbar1 : lbar0));
            loads_pending |= 1u << q;
        }
    }
    // thread 0: wait until every warp has read the TMEM half (its previous
    // chunk), wait for the copy of chunk q (streamed table), issue the MMAs
    auto issue = [&](uint32_t tmem_d, int chunk, long q, uint32_t bar) {
        const int hh = chunk & 1;
        if ((half_used >> hh) & 1u) {
            if (!mbar_wait(((hh) ? ebar1 : ebar0), (ephase >> hh) & 1u)) return;   // no MMA: the MMA wait expires
            ephase ^= 1u << hh;
            half_used &= ~(1u << hh);
        }
        uint32_t b_chunk;
        if constexpr (kStream) {
            const int buf = (int)(q & 1);
            if (!mbar_wait(((buf) ? lbar1 : lbar0), (lphase >> buf) & 1u)) return;   // no MMA: the MMA wait expires
            lphase ^= 1u << buf;
            loads_pending &= ~(1u << buf);
            b_chunk = b_base + (uint32_t)buf * Sh::ChunkBytes;
        } else {
            b_chunk = b_base + (uint32_t)chunk * Sh::ChunkBytes;
        }
        issue_chunk<KP>(tmem_d, a_base, b_chunk, bar);
        half_used |= 1u << hh;
        mma_pending |= 1u << hh;
    };

    const int lane_t = t & 127;            // TMEM lane = voxel of the tile
    const int grp = t >> 7;                // column group: columns grp * 256 / kGroups ...
    long qbase = 0;                        // chunks issued by this CTA before this tile
    // the next tile's problem (segments in tile order), unit, voxel, w and
    // raw components: threads t and t + 128 share voxel t of the tile, each
    // fetching half of the KP columns
    constexpr int KH = KP / 2;
    int sidx = 0;
    size_t i_n = 0, v_n = 0;
    bool in_n = false;
    float wv_n = 0.f;
    CT raw[KH];
    auto fetch = [&](size_t tl) {
        sidx = rot::seg_of(a.b, (uint32_t)tl, sidx);
        const RotSeg& sg = a.b.seg[sidx];
        i_n = sg.u0 + (tl - sg.tile0) * 128 + lane_t;
        in_n = i_n < rot::list_end(a.list, sg.u1);
        v_n = in_n ? rot::unit_voxel(sg.box, a.list, (uint32_t)i_n) : 0;
        wv_n = in_n ? __ldg(sg.w + v_n) : 0.f;
        const CT* corr = reinterpret_cast<const CT*>(sg.corr);
        if (grp == 0) a_half_fetch<N, 0, KP>(corr, sg.nvox, v_n, in_n, raw);
        else a_half_fetch<N, 1, KP>(corr, sg.nvox, v_n, in_n, raw);
    };
    if (blockIdx.x < ntiles) fetch(blockIdx.x);
    for (size_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, qbase += kChunks) {
        const bool more_tiles = tile + gridDim.x < ntiles;
        const int cur = sidx;
        const size_t i = i_n, v = v_n;
        const bool in_range = in_n;
        // components, score, normalised FP16 row of A; the two halves of the
        // sum of squares meet in the merge buffer (free until the tile's end)
        float score = 0.f;
        {
            float C[KH];
            const float part = grp == 0 ? a_half_finish<N, 0, KP>(raw, wv_n, C)
                                        : a_half_finish<N, 1, KP>(raw, wv_n, C);
            float* ssx = reinterpret_cast<float*>(merge);
            if (grp == 1) ssx[lane_t] = part;
            __syncthreads();
            // the two halves in the order of rot::score_split (KP / 2 == the split)
            static_assert(KH == rot::score_split<N>(), "score halves");
            const float ss = grp == 0 ? part + ssx[lane_t] : 0.f;
            score = sqrtf(ss);                      // group 0 keeps the score
            if (grp == 0) ssx[128 + lane_t] = score;
            __syncthreads();
            const float sc = grp == 0 ? score : ssx[128 + lane_t];
            const float inv = sc > 0.f ? 1.f / sc : 0.f;
            if (grp == 0) a_half_store<N, 0, KP>(C, inv, As, lane_t);
            else a_half_store<N, 1, KP>(C, inv, As, lane_t);
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();
        if (t == 0) issue(tmem, 0, qbase, bar0);
        if (more_tiles) fetch(tile + gridDim.x);      // lands during the epilogue

        // packed keys: the float bits of phi + 1 with the low 11 bits replaced
        // by (2047 - grid index): one integer max gives the best point of a
        // region (ties: lower index) at 2.4e-4 resolution of the normalised
        // phi; top holds the 8 best region keys, descending
        int top[rot::kMaxCand];
#pragma unroll
        for (int k = 0; k < rot::kMaxCand; ++k) top[k] = INT_MIN;
        // MMAs of chunk cc done (bounded wait); with a streamed table its
        // buffer then takes chunk cc + 2
        auto wait_chunk = [&](int cc) -> bool {
            const int hh = cc & 1;
            if (!mbar_wait(hh ? bar1 : bar0, (phase >> hh) & 1u)) return false;
            phase ^= 1u << hh;
            if (t == 0) mma_pending &= ~(1u << hh);
            if (kStream && t == 0 && (cc + 2 < kChunks || more_tiles)) {
                const int buf = (int)((qbase + cc) & 1);
                const int nxt = (cc + 2) % kChunks;
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                bulk_load(b_base + (uint32_t)buf * Sh::ChunkBytes,
                          gsrc + (size_t)nxt * Sh::ChunkBytes, Sh::ChunkBytes, ((buf) ? lbar1 : lbar0));
                loads_pending |= 1u << buf;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            return true;
        };
        // this warp's 32 lanes, its column group, TMEM half hh
        auto cols = [&](int hh) {
            return tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)hh * kChunkN +
                   (uint32_t)grp * (kChunkN / kGroups);
        };
        // each chunk is read as four loads of 32 columns, the next one in
        // flight while the previous one is reduced (a load of the next chunk
        // during the last one measured faster alone but needs ~160 registers,
        // which leaves no room for the refinement kernel running beside this
        // one); four region maxima at a time go into the top-8 list
        static_assert(kChunkN / kGroups == 128, "four 32-column loads per chunk");
        uint32_t ra[32], rb[32];
#pragma unroll 1
        for (int c = 0; c < kChunks && ok; ++c) {
            const int h = c & 1;
            if (c + 1 < kChunks && t == 0)
                issue(tmem + (uint32_t)((c + 1) & 1) * kChunkN, c + 1, qbase + c + 1,
                      ((c + 1) & 1) ? bar1 : bar0);
            if (!wait_chunk(c)) { ok = false; break; }
            tmem_ld32(cols(h), ra);
            const int low0 = 2047 - (c * kChunkN + grp * (kChunkN / kGroups));
            int nk[4];
            tmem_wait32(ra);
            tmem_ld32(cols(h) + 32, rb);
            region_max32(ra, low0, nk[0], nk[1]);
            tmem_wait32(rb);
            tmem_ld32(cols(h) + 64, ra);
            region_max32(rb, low0 - 32, nk[2], nk[3]);
            cx(nk[0], nk[1]); cx(nk[2], nk[3]); cx(nk[0], nk[2]); cx(nk[1], nk[3]); cx(nk[1], nk[2]);
            merge4(top, nk);
            tmem_wait32(ra);
            tmem_ld32(cols(h) + 96, rb);
            region_max32(ra, low0 - 64, nk[0], nk[1]);
            tmem_wait32(rb);
            // no block barrier per chunk: warps move on independently; this
            // warp has read half h, so chunk c + 2 may overwrite it
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncwarp();
            if ((t & 31) == 0)
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(((h) ? ebar1 : ebar0)) : "memory");
            region_max32(rb, low0 - 96, nk[2], nk[3]);
            cx(nk[0], nk[1]); cx(nk[2], nk[3]); cx(nk[0], nk[2]); cx(nk[1], nk[3]); cx(nk[1], nk[2]);
            merge4(top, nk);
        }
        if (!__syncthreads_and(ok)) {
            ok = false;
            if (t == 0) {
                atomicExch(status, TTM_ERR_TIMEOUT);
                // MMAs still in flight finish before the tensor memory is released
                for (int hh = 0; hh < 2; ++hh)
                    if ((mma_pending >> hh) & 1u) mbar_wait(hh ? bar1 : bar0, (phase >> hh) & 1u);
            }
            break;
        }
        // merge the column groups' lists into group 0's
        if (grp > 0) {
#pragma unroll
            for (int k = 0; k < rot::kMaxCand; ++k) merge[((grp - 1) * 8 + k) * 128 + lane_t] = top[k];
        }
        __syncthreads();
        if (grp == 0) {
#pragma unroll 1
            for (int g2 = 1; g2 < kGroups; ++g2) {
                int other[rot::kMaxCand];
#pragma unroll
                for (int k = 0; k < rot::kMaxCand; ++k) other[k] = merge[((g2 - 1) * 8 + k) * 128 + lane_t];
                merge8(top, other);
            }
            int ti[rot::kMaxCand];
#pragma unroll
            for (int k = 0; k < rot::kMaxCand; ++k) ti[k] = top[k] == INT_MIN ? 0xFFFF : 2047 - (top[k] & 2047);
            if (in_range) {
                const RotSeg& sg = a.b.seg[cur];
                sg.score[v] = score;
                rot::store_candidates(sg.cand, i, ti, score > 0.f);
            }
        }
        __syncthreads();     // merge buffer and A are reused by the next tile
    }
    // copies still in flight (only after an expired wait) land before exit
    if (kStream && t == 0) {
        for (int b = 0; b < 2; ++b)
            if ((loads_pending >> b) & 1u) mbar_wait(((b) ? lbar1 : lbar0), (lphase >> b) & 1u);
    }
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;\n" ::"r"(tmem) : "memory");
}

}  // namespace

template <typename CT, int N, int G>
static ttm_status launch_tc_t(const rot::SearchArgs& s, const uint16_t* grid_fp16, int* status,
                              cudaStream_t st, long long* cnt) {
    constexpr uint32_t smem = TcShape<n_comp(N), G>::Smem;
    TTM_CUDA_TRY(cudaFuncSetAttribute(search_tc_kernel<CT, N, G>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0, sms = 0;
    TTM_CUDA_TRY(cudaGetDevice(&dev));
    TTM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const size_t ntiles = s.b.ntiles;
    if (ntiles == 0) return TTM_OK;
    const unsigned grid = (unsigned)(ntiles < (size_t)sms ? ntiles : (size_t)sms);
    search_tc_kernel<CT, N, G><<<grid, kThreads, smem, st>>>(
        s, reinterpret_cast<const uint4*>(grid_fp16), status);
    return after_launch(cnt);
}

// grids of 2048 points in 128 regions, or 1024 points in 64 regions, of 16
bool search_tc_supported(int n_order, int n_grid, int n_cells) {
    return (n_order == 4 || n_order == 6) && (n_grid == 2048 || n_grid == 1024) &&
           n_cells == n_grid / 16;
}

ttm_status launch_search_tc(int n_order, const rot::SearchArgs& s, const uint16_t* grid_fp16,
                            int* status, bool bf16, cudaStream_t st, long long* cnt) {
    if ((s.n_grid != 2048 && s.n_grid != 1024) || !grid_fp16) return TTM_ERR_UNSUPPORTED;
    const bool g1 = s.n_grid == 1024;
    if (n_order == 4) {
        if (g1) return bf16 ? launch_tc_t<__nv_bfloat16, 4, 1024>(s, grid_fp16, status, st, cnt)
                            : launch_tc_t<float, 4, 1024>(s, grid_fp16, status, st, cnt);
        return bf16 ? launch_tc_t<__nv_bfloat16, 4, 2048>(s, grid_fp16, status, st, cnt)
                    : launch_tc_t<float, 4, 2048>(s, grid_fp16, status, st, cnt);
    }
    if (n_order == 6) {
        if (g1) return bf16 ? launch_tc_t<__nv_bfloat16, 6, 1024>(s, grid_fp16, status, st, cnt)
                            : launch_tc_t<float, 6, 1024>(s, grid_fp16, status, st, cnt);
        return bf16 ? launch_tc_t<__nv_bfloat16, 6, 2048>(s, grid_fp16, status, st, cnt)
                    : launch_tc_t<float, 6, 2048>(s, grid_fp16, status, st, cnt);
    }
    return TTM_ERR_UNSUPPORTED;
}

// FP16 grid table in the kernel's shared-memory layout, chunk by chunk of 256
// points: element (g, k) of the 2048 x KP matrix [mu_k q_g^k | 1 | 0...] at
// chunk g / 256, core matrix (k / 8, (g % 256) / 8), row g % 8, column k % 8,
// core matrices ordered k-block-major within the chunk.
void build_grid_fp16(const float* m_rows, int K, int K4, int n_grid, std::vector<uint16_t>& out) {
    const int KP = ((K + 1 + 15) / 16) * 16;
    out.assign((size_t)n_grid * KP, 0);
    for (int g = 0; g < n_grid; ++g)
        for (int k = 0; k < KP; ++k) {
            // column K holds the constant 1 paired with A's constant column,
            // adding +1 to every phi
            float v = k < K ? m_rows[(size_t)g * K4 + k] : (k == K ? 1.f : 0.f);
            __half h = __float2half_rn(v);
            const int c = g / kChunkN, gl = g % kChunkN;
            const size_t idx = (size_t)c * kChunkN * KP +
                               ((((size_t)(k / 8) * (kChunkN / 8) + gl / 8) * 8 + gl % 8) * 8 + k % 8);
            out[idx] = __half_as_ushort(h);
        }
}

}  // namespace ttm
