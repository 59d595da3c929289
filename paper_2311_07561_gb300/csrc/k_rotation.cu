// Dispatch of the per-voxel score and rotation kernel by tensor order.
#include "k_rotation.cuh"

namespace ttm {

int rotation_row_stride(int n_order) { return (n_comp(n_order) + 3) & ~3; }

static void fill_args(const RotBatch& b, const RotGrid& g, rot::SearchArgs& sa,
                      rot::PolishArgs& pa, const UnitList& list) {
    sa.b = b; pa.b = b;
    sa.list = list; pa.list = list;
    sa.gm = g.d_m; sa.cell_end = g.d_cell_end; sa.n_grid = g.n_grid;
    pa.gq = g.d_q; pa.n_cand = g.n_cand; pa.newton = g.newton; pa.n_refine = g.n_refine;
}

// a batch's units lie in their problems' interiors; unit lists serve one problem
static bool batch_ok(const RotBatch& b, const UnitList& list) {
    if (b.n < 1 || b.n > kMaxRotSegs || (list.idx && b.n != 1)) return false;
    for (int k = 0; k < b.n; ++k) {
        const RotSeg& s = b.seg[k];
        if (s.box.count() > 0xFFFFFFFFull || (!list.idx && s.u1 > s.box.count()) || s.u1 < s.u0)
            return false;
    }
    return true;
}

RotBatch one_problem_batch(const void* corr, const float* w, size_t nvox, const VoxBox& box,
                           uint32_t u0, uint32_t u1, uint16_t* cand, float* score, float* quat,
                           float* lambda, float* comp_out) {
    RotSeg s;
    s.corr = corr; s.w = w; s.nvox = nvox; s.box = box; s.u0 = u0; s.u1 = u1 > u0 ? u1 : u0;
    s.cand = cand; s.score = score; s.quat = quat; s.lambda = lambda; s.comp_out = comp_out;
    RotBatch b;
    b.add(s);
    return b;
}

ttm_status launch_rotation_search(int n_order, const RotBatch& b, bool bf16, const RotGrid& g,
                                  int* status, cudaStream_t st, long long* cnt,
                                  const UnitList& list) {
    if (!batch_ok(b, list)) return TTM_ERR_UNSUPPORTED;
    if (b.ntiles == 0) return TTM_OK;
    rot::SearchArgs sa;
    rot::PolishArgs pa;
    fill_args(b, g, sa, pa, list);
    if (g.d_gtab && search_tc_supported(n_order, g.n_grid, g.n_cells))
        return launch_search_tc(n_order, sa, g.d_gtab, status, bf16, st, cnt);
    switch (n_order) {
        case 2: return launch_rotation_n<2>(sa, pa, false, true, bf16, st, cnt);
        case 4: return launch_rotation_n<4>(sa, pa, false, true, bf16, st, cnt);
        case 6: return launch_rotation_n<6>(sa, pa, false, true, bf16, st, cnt);
        case 8: return launch_rotation_n<8>(sa, pa, false, true, bf16, st, cnt);
        default: return TTM_ERR_UNSUPPORTED;
    }
}

ttm_status launch_rotation_polish(int n_order, const RotBatch& b, bool bf16, const RotGrid& g,
                                  cudaStream_t st, long long* cnt, const UnitList& list) {
    if (!batch_ok(b, list)) return TTM_ERR_UNSUPPORTED;
    if (b.ntiles == 0) return TTM_OK;
    rot::SearchArgs sa;
    rot::PolishArgs pa;
    fill_args(b, g, sa, pa, list);
    switch (n_order) {
        case 2: return launch_rotation_n<2>(sa, pa, true, false, bf16, st, cnt);
        case 4: return launch_rotation_n<4>(sa, pa, true, false, bf16, st, cnt);
        case 6: return launch_rotation_n<6>(sa, pa, true, false, bf16, st, cnt);
        case 8: return launch_rotation_n<8>(sa, pa, true, false, bf16, st, cnt);
        default: return TTM_ERR_UNSUPPORTED;
    }
}

ttm_status launch_rotation_search(int n_order, const void* corr, bool bf16, const float* w,
                                  size_t nvox, const VoxBox& box, uint32_t u0, uint32_t u1,
                                  const RotGrid& g, uint16_t* cand, int* status, float* score,
                                  cudaStream_t st, long long* cnt, const UnitList& list) {
    if (box.count() > 0xFFFFFFFFull || (!list.idx && u1 > box.count())) return TTM_ERR_UNSUPPORTED;
    if (u1 <= u0) return TTM_OK;
    const RotBatch b = one_problem_batch(corr, w, nvox, box, u0, u1, cand, score, nullptr,
                                         nullptr, nullptr);
    return launch_rotation_search(n_order, b, bf16, g, status, st, cnt, list);
}

ttm_status launch_rotation_polish(int n_order, const void* corr, bool bf16, const float* w,
                                  size_t nvox, const VoxBox& box, uint32_t u0, uint32_t u1,
                                  const RotGrid& g, const uint16_t* cand, const float* score,
                                  float* quat, float* lambda, float* comp_out, cudaStream_t st,
                                  long long* cnt, const UnitList& list) {
    if (box.count() > 0xFFFFFFFFull || (!list.idx && u1 > box.count())) return TTM_ERR_UNSUPPORTED;
    if (u1 <= u0) return TTM_OK;
    const RotBatch b = one_problem_batch(corr, w, nvox, box, u0, u1, const_cast<uint16_t*>(cand),
                                         const_cast<float*>(score), quat, lambda, comp_out);
    return launch_rotation_polish(n_order, b, bf16, g, st, cnt, list);
}

template <int N>
static ttm_status score_only_n(const void* corr, bool bf16, const float* w, int X, int Y, int Z,
                               const VoxBox& box, float* score, cudaStream_t st, long long* cnt) {
    dim3 grid((unsigned)((X + 127) / 128), (unsigned)Y, (unsigned)Z);
    const size_t nvox = (size_t)X * Y * Z;
    if (bf16)
        rot::score_only_kernel<N, __nv_bfloat16><<<grid, 128, 0, st>>>(
            reinterpret_cast<const __nv_bfloat16*>(corr), w, X, Y, nvox, box, score);
    else
        rot::score_only_kernel<N, float><<<grid, 128, 0, st>>>(
            reinterpret_cast<const float*>(corr), w, X, Y, nvox, box, score);
    return after_launch(cnt);
}

ttm_status launch_score_only(int n_order, const void* corr, bool bf16, const float* w, int X,
                             int Y, int Z, const VoxBox& box, float* score, cudaStream_t st,
                             long long* cnt) {
    if (Y > 65535 || Z > 65535) return TTM_ERR_UNSUPPORTED;
    switch (n_order) {
        case 2: return score_only_n<2>(corr, bf16, w, X, Y, Z, box, score, st, cnt);
        case 4: return score_only_n<4>(corr, bf16, w, X, Y, Z, box, score, st, cnt);
        case 6: return score_only_n<6>(corr, bf16, w, X, Y, Z, box, score, st, cnt);
        case 8: return score_only_n<8>(corr, bf16, w, X, Y, Z, box, score, st, cnt);
        default: return TTM_ERR_UNSUPPORTED;
    }
}

namespace {

// Exterior values for the voxels outside the interior box: score 0,
// q = (1, 0, 0, 0), lambda 0 and (optionally) C = 0.  One thread per voxel of
// an x-row; block (., y, z).
__global__ void exterior_fill_kernel(VoxBox b, int K, size_t nvox, float* score, float4* quat,
                                     float* lambda, float* comp_out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= b.X) return;
    const bool row_in = (uint32_t)(y - b.y0) < b.ny && (uint32_t)(z - b.z0) < b.nz;
    if (row_in && (uint32_t)(x - b.x0) < b.nx) return;
    const size_t v = ((size_t)z * b.Y + y) * b.X + x;
    score[v] = 0.f;
    quat[v] = make_float4(1.f, 0.f, 0.f, 0.f);
    if (lambda) lambda[v] = 0.f;
    if (comp_out)
        for (int k = 0; k < K; ++k) comp_out[(size_t)k * nvox + v] = 0.f;
}

}  // namespace

ttm_status launch_exterior_fill(int Z, const VoxBox& box, int K, float* score, float* quat,
                                float* lambda, float* comp_out, cudaStream_t st, long long* cnt) {
    if (box.X < 1 || box.Y < 1 || Z < 1 || box.Y > 65535 || Z > 65535) return TTM_ERR_UNSUPPORTED;
    dim3 grid((unsigned)((box.X + 127) / 128), (unsigned)box.Y, (unsigned)Z);
    exterior_fill_kernel<<<grid, 128, 0, st>>>(box, K, (size_t)box.X * box.Y * Z, score,
                                               reinterpret_cast<float4*>(quat), lambda, comp_out);
    return after_launch(cnt);
}

}  // namespace ttm
