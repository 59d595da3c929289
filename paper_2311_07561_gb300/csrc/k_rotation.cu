// Dispatch of the per-voxel score and rotation kernel by tensor order.
#include "k_rotation.cuh"

namespace ttm {

int rotation_row_stride(int n_order) { return (n_comp(n_order) + 3) & ~3; }

static void fill_args(const void* corr, const float* w, size_t nvox, const RotGrid& g,
                      uint16_t* cand, float* score, float* quat, float* lambda, float* comp_out,
                      rot::SearchArgs& sa, rot::PolishArgs& pa) {
    sa.corr = corr; sa.w = w; sa.nvox = nvox; sa.score = score; sa.cand = cand;
    sa.gm = g.d_m; sa.cell_end = g.d_cell_end; sa.n_grid = g.n_grid;
    pa.corr = corr; pa.w = w; pa.nvox = nvox; pa.score = score; pa.cand = cand; pa.quat = quat;
    pa.lambda = lambda; pa.comp_out = comp_out; pa.gq = g.d_q; pa.n_cand = g.n_cand;
    pa.newton = g.newton;
}

ttm_status launch_rotation_search(int n_order, const void* corr, bool bf16, const float* w,
                                  size_t nvox, const RotGrid& g, uint16_t* cand, int* status,
                                  float* score, cudaStream_t st, long long* cnt) {
    rot::SearchArgs sa;
    rot::PolishArgs pa;
    fill_args(corr, w, nvox, g, cand, score, nullptr, nullptr, nullptr, sa, pa);
    if (n_order == 4 && g.d_gtab)
        return launch_search_tc4(sa, g.d_gtab, g.d_endbits, status, bf16, st, cnt);
    switch (n_order) {
        case 2: return launch_rotation_n<2>(sa, pa, false, true, bf16, st, cnt);
        case 4: return launch_rotation_n<4>(sa, pa, false, true, bf16, st, cnt);
        case 6: return launch_rotation_n<6>(sa, pa, false, true, bf16, st, cnt);
        case 8: return launch_rotation_n<8>(sa, pa, false, true, bf16, st, cnt);
        default: return TTM_ERR_UNSUPPORTED;
    }
}

ttm_status launch_rotation_polish(int n_order, const void* corr, bool bf16, const float* w,
                                  size_t nvox, const RotGrid& g, const uint16_t* cand,
                                  const float* score, float* quat, float* lambda, float* comp_out,
                                  cudaStream_t st, long long* cnt) {
    rot::SearchArgs sa;
    rot::PolishArgs pa;
    fill_args(corr, w, nvox, g, const_cast<uint16_t*>(cand), const_cast<float*>(score), quat,
              lambda, comp_out, sa, pa);
    switch (n_order) {
        case 2: return launch_rotation_n<2>(sa, pa, true, false, bf16, st, cnt);
        case 4: return launch_rotation_n<4>(sa, pa, true, false, bf16, st, cnt);
        case 6: return launch_rotation_n<6>(sa, pa, true, false, bf16, st, cnt);
        case 8: return launch_rotation_n<8>(sa, pa, true, false, bf16, st, cnt);
        default: return TTM_ERR_UNSUPPORTED;
    }
}

}  // namespace ttm
