// Dispatch of the per-voxel score and rotation kernel by tensor order.
#include "k_rotation.cuh"

namespace ttm {

int rotation_row_stride(int n_order) { return (n_comp(n_order) + 3) & ~3; }

ttm_status launch_rotation(int n_order, const float* corr, const float* w, size_t nvox, int X,
                           int Y, int Z, int s, const RotGrid& g, float* score, float* quat,
                           float* lambda, float* comp_out, cudaStream_t st, long long* cnt) {
    (void)X; (void)Y; (void)Z; (void)s;
    rot::RotArgs a;
    a.corr = corr; a.w = w; a.nvox = nvox; a.score = score; a.quat = quat; a.lambda = lambda;
    a.comp_out = comp_out; a.gq = g.d_q; a.gm = g.d_m; a.cell_end = g.d_cell_end;
    a.n_grid = g.n_grid; a.n_cand = g.n_cand; a.newton = g.newton;
    switch (n_order) {
        case 2: return launch_rotation_n<2>(a, st, cnt);
        case 4: return launch_rotation_n<4>(a, st, cnt);
        case 6: return launch_rotation_n<6>(a, st, cnt);
        case 8: return launch_rotation_n<8>(a, st, cnt);
        default: return TTM_ERR_UNSUPPORTED;
    }
}

}  // namespace ttm
