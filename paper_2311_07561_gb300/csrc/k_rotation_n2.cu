// Per-voxel score and rotation kernel for tensor order n = 2.
#include "k_rotation.cuh"

namespace ttm {

template <>
ttm_status launch_rotation_n<2>(const rot::RotArgs& a, cudaStream_t st, long long* cnt) {
    return rot::launch_n<2>(a, st, cnt);
}

}  // namespace ttm
