// Per-voxel score and rotation kernel for tensor order n = 6.
#include "k_rotation.cuh"

namespace ttm {

template <>
ttm_status launch_rotation_n<6>(const rot::RotArgs& a, cudaStream_t st, long long* cnt) {
    return rot::launch_n<6>(a, st, cnt);
}

}  // namespace ttm
