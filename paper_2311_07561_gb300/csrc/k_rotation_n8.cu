// Per-voxel score and rotation kernel for tensor order n = 8.
#include "k_rotation.cuh"

namespace ttm {

template <>
ttm_status launch_rotation_n<8>(const rot::RotArgs& a, cudaStream_t st, long long* cnt) {
    return rot::launch_n<8>(a, st, cnt);
}

}  // namespace ttm
