// Score/search and refinement kernels for tensor order n = 4.
#include "k_rotation.cuh"

namespace ttm {

template <>
ttm_status launch_rotation_n<4>(const rot::SearchArgs& s, const rot::PolishArgs& p,
                                  bool search_done, bool search_only, bool bf16,
                                  cudaStream_t st, long long* cnt) {
    return rot::launch_n<4>(s, p, search_done, search_only, bf16, st, cnt);
}

}  // namespace ttm
