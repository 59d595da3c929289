// Self-check of the bounded device-side wait: one CTA waits, with the poll
// loop the tensor-core kernels wait with (mbar_wait_bounded), on an mbarrier
// phase that completes only if the CTA itself arrives on it first.
#include "ttm_internal.h"

namespace ttm {

namespace {

__global__ void wait_probe_kernel(long polls, int arrive, int* status) {
    __shared__ __align__(8) uint64_t bar;
    const uint32_t b = (uint32_t)__cvta_generic_to_shared(&bar);
    if (threadIdx.x == 0)
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(b) : "memory");
    __syncthreads();
    if (arrive && threadIdx.x == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(b) : "memory");
    __syncthreads();
    if (threadIdx.x == 0) *status = mbar_wait_bounded(b, 0u, polls) ? TTM_OK : TTM_ERR_TIMEOUT;
}

}  // namespace

ttm_status launch_wait_probe(long polls, int arrive, int* d_status, cudaStream_t st,
                             long long* cnt) {
    wait_probe_kernel<<<1, 32, 0, st>>>(polls, arrive, d_status);
    return after_launch(cnt);
}

}  // namespace ttm
