// Tensor-template build that allocates nothing.
//
// Some callers cannot allocate device memory: host applications that own all
// GPU memory through their own pool or a fixed budget and do not let plug-in
// libraries call cudaMalloc behind their back, and pipelines that must not pay
// the implicit device synchronisation and fragmentation of cudaMalloc/cudaFree.
// For them, ttm_build_tensor_template_noalloc runs the same kernels as
// ttm_build_tensor_template but takes its scratch (the per-call header and the
// chunk of rotated, normalised template copies) from one fixed array that
// lives in this file.  The caller still provides the inputs and the output
// components; nothing is allocated, neither here nor by any library routine.
#include <cstdint>
#include <mutex>

#include "ttm_internal.h"

namespace ttm {
namespace {

constexpr size_t kNoallocHeader = 256;

bool aligned4(const void* p) { return ((uintptr_t)p % 4) == 0; }

// The fixed scratch.  Every GPU that loads the library holds these bytes until
// the process exits.  In host code this name is only a stand-in for the symbol,
// never a device address: the address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[TTM_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the fixed scratch on the current device, looked up once
// per device (with that device current) and cached.  The cached address is
// not refreshed: after cudaDeviceReset on a device it is stale.
ttm_status scratch_address(void** out) {
    int dev = -1;
    TTM_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return TTM_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        TTM_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        if (!p) return TTM_ERR_CUDA;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return TTM_OK;
}

}  // namespace
}  // namespace ttm

using namespace ttm;

extern "C" ttm_status ttm_build_tensor_template_noalloc(const float* d_template, const float* d_mask,
                                                        int s, int n_order, const float* d_quats,
                                                        const float* d_weights, int n_rot,
                                                        float* d_components, ttm_tt_desc* desc,
                                                        void* stream) {
    if (!d_template || !d_mask || !d_quats || !d_components || !desc) return TTM_ERR_INVALID_ARG;
    if (s < 3 || s > 128 || n_rot < 1) return TTM_ERR_INVALID_ARG;
    if (n_order < 2 || n_order > 8 || (n_order & 1)) return TTM_ERR_UNSUPPORTED;
    const size_t s3 = (size_t)s * s * s;
    const size_t per_rot = s3 * sizeof(float);
    // one rotated copy must fit next to the header
    if (kNoallocHeader + per_rot > (size_t)TTM_NOALLOC_SCRATCH_BYTES) return TTM_ERR_WORKSPACE;
    // the same pointer checks as the regular build: the kernels read and write
    // these arrays as float
    if (!aligned4(d_template) || !aligned4(d_mask) || !aligned4(d_quats) ||
        !aligned4(d_components) || !aligned4(d_weights))
        return TTM_ERR_INVALID_ARG;
    void* base = nullptr;
    TTM_TRY(scratch_address(&base));
    cudaStream_t st = (cudaStream_t)stream;
    long long cnt = 0;
    char* ws = (char*)base;
    double* d_msum = (double*)ws;
    int* d_bad = (int*)(ws + 8);
    float* rot = (float*)(ws + kNoallocHeader);
    size_t nj_max = ((size_t)TTM_NOALLOC_SCRATCH_BYTES - kNoallocHeader) / per_rot;
    const int nj = (int)(nj_max < (size_t)n_rot ? nj_max : (size_t)n_rot);
    // the array keeps the previous call's contents: clear the header
    TTM_CUDA_TRY(cudaMemsetAsync(ws, 0, kNoallocHeader, st));
    TTM_TRY(launch_mask_sum(d_mask, s, d_msum, st, &cnt));
    double msum = 0.0;
    TTM_CUDA_TRY(cudaMemcpyAsync(&msum, d_msum, sizeof(double), cudaMemcpyDeviceToHost, st));
    TTM_CUDA_TRY(cudaStreamSynchronize(st));
    if (!(msum > 0.0)) return TTM_ERR_INVALID_ARG;
    for (int j0 = 0; j0 < n_rot; j0 += nj) {
        const int cnt_j = n_rot - j0 < nj ? n_rot - j0 : nj;
        TTM_TRY(launch_rotate_normalise(d_template, d_mask, s, d_quats, j0, cnt_j, rot, msum, d_bad,
                                        st, &cnt));
        TTM_TRY(launch_fold_components(n_order, d_quats, d_weights, n_rot, j0, cnt_j, rot, (int)s3,
                                       d_components, j0 == 0, st, &cnt));
    }
    int bad = 0;
    TTM_CUDA_TRY(cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    TTM_CUDA_TRY(cudaStreamSynchronize(st));
    if (bad) return TTM_ERR_NUMERIC;
    desc->n_order = n_order;
    desc->K = n_comp(n_order);
    desc->s = s;
    desc->centre = s / 2;
    desc->n_rot = n_rot;
    desc->reserved = 0;
    desc->mask_sum = msum;
    return TTM_OK;
}
