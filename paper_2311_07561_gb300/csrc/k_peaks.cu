// Peaks of the TTM position score (Sec. 3.4 of the paper: the Frobenius norm
// of C_n(x) locates candidate matches).  A voxel is a peak when its score
// exceeds the threshold and beats every other voxel of the (2r+1)^3 cube
// around it; equal scores go to the lower linear index.
//
// Three separable passes compute the cube maximum (x, then y, then z); the
// last pass keeps the voxels equal to their cube maximum, resolves exact ties
// by scanning the cube of those few voxels, and appends them to a list.
#include "ttm_internal.h"

namespace ttm {

namespace {

struct PeakRec {
    int idx;
    float score;
    float lambda;
    float q[4];
    int pad;
};

__global__ void max_x_kernel(const float* __restrict__ in, float* __restrict__ out, int X, int Y,
                             int Z, int r) {
    size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t n = (size_t)X * Y * Z;
    if (v >= n) return;
    int x = (int)(v % X);
    float m = -INFINITY;
    for (int d = -r; d <= r; ++d) {
        int xx = x + d;
        if (xx >= 0 && xx < X) m = fmaxf(m, in[v + d]);
    }
    out[v] = m;
}

__global__ void max_y_kernel(const float* __restrict__ in, float* __restrict__ out, int X, int Y,
                             int Z, int r) {
    size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t n = (size_t)X * Y * Z;
    if (v >= n) return;
    int y = (int)((v / X) % Y);
    float m = -INFINITY;
    for (int d = -r; d <= r; ++d) {
        int yy = y + d;
        if (yy >= 0 && yy < Y) m = fmaxf(m, in[(long long)v + (long long)d * X]);
    }
    out[v] = m;
}

__global__ void peak_z_kernel(const float* __restrict__ score, const float* __restrict__ mxy,
                              const float* __restrict__ quat, const float* __restrict__ lam,
                              int X, int Y, int Z, int r, float thr, PeakRec* list, int cap,
                              int* count) {
    size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t n = (size_t)X * Y * Z;
    if (v >= n) return;
    const float s = score[v];
    if (!(s > thr)) return;
    const int x = (int)(v % X), y = (int)((v / X) % Y), z = (int)(v / ((size_t)X * Y));
    const size_t plane = (size_t)X * Y;
    float m = -INFINITY;
    for (int d = -r; d <= r; ++d) {
        int zz = z + d;
        if (zz >= 0 && zz < Z) m = fmaxf(m, mxy[(long long)v + (long long)d * (long long)plane]);
    }
    if (s < m) return;
    // s is the cube maximum; an equal score at a lower linear index wins
    for (int dz = -r; dz <= 0; ++dz) {
        int zz = z + dz;
        if (zz < 0 || zz >= Z) continue;
        for (int dy = -r; dy <= r; ++dy) {
            int yy = y + dy;
            if (yy < 0 || yy >= Y) continue;
            if (dz == 0 && dy > 0) break;
            for (int dx = -r; dx <= r; ++dx) {
                int xx = x + dx;
                if (xx < 0 || xx >= X) continue;
                if (dz == 0 && dy == 0 && dx >= 0) break;
                if (score[((size_t)zz * Y + yy) * X + xx] == s) return;
            }
        }
    }
    int slot = atomicAdd(count, 1);
    if (slot >= cap) return;
    PeakRec rec;
    rec.idx = (int)v;
    rec.score = s;
    rec.lambda = lam ? lam[v] : 0.f;
    const float4 q = quat ? reinterpret_cast<const float4*>(quat)[v] : make_float4(1.f, 0.f, 0.f, 0.f);
    rec.q[0] = q.x; rec.q[1] = q.y; rec.q[2] = q.z; rec.q[3] = q.w;
    rec.pad = 0;
    list[slot] = rec;
}

// Running maximum of c_j(x) = w(x) corr_j(x) over a batch of rotations j0..j0+nb-1
// (Algorithm 1 reduced over the rotation set); first index wins ties.
__global__ void best_rotation_kernel(const float* __restrict__ corr, int nb, int j0,
                                     const float* __restrict__ w, size_t nvox,
                                     float* __restrict__ best, int* __restrict__ best_j, int first) {
    const size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvox) return;
    const float wv = w[v];
    float b = first ? -INFINITY : best[v];
    int bj = first ? 0 : best_j[v];
    for (int j = 0; j < nb; ++j) {
        const float c = wv * corr[(size_t)j * nvox + v];
        if (c > b) { b = c; bj = j0 + j; }
    }
    best[v] = b;
    best_j[v] = bj;
}

}  // namespace

ttm_status launch_best_rotation(const float* corr, int nb, int j0, const float* w, size_t nvox,
                                float* best, int* best_j, bool first, cudaStream_t st,
                                long long* cnt) {
    best_rotation_kernel<<<(unsigned)((nvox + 255) / 256), 256, 0, st>>>(corr, nb, j0, w, nvox, best,
                                                                          best_j, first ? 1 : 0);
    return after_launch(cnt);
}

size_t peak_record_bytes() { return sizeof(PeakRec); }

ttm_status launch_peak_candidates_full(const float* score, const float* quat, const float* lam,
                                       int X, int Y, int Z, float thr, int radius, float* tmp_a,
                                       float* tmp_b, void* list, int cap, int* d_count,
                                       cudaStream_t st, long long* cnt) {
    const size_t n = (size_t)X * Y * Z;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    max_x_kernel<<<blocks, 256, 0, st>>>(score, tmp_a, X, Y, Z, radius);
    TTM_TRY(after_launch(cnt));
    max_y_kernel<<<blocks, 256, 0, st>>>(tmp_a, tmp_b, X, Y, Z, radius);
    TTM_TRY(after_launch(cnt));
    peak_z_kernel<<<blocks, 256, 0, st>>>(score, tmp_b, quat, lam, X, Y, Z, radius, thr,
                                          reinterpret_cast<PeakRec*>(list), cap, d_count);
    return after_launch(cnt);
}

}  // namespace ttm
