// Internal declarations shared by the C ABI and the kernel files.
#pragma once

#include <vector>

#include "ttm_common.cuh"

namespace ttm {

// One x-run of a binary mask: mask(c + dx, c + dy, c + dz) = 1 for
// dx in [x0, x1], all offsets relative to the box centre c.
struct MaskRun {
    int dy, dz, x0, x1;
};

// Plan-side image of one template.
struct TemplateData {
    ttm_tt_desc desc{};
    const float* d_comp = nullptr;      // caller-owned K x s^3 components
    float* d_mask = nullptr;            // plan copy of the mask (s^3)
    bool soft = false;                  // mask values in (0, 1) occur: FFT path only
    std::vector<MaskRun> runs;          // mask as x-runs, sorted by (dz, dy)
    int n_taps = 0;                     // mask voxels
    int dz_min = 0, dz_max = -1, dy_min = 0, dy_max = -1, x_min = 0, x_max = -1;
    MaskRun* d_runs = nullptr;          // device copy of runs
    int* d_run_tap0 = nullptr;          // first tap index of every run
    int* d_dz_run0 = nullptr;           // first run of every dz plane (dz_max-dz_min+2)
    float* d_taps = nullptr;            // n_taps x K component values, tap-major
    // tensor-core direct path (small masks): FP16 table of T / max|T| in the
    // kernel's layout, per-tap offsets (dx, dy, dz) packed, and max|T|
    uint16_t* d_tc_tab = nullptr;
    int* d_tap_dxyz = nullptr;
    float tc_scale = 1.f;
    // FFT path (allocated when some problem with this template uses it)
    void* d_spec = nullptr;             // K template spectra per FFT shape
    int spec_shape[3] = {0, 0, 0};
};

// Padded FFT box of a problem and its twiddle tables (plan-owned).
struct FftShape {
    int Xp = 0, Yp = 0, Zp = 0;
    const float2* d_tw_x = nullptr;   // exp(-2 pi i k / Xp), k < Xp
    const float2* d_tw_y = nullptr;
    const float2* d_tw_z = nullptr;
    size_t nspec() const { return (size_t)(Xp / 2 + 1) * Yp * Zp; }
};

struct ProblemData {
    int X = 0, Y = 0, Z = 0;
    int tmpl = 0;
    int path = TTM_PATH_DIRECT;
    FftShape fft;
    bool mixed = false;                // bf16 spectra, products and correlation maps
    bool tc_direct = false;            // direct path on the tensor cores (FP16 operands)
    int spec_index = -1;               // template spectra set used (FFT path)
    double tune_ms[2] = {-1.0, -1.0};  // autotuner: direct, FFT (ms), -1 = not timed
    size_t lp_off = 0;                 // workspace offset of the prefiltered volume (+ scratch)
    // resident waves (plan option batch_mib): workspace offsets of this
    // problem's correlation maps and search candidates
    size_t res_corr_off = 0, res_cand_off = 0;
    size_t nvox() const { return (size_t)X * Y * Z; }
};

// Template spectra for one (template, FFT box): K half spectra, scaled by 1/N.
struct SpecSet {
    int tmpl = 0, Xp = 0, Yp = 0, Zp = 0;
    bool mixed = false;
    float2* d_spec = nullptr;          // FP32: K component spectra
    void* d_spec_bf = nullptr;         // mixed precision: K component spectra in bf16
    float2* d_mask_spec = nullptr;     // FP32 mask spectrum (local statistics)
};

// Interior box of an X x Y x Z volume for template edge s: the voxels whose
// whole s^3 box lies inside the volume, [c, n - s + c] per axis (c = s / 2).
// The rotation kernels enumerate only these voxels, x fastest; unit i maps to
// the voxel with linear index voxel(i).
struct VoxBox {
    int X = 0, Y = 0;
    int x0 = 0, y0 = 0, z0 = 0;
    uint32_t nx = 0, ny = 0, nz = 0;
    __host__ __device__ size_t count() const { return (size_t)nx * ny * nz; }
    __device__ __forceinline__ size_t voxel(uint32_t i) const {
        const uint32_t r = i / nx, x = i - r * nx;
        const uint32_t z = r / ny, y = r - z * ny;
        return ((size_t)(z0 + z) * Y + (y0 + y)) * X + (x0 + x);
    }
};

// Optional unit list of the rotation kernels: unit i is the voxel idx[i *
// stride] instead of box.voxel(i), the number of units is read on the device
// from *count (clamped to the launch's u1), and with out_stride > 0 the
// refinement writes q to quat[i * out_stride + 0..3] and lambda to
// lambda[i * out_stride] instead of the voxel-indexed maps.
struct UnitList {
    const int* idx = nullptr;
    int stride = 0;
    const int* count = nullptr;
    int out_stride = 0;
};

// One problem's share of a rotation launch: its correlation maps, w, search
// candidates and output maps, and the interior units [u0, u1) the launch
// visits, which occupy tiles tile0, tile0 + 1, ... of the launch's tile space
// (tiles of 128 units; a tile never spans two problems).
struct RotSeg {
    const void* corr = nullptr;   // K x nvox, float or bf16
    const float* w = nullptr;
    float* score = nullptr;
    uint16_t* cand = nullptr;     // 8 candidate grid indices per unit
    float* quat = nullptr;        // 4 x nvox
    float* lambda = nullptr;      // nullable
    float* comp_out = nullptr;    // nullable, K x nvox
    size_t nvox = 0;
    VoxBox box;
    uint32_t u0 = 0, u1 = 0, tile0 = 0, pad = 0;
};

// The problems of one rotation launch, in tile order; one launch serves up to
// kMaxRotSegs problems (the table travels in the kernel's parameters).
constexpr int kMaxRotSegs = 24;
constexpr int kRotTile = 128;
struct RotBatch {
    int n = 0;
    uint32_t ntiles = 0;          // tiles of all segments
    RotSeg seg[kMaxRotSegs];
    // appends units [u0, u1) of a problem; false when the table is full
    bool add(const RotSeg& s) {
        if (n == kMaxRotSegs) return false;
        seg[n] = s;
        seg[n].tile0 = ntiles;
        ntiles += (s.u1 - s.u0 + kRotTile - 1) / kRotTile;
        ++n;
        return true;
    }
};

inline VoxBox interior_box(int X, int Y, int Z, int s) {
    VoxBox b;
    b.X = X; b.Y = Y;
    const int c = s / 2;
    b.x0 = c; b.y0 = c; b.z0 = c;
    b.nx = X >= s ? (uint32_t)(X - s + 1) : 0u;
    b.ny = Y >= s ? (uint32_t)(Y - s + 1) : 0u;
    b.nz = Z >= s ? (uint32_t)(Z - s + 1) : 0u;
    return b;
}

// Voxels whose inverse-FFT outputs are used (inclusive bounds): the inverse
// passes skip the z planes, y rows and x samples outside it.
struct FftKeep {
    int x0, x1, y0, y1, z0, z1;
};
inline FftKeep fft_keep_interior(int X, int Y, int Z, int s) {
    const int c = s / 2;
    return FftKeep{c, X - s + c, c, Y - s + c, c, Z - s + c};
}
inline FftKeep fft_keep_all(int X, int Y, int Z) { return FftKeep{0, X - 1, 0, Y - 1, 0, Z - 1}; }

// Rotation search grid (device tables owned by the plan).
struct RotGrid {
    int n_grid = 0, n_cells = 0, n_cand = 0, newton = 0, n_refine = 0;
    float* d_q = nullptr;        // n_grid x 4 unit quaternions, a >= 0, sorted by cell
    float* d_m = nullptr;        // n_grid x K: mu_alpha q_g^alpha
    int* d_cell_end = nullptr;   // n_grid: 1 if the next point starts a new cell
    uint16_t* d_gtab = nullptr;  // orders 4 and 6, 2048 points: FP16 table in tensor-core layout
    uint32_t* d_endbits = nullptr;  // region ends as a bitmask (n_grid / 32 words)
};

}  // namespace ttm

namespace ttm {
enum KernelClass {
    KC_MOMENTS = 0, KC_LOCAL_STATS, KC_DIRECT_CORR, KC_ROTATION, KC_FFT_FORWARD, KC_FFT_SPECTRUM,
    KC_FFT_INVERSE, KC_PEAKS, KC_TEMPLATE, KC_FFT_PLAN, KC_POLISH, KC_EXTERIOR,
    KC_ROT_STAGE   // span of a whole score/rotation stage (not a kernel)
};
struct TimedLaunch {
    int cls;
    cudaEvent_t start, stop;
    long long n;
};
}  // namespace ttm

struct ttm_plan_s {
    std::vector<ttm::TemplateData> tmpl;
    std::vector<ttm::ProblemData> prob;
    ttm_plan_opts opts{};
    int n_order = 4;
    int K = 35;
    ttm::RotGrid grid;
    std::vector<ttm::SpecSet> specs;
    std::vector<std::pair<int, float2*>> twiddles;   // length -> device table
    size_t ws_bytes = 0;
    // resident waves: problem ranges [first, second) whose correlation maps
    // are in the workspace together, and the offset of the spectra scratch
    // after them (empty: one problem at a time)
    std::vector<std::pair<int, int>> waves;
    size_t wave_scratch_off = 0;
    long long launches = 0;
    bool timing = false;
    std::vector<ttm::TimedLaunch> timed;   // pending event pairs
    std::vector<cudaEvent_t> event_pool;
    // rotation stage pipelining: search on hi, refinement on lo, chunk by chunk
    int rot_chunks = 1;
    cudaStream_t s_hi = nullptr, s_lo = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    std::vector<cudaEvent_t> ev_chunk;
};

namespace ttm {

// ---- workspace layout helpers ----
inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// ---- kernel launchers (each returns TTM_OK or TTM_ERR_CUDA) ----

// sum f and sum f^2 over a whole volume into d_acc[0..1] (FP64, must be zeroed)
ttm_status launch_volume_moments(const float* f, size_t n, double* d_acc, cudaStream_t st,
                                 long long* cnt);

// Gaussian prefilter (k_lowpass.cu): out = h * in, tmp is scratch of the
// same size; in, tmp and out must be distinct
bool lowpass_sigma_ok(float sigma);
ttm_status launch_lowpass(const float* in, int X, int Y, int Z, float sigma, float* tmp,
                          float* out, cudaStream_t st, long long* cnt);

// deterministic pseudo-random values in [-1, 1) (autotuner input)
ttm_status launch_fill_random(float* f, size_t n, uint32_t seed, cudaStream_t st, long long* cnt);

ttm_status launch_local_stats(const float* f, int X, int Y, int Z, const TemplateData& T,
                              const double* d_moments, float* w, cudaStream_t st,
                              long long* cnt);

ttm_status launch_direct_corr(const float* f, int X, int Y, int Z, const TemplateData& T,
                              int K, float* corr, cudaStream_t st, long long* cnt);

// direct correlation as an implicit GEMM on the tensor cores (interior voxels)
int direct_tc_columns(int K);
size_t direct_tc_smem(int K, int n_taps);
bool direct_tc_supported(int K, int n_taps);
void build_direct_tc_table(const std::vector<float>& taps, int n_taps, int K,
                           std::vector<uint16_t>& out, float* t_scale);
ttm_status launch_direct_tc(const float* f, int X, int Y, int Z, const TemplateData& T, int K,
                            const double* d_moments, float* corr, int* status, cudaStream_t st,
                            long long* cnt);

// one CTA waiting `polls` polls on an mbarrier phase (arrive = 1: the CTA
// completes it first); *d_status = TTM_OK or TTM_ERR_TIMEOUT
ttm_status launch_wait_probe(long polls, int arrive, int* d_status, cudaStream_t st,
                             long long* cnt);

// per-voxel score + candidate search (tensor cores for order 4 with the
// default 2048-point grid, CUDA cores otherwise) and refinement, over the
// interior box only; launch_exterior_fill writes the exterior values (score 0,
// q = (1, 0, 0, 0), lambda 0, C 0) of the voxels outside it.  cand holds one
// 16-byte record per interior voxel.
// Both visit the interior units [u0, u1) of box (unit i = voxel box.voxel(i)).
ttm_status launch_rotation_search(int n_order, const void* corr, bool bf16, const float* w,
                                  size_t nvox, const VoxBox& box, uint32_t u0, uint32_t u1,
                                  const RotGrid& g, uint16_t* cand, int* status, float* score,
                                  cudaStream_t st, long long* cnt,
                                  const UnitList& list = UnitList());
ttm_status launch_rotation_polish(int n_order, const void* corr, bool bf16, const float* w,
                                  size_t nvox, const VoxBox& box, uint32_t u0, uint32_t u1,
                                  const RotGrid& g, const uint16_t* cand, const float* score,
                                  float* quat, float* lambda, float* comp_out, cudaStream_t st,
                                  long long* cnt, const UnitList& list = UnitList());
// The same over a batch of problems: one launch visits the units of every
// segment of b (all with the same map type); a unit list needs b.n == 1.
ttm_status launch_rotation_search(int n_order, const RotBatch& b, bool bf16, const RotGrid& g,
                                  int* status, cudaStream_t st, long long* cnt,
                                  const UnitList& list = UnitList());
ttm_status launch_rotation_polish(int n_order, const RotBatch& b, bool bf16, const RotGrid& g,
                                  cudaStream_t st, long long* cnt,
                                  const UnitList& list = UnitList());
RotBatch one_problem_batch(const void* corr, const float* w, size_t nvox, const VoxBox& box,
                           uint32_t u0, uint32_t u1, uint16_t* cand, float* score, float* quat,
                           float* lambda, float* comp_out);
// score = ||w Corr||_F at the interior voxels, 0 outside (no rotation)
ttm_status launch_score_only(int n_order, const void* corr, bool bf16, const float* w, int X,
                             int Y, int Z, const VoxBox& box, float* score, cudaStream_t st,
                             long long* cnt);
ttm_status launch_exterior_fill(int Z, const VoxBox& box, int K, float* score, float* quat,
                                float* lambda, float* comp_out, cudaStream_t st, long long* cnt);
// FP16 grid table of the tensor-core search (2048 points, K components + the
// constant column, padded to a multiple of 16, chunk-major core-matrix layout)
void build_grid_fp16(const float* m_rows, int K, int K4, int n_grid, std::vector<uint16_t>& out);
bool search_tc_supported(int n_order, int n_grid, int n_cells);

// tensor template build
ttm_status launch_rotate_normalise(const float* t, const float* m, int s, const float* quats,
                                   int j0, int nj, float* out, double mask_sum, int* d_bad,
                                   cudaStream_t st, long long* cnt);
ttm_status launch_mask_sum(const float* m, int s, double* d_out, cudaStream_t st,
                           long long* cnt);
ttm_status launch_fold_components(int n_order, const float* quats, const float* weights,
                                  int n_rot_total, int j0, int nj, const float* rot, int s3,
                                  float* comp, bool first, cudaStream_t st, long long* cnt);

// FFT path
bool fft_length_ok(int L);
int fft_good_length(int n);
// mode 0: F(f); 1: F(f - mean); 2: F((f - mean)^2), mean from moments (sum f first)
ttm_status launch_fft_forward(const float* f, int X, int Y, int Z, const FftShape& S,
                              float2* spec, cudaStream_t st, long long* cnt, int mode = 0,
                              double* moments = nullptr);
bool fft_template_length(int L);
// mixed precision (bf16 storage, FP32 arithmetic); lengths 16..1024 only
ttm_status launch_fft_spectrum_inverse_z_bf16(const float2* spec, const void* tspec, int K,
                                              const FftShape& S, void* prod, const FftKeep& keep,
                                              cudaStream_t st, long long* cnt);
// status: device word that records TTM_ERR_TIMEOUT if a bounded copy wait expires
ttm_status launch_fft_inverse_yx_bf16(void* prod, int K, int X, int Y, int Z, const FftShape& S,
                                      void* corr, int* status, const FftKeep& keep,
                                      cudaStream_t st, long long* cnt);
ttm_status launch_spectra_to_bf16(const float2* a, void* b, size_t n, cudaStream_t st, long long* cnt);
// w from FP32 FFT window sums; windows whose FP32 rounding bound exceeds the
// tolerance get w = -1 and are counted in *flagged for launch_exact_stats
ttm_status launch_stats_from_sums(const float* s1, const float* s2, float* w, int X, int Y, int Z,
                                  int s, double mask_sum, const double* moments,
                                  unsigned int* flagged, cudaStream_t st, long long* cnt);
// exact FP64 window sums and w at the voxels flagged by launch_stats_from_sums
ttm_status launch_exact_stats(const float* f, float* w, int X, int Y, int Z,
                              const TemplateData& T, const double* moments,
                              const unsigned int* flagged, cudaStream_t st, long long* cnt);
// keep: the voxels whose outputs are used (z range for the multiply pass)
ttm_status launch_fft_spectrum_inverse_z(const float2* spec, const float2* tspec, int K,
                                         const FftShape& S, float2* prod, const FftKeep& keep,
                                         cudaStream_t st, long long* cnt);
ttm_status launch_fft_inverse_yx(float2* prod, int K, int X, int Y, int Z, const FftShape& S,
                                 float* corr, int* status, const FftKeep& keep, cudaStream_t st,
                                 long long* cnt);
ttm_status launch_template_spectra(const float* comp, int K, int s, const FftShape& S,
                                   float* pad, float2* tspec, cudaStream_t st, long long* cnt);

// classical comparator
ttm_status launch_best_rotation(const float* corr, int nb, int j0, const float* w, size_t nvox,
                                float* best, int* best_j, bool first, cudaStream_t st,
                                long long* cnt);

// peaks
size_t peak_record_bytes();
ttm_status launch_peak_candidates_full(const float* score, const float* quat, const float* lam,
                                       int X, int Y, int Z, float thr, int radius, float* tmp_a,
                                       float* tmp_b, void* list, int cap, int* d_count,
                                       cudaStream_t st, long long* cnt);

// padded row length of the rotation-grid monomial table
int rotation_row_stride(int n_order);

}  // namespace ttm
