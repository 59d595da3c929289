/*
 * ttm.h -- C ABI of the GB300 (sm_103a) tensorial template matching engine.
 *
 * Tensorial template matching (TTM) is the method of Almira, Phelippeau and
 * Martinez-Sanchez, "Fast Normalized Cross-Correlation for Template Matching
 * with Rotations" (arXiv 2311.07561).  A template t is rotated through SO(3)
 * once, and every rotated, masked, normalised copy is folded into one
 * symmetric tensor template with K = C(n+3, n) independent components
 * (Sec. 3.2).  A volume f is then correlated with those K components instead
 * of with thousands of rotated copies; each voxel's K normalised correlations
 * C_n(x) give a position score (the Frobenius norm, Sec. 3.4) and a rotation
 * (the dominant Z-eigenvector of C_n(x), Sec. 3.3, Theorem 3.1).
 *
 * Conventions used by every entry point
 * -------------------------------------
 * - Volumes are float32, laid out [Z][Y][X] contiguous (x fastest).  Their
 *   sizes are given as (X, Y, Z).
 * - A template box is a cube of edge s, laid out [s][s][s] the same way; its
 *   centre is voxel c = floor(s/2) on every axis.  The mask m is a float32
 *   array of the same shape.
 * - Quaternions are four float32 (a, b, c, d), real part first.  The rotation
 *   R of a unit quaternion q maps a column vector v = (x, y, z) to q v q*.  The
 *   rotated template is t_R(u) = t(c + R^-1 (u - c)) (Sec. 2: t_R = O_{R^-1} t),
 *   resampled trilinearly with zero outside the box.
 * - Tensor components are indexed by sorted index tuples i1 <= ... <= in over
 *   {0, 1, 2, 3} (the quaternion components a, b, c, d), in lexicographic
 *   order: for n = 4, component 0 is (0,0,0,0), component 1 is (0,0,0,1), ...,
 *   component 34 is (3,3,3,3).
 * - Correlation values are defined on the interior of a volume: voxels whose
 *   whole s^3 template box lies inside it.  Every output map is written in
 *   full; voxels outside the interior get score 0, lambda 0, quaternion
 *   (1, 0, 0, 0) and w = 0.
 * - Pointers named d_* are device pointers (cudaMalloc or any allocator on
 *   the current device); h_* are host pointers.  The caller owns every buffer
 *   it passes in, including the workspaces; the library never frees them.
 * - stream is a cudaStream_t passed as void* (NULL = the legacy default
 *   stream).  Calls are asynchronous on that stream unless stated otherwise.
 *   Argument errors are detected on the host and returned before any work is
 *   queued.
 * - Every call returns a ttm_status; TTM_OK is 0, errors are negative.
 *
 * The library is compiled for sm_103a only.  There is no CPU fallback: on a
 * machine without a suitable GPU every compute entry point returns
 * TTM_ERR_CUDA.
 */
#ifndef TTM_H_
#define TTM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int ttm_status;

#define TTM_OK                 0
#define TTM_ERR_INVALID_ARG   -1  /* null pointer, bad size, misaligned buffer */
#define TTM_ERR_UNSUPPORTED   -2  /* odd order n, n > 8, soft mask off the FFT path */
#define TTM_ERR_OUT_OF_MEMORY -3  /* a plan-owned allocation failed            */
#define TTM_ERR_CUDA          -4  /* a CUDA runtime call or launch failed       */
#define TTM_ERR_TIMEOUT       -5  /* a bounded device-side wait ran out         */
#define TTM_ERR_NUMERIC       -6  /* non-finite values where finite are needed  */
#define TTM_ERR_WORKSPACE     -7  /* workspace missing or smaller than required */

/* Description of a built tensor template (filled by ttm_build_tensor_template). */
typedef struct ttm_tt_desc {
    int n_order;      /* tensor order n (even, 2..8)                          */
    int K;            /* number of independent components, C(n+3, n)          */
    int s;            /* edge of the cubic template box                       */
    int centre;       /* floor(s/2)                                           */
    int n_rot;        /* number of quadrature rotations folded in             */
    int reserved;
    double mask_sum;  /* <1, m>, the squared S-norm of the constant image     */
} ttm_tt_desc;

/* One detected peak (ttm_extract_peaks). */
typedef struct ttm_peak {
    int x, y, z;      /* voxel                                                */
    float score;      /* ||C_n(x)||_F                                         */
    float lambda;     /* dominant Z-eigenvalue, phi(q)                        */
    float q[4];       /* dominant Z-eigenvector, canonical (a >= 0)           */
} ttm_peak;

/* Correlation path. */
#define TTM_PATH_AUTO   0   /* planner picks FFT or direct per problem         */
#define TTM_PATH_DIRECT 1   /* direct sum over the mask support                */
#define TTM_PATH_FFT    2   /* FFT with the fused K-way spectrum multiply      */
#define TTM_PATH_TUNE   3   /* planner times both paths on a random volume of  */
                            /* each distinct problem shape (local statistics + */
                            /* K correlations, 1 warm-up + 2 timed runs each) */
                            /* and keeps the faster, wherever its cost model  */
                            /* puts them within 8x of each other (else the    */
                            /* model decides); plan creation then takes longer */
                            /* and needs scratch memory for one problem       */

/* Precision of the correlation step.  In both modes all arithmetic is FP32
 * except the rotation search of orders 4 and 6, which runs on the tensor cores
 * with FP16 operands and FP32 accumulation.  TTM_PREC_MIXED stores the template
 * spectra, the K product spectra and the K correlation maps of the FFT path
 * in bf16 (half the memory and traffic; FFT lengths 16..1024, other problems
 * stay FP32), and runs the direct path as an implicit GEMM on the tensor
 * cores (FP16 operands, FP32 accumulation; masks with up to ~1900 voxels for
 * order 4, ~950 for order 6; larger masks stay on the CUDA cores).  Expected
 * error vs FP32: |dC|, |dscore|, |dlambda| <= 5e-3. */
#define TTM_PREC_FP32   0
#define TTM_PREC_MIXED  1

typedef struct ttm_plan_opts {
    int path;           /* TTM_PATH_*                                          */
    int precision;      /* TTM_PREC_*                                          */
    int n_grid;         /* rotation search grid size; 0 = default (2048, or    */
                        /* 1024 with TTM_PREC_MIXED), <= 65535                */
    int n_cells;        /* regions of the grid; 0 = default (n_grid / 16);    */
                        /* must divide n_grid                                  */
    int n_candidates;   /* regions polished per voxel; 0 = default (8, or 2 at */
                        /* order 6)                                            */
    int newton_steps;   /* Newton steps per refined point; 0 = default (3, or  */
                        /* 2 at order 6)                                       */
    int rotation_chunks; /* split the interior into this many chunks and run  */
                         /* the search of chunk i+1 (high-priority stream)    */
                         /* beside the refinement of chunk i (low priority);  */
                         /* 0 = default (8), 1 = one search then one refinement */
    float lowpass_sigma; /* > 0: the volume is prefiltered by a Gaussian of   */
                         /* this sigma (voxels, <= 7.9; ttm_lowpass) inside   */
                         /* ttm_local_stats, ttm_correlate, ttm_match_peaks;  */
                         /* filter the template the same way before           */
                         /* ttm_build_tensor_template.  0 = none (h = identity) */
    int n_refined;       /* best points after the power steps that take the  */
                         /* Newton steps; 0 = default (4, or 2 at order 6), <= 4 */
    int batch_mib;       /* > 0: resident waves.  ttm_correlate keeps the     */
                         /* correlation maps and search candidates of         */
                         /* consecutive problems (same map type) in the       */
                         /* workspace together, up to this many MiB per wave, */
                         /* and runs the score/rotation stage of a wave as    */
                         /* one search launch and one refinement launch per   */
                         /* rotation chunk over a table of (problem, units)   */
                         /* segments (up to 24 problems per launch).  The     */
                         /* workspace grows by the largest wave.  0 = one     */
                         /* problem at a time.  <= 2^20                       */
} ttm_plan_opts;

typedef struct ttm_plan_s* ttm_plan_t;

/* Human-readable name of a status code (static storage). */
const char* ttm_status_string(ttm_status status);

/* Number of CUDA devices the library's runtime sees (0 when none). */
int ttm_device_count(void);

/* ------------------------------------------------------------------------
 * Tensor template (Sec. 3.2; normalisation as in Algorithm 1 and the
 * formulas for ||P_S t||_S and <t, 1>_S at the end of Sec. 2).
 *
 * For every quadrature node j the template is rotated (t_j = t_{R_j}),
 * masked and S-normalised,
 *     t~_j = m (t_j - <t_j, m>/<1, m>) / sqrt(<t_j^2, m> - <t_j, m>^2/<1, m>),
 * and folded into the components
 *     T_alpha(z) = sum_j w_j q_j^alpha t~_j(z),   q^alpha = q_i1 ... q_in,
 * a quadrature of T(z) = int R^(n) S(t)_R(z) dR for the normalised Haar
 * measure.  The low-pass filter h of Sec. 2 is the identity.
 *
 * ttm_build_workspace_size: bytes of device workspace ttm_build_tensor_template
 *   needs for (s, n_order, n_rot).
 * ttm_build_tensor_template:
 *   d_template   s^3 float32, the raw template.
 *   d_mask       s^3 float32, the mask m (any non-negative values).
 *   s            box edge, 3 <= s <= 128.
 *   n_order      even, 2 <= n_order <= 8.
 *   d_quats      n_rot x 4 float32 unit quaternions (normalised on use).
 *   d_weights    n_rot float32 weights, or NULL for 1/n_rot each.
 *   d_components output, K x s^3 float32, component order as above.
 *   d_workspace  >= ttm_build_workspace_size bytes, 256-byte aligned.
 *   desc         output (host), filled on success.
 * Synchronises the stream (the descriptor needs <1, m> on the host).
 * Errors: TTM_ERR_INVALID_ARG (null pointer, s or n_rot out of range),
 * TTM_ERR_UNSUPPORTED (n_order odd or out of range), TTM_ERR_WORKSPACE,
 * TTM_ERR_NUMERIC (a rotated copy has zero variance under the mask),
 * TTM_ERR_CUDA.
 * ---------------------------------------------------------------------- */
ttm_status ttm_build_workspace_size(int s, int n_order, int n_rot, size_t* bytes);
ttm_status ttm_build_tensor_template(const float* d_template, const float* d_mask, int s,
                                     int n_order, const float* d_quats, const float* d_weights,
                                     int n_rot, float* d_components, void* d_workspace,
                                     size_t workspace_bytes, ttm_tt_desc* desc, void* stream);

/* ------------------------------------------------------------------------
 * Tensor-template build that allocates nothing.  The paper has no
 * counterpart; this entry point is for callers that cannot allocate device
 * memory: host applications that own every byte of GPU memory through their
 * own pool or a fixed budget and do not let a library call cudaMalloc, and
 * pipelines that cannot accept the implicit device synchronisation and
 * fragmentation of cudaMalloc/cudaFree.  It computes what
 * ttm_build_tensor_template computes, with the same arguments minus the
 * workspace: its scratch is one fixed array of TTM_NOALLOC_SCRATCH_BYTES
 * (8 MiB) inside the library, which every GPU that loads the library holds
 * until the process exits.  No cudaMalloc, cudaFree or allocating library
 * routine is called.
 * Limit: one rotated s^3 float32 copy plus a 256-byte header must fit the
 * array, so s <= 127; a larger s returns TTM_ERR_WORKSPACE before any work.
 * The first call on a device looks up the array's device address with
 * cudaGetSymbolAddress (once per device, with that device current) and
 * caches it; make that first call before any stream capture.  The cached
 * address is never looked up again, so after cudaDeviceReset on a device the
 * entry point must not be called there for the rest of the process.
 * Pointers must be 4-byte aligned (else TTM_ERR_INVALID_ARG, before any work).
 * Every call uses the same array and it keeps the previous call's contents
 * (the call clears what must start at zero).  Calls that overlap on the GPU
 * -- on two streams, or from two host threads -- race on the array.
 * Synchronises the stream.  Errors as for ttm_build_tensor_template.
 * ---------------------------------------------------------------------- */
#define TTM_NOALLOC_SCRATCH_BYTES 8388608
ttm_status ttm_build_tensor_template_noalloc(const float* d_template, const float* d_mask, int s,
                                             int n_order, const float* d_quats,
                                             const float* d_weights, int n_rot,
                                             float* d_components, ttm_tt_desc* desc, void* stream);

/* ------------------------------------------------------------------------
 * Plan.  A plan fixes a batch of problems; problem p matches volume p (size
 * vol_dims[3p..3p+2] = X, Y, Z) against template tmpl_index[p].  Template k
 * is described by descs[k], its components by d_components[k] (K x s^3,
 * caller-owned, read during ttm_plan only when the FFT path is chosen and
 * kept referenced by the direct path: they must stay valid until
 * ttm_plan_destroy) and its mask by d_masks[k] (s^3, read during ttm_plan).
 * Mask values lie in [0, 1] (else TTM_ERR_INVALID_ARG).  A binary mask
 * (0 or 1) allows every path.  A soft mask (weights, e.g. a raised-cosine
 * edge; the NCC becomes the m-weighted Pearson correlation of Sec. 2's
 * S-inner product) runs on the FFT path only, with FFT window sums: its
 * problems need an FFT box whose x length is one of the compiled lengths
 * 16 32 48 64 80 96 128 144 160 192 240 256 288 320 384 480 512 576 640 768
 * 960 1024, and TTM_PATH_DIRECT returns TTM_ERR_UNSUPPORTED.
 * opts may be NULL (defaults).  The plan allocates and owns only its tables
 * and precomputed template spectra.  Synchronises the stream.
 * Errors: TTM_ERR_INVALID_ARG (null pointer, volume smaller than its box,
 * template index out of range, mask values outside [0, 1], or an option out
 * of range: path, precision, negative counts, n_grid > 65535, n_cells not
 * dividing n_grid, n_candidates > 8, newton_steps > 64, n_refined > 4,
 * lowpass_sigma; all
 * checked before any device work), TTM_ERR_UNSUPPORTED (odd order or mixed
 * orders, n > 8, soft mask off the FFT path, volume of 2^31 voxels or more),
 * TTM_ERR_NUMERIC (non-finite components), TTM_ERR_OUT_OF_MEMORY,
 * TTM_ERR_CUDA.
 * ---------------------------------------------------------------------- */
ttm_status ttm_plan(ttm_plan_t* out, int n_problems, const int* vol_dims, const int* tmpl_index,
                    int n_templates, const ttm_tt_desc* descs, const float* const* d_components,
                    const float* const* d_masks, const ttm_plan_opts* opts, void* stream);

/* Bytes of device workspace ttm_local_stats, ttm_correlate and
 * ttm_extract_peaks need (one workspace serves all three). */
ttm_status ttm_plan_workspace_size(ttm_plan_t plan, size_t* bytes);

/* Path the plan chose for problem p (TTM_PATH_DIRECT or TTM_PATH_FFT). */
ttm_status ttm_plan_problem_path(ttm_plan_t plan, int problem, int* path);

/* Autotuner timings of problem p (TTM_PATH_TUNE): ms[0] = direct path,
 * ms[1] = FFT path (local statistics + K correlations, best of 2 runs), or
 * -1 where a path was not timed (the cost model decided).  Host-only. */
ttm_status ttm_plan_problem_tuning(ttm_plan_t plan, int problem, double* ms);

/* *on = 1 when problem p's direct correlation runs on the tensor cores (FP16
 * operands, TTM_PREC_MIXED), else 0.  Host-only. */
ttm_status ttm_plan_problem_tensor_direct(ttm_plan_t plan, int problem, int* on);

/* Padded FFT box of problem p: box[0..2] = (Xp, Yp, Zp), each the smallest
 * supported length 2^p 3^a 5^b (16..1024), else a power of two, not below
 * the volume's extent (circular correlation on the padded box equals the
 * linear one on the interior, Sec. 2 of the paper).  Zeros on the direct
 * path.  Host-only; TTM_ERR_INVALID_ARG for a bad plan, problem or pointer. */
ttm_status ttm_plan_problem_fft_box(ttm_plan_t plan, int problem, int* box);

/* Self-check of the bounded device-side waits (no counterpart in the paper:
 * engine infrastructure).  Launches one CTA that waits,
 * with the poll loop every tensor-core kernel waits with, on an mbarrier
 * phase: with arrive = 1 the CTA completes that phase itself first; with
 * arrive = 0 nothing does, so the wait must run out after `polls` polls
 * (1 .. 2^24).  *status_out receives TTM_OK (the phase completed) or
 * TTM_ERR_TIMEOUT (the wait ran out).  The kernel returns either way, so the
 * context stays usable.  Synchronises the stream.  Errors:
 * TTM_ERR_INVALID_ARG (polls out of range, null status_out), TTM_ERR_CUDA. */
ttm_status ttm_probe_bounded_wait(long long polls, int arrive, int* status_out, void* stream);

/* Kernel launches the plan has queued so far (for accounting). */
ttm_status ttm_plan_launch_count(ttm_plan_t plan, long long* launches);

/* Resident waves of the plan (option batch_mib; batching has no counterpart
 * in the paper, which matches one volume at a time): *n_waves = their number (0
 * when problems run one at a time); with first != NULL, first[0..n_waves-1]
 * receives the first problem of each wave (the caller sizes it from a call
 * with first = NULL).  Host-only; TTM_ERR_INVALID_ARG for a bad plan or
 * pointer. */
ttm_status ttm_plan_waves(ttm_plan_t plan, int* n_waves, int* first);

/* Status recorded by the device during the calls queued since the last
 * ttm_local_stats or ttm_correlate on this workspace (each starts by clearing
 * it; a bounded wait inside a kernel that ran out records TTM_ERR_TIMEOUT
 * there instead of hanging).  Synchronises the stream; returns TTM_OK or the
 * recorded error. */
ttm_status ttm_plan_device_status(ttm_plan_t plan, void* d_workspace, size_t workspace_bytes,
                                  void* stream);

/* Per-kernel timing.  With timing enabled the plan records a CUDA event pair
 * on the launch stream around every kernel it queues.  ttm_plan_timing waits
 * for those events, adds the elapsed times per kernel class into ms[c] and the
 * launch counts into launches[c] for c < n_classes (either array may be NULL),
 * and forgets them.  Class names come from ttm_kernel_class_name; there are
 * TTM_KERNEL_CLASSES classes.  The last, "rotation_stage", is not a kernel
 * but a span: the wall time of each problem's (or resident wave's)
 * score/rotation stage on the launch stream, with its search and refinement
 * overlapped on the plan's two rotation streams; its launches are counted in
 * their own classes as well. */
#define TTM_KERNEL_CLASSES 13
ttm_status ttm_plan_enable_timing(ttm_plan_t plan, int enable);
ttm_status ttm_plan_timing(ttm_plan_t plan, double* ms, long long* launches, int n_classes);
const char* ttm_kernel_class_name(int kernel_class);

/* Frees everything the plan owns.  NULL is ignored. */
void ttm_plan_destroy(ttm_plan_t plan);

/* ------------------------------------------------------------------------
 * Local statistics: the NCC denominators (Sec. 2,
 *   ||P_S tau_x f||_S^2 = <(tau_x f)^2, m> - <tau_x f, m>^2 / <1, m>,
 * and Algorithm 1, image block).  For every problem p writes
 *   w(x) = 1 / sqrt(S2(x) - S1(x)^2 / <1, m>),
 *   S1(x) = sum_u m(u) f(x + u - c),  S2(x) = sum_u m(u) f(x + u - c)^2,
 * into d_w[p] (X*Y*Z float32).  w = 0 outside the interior and where the
 * local variance S2 - S1^2/<1,m> is at most 1e-6 * <1,m> * var(f), var(f)
 * being the variance of the whole volume.  S1 and S2 are accumulated in FP32
 * after subtracting a per-tile reference value; the variance is formed in
 * FP64.  d_vols[p] is read, never written.
 * Errors: TTM_ERR_INVALID_ARG, TTM_ERR_WORKSPACE, TTM_ERR_CUDA.
 * ---------------------------------------------------------------------- */
ttm_status ttm_local_stats(ttm_plan_t plan, const float* const* d_vols, float* const* d_w,
                           void* d_workspace, size_t workspace_bytes, void* stream);

/* ------------------------------------------------------------------------
 * Correlation with the K components, TTM score and rotation (Sec. 3.2-3.4).
 * For every problem p and interior voxel x:
 *   C_alpha(x) = w(x) sum_u f(x + u - c) T_alpha(u)          (Sec. 3.2)
 *   score(x)   = ||C_n(x)||_F = sqrt(sum_alpha mu_alpha C_alpha^2),
 *                mu_alpha = n! / prod(multiplicities)         (Sec. 3.4)
 *   lambda(x)  = max_{|Q|=1} phi(Q), phi(Q) = sum_alpha mu_alpha C_alpha Q^alpha
 *   q(x)       = its maximiser, the dominant Z-eigenvector     (Sec. 3.3)
 * The maximum is searched on a fixed grid of n_grid unit quaternions split
 * into n_cells regions of equal size (for orders 4 and 6 with the default
 * grid this search runs on the tensor cores in FP16 with FP32 accumulation;
 * orders 2 and 8 search on the CUDA cores); the best grid point of each of the
 * n_candidates best regions is refined by shifted power iterations (shift
 * (n-1) score, Kolda & Mayo 2011), the best of them by Riemannian Newton
 * steps, and the largest refined value is kept.  q is canonical: a >= 0.
 *   d_w          from ttm_local_stats.
 *   d_score      X*Y*Z float32 per problem (required).
 *   d_quat       X*Y*Z*4 float32 per problem, (a,b,c,d) per voxel (required).
 *   d_lambda     X*Y*Z float32 per problem, or NULL.
 *   d_components_out  NULL, or per problem K*X*Y*Z float32 receiving C_alpha
 *                (component-major) for inspection.
 * Errors: TTM_ERR_INVALID_ARG, TTM_ERR_WORKSPACE, TTM_ERR_CUDA.
 * ---------------------------------------------------------------------- */
ttm_status ttm_correlate(ttm_plan_t plan, const float* const* d_vols, const float* const* d_w,
                         float* const* d_score, float* const* d_quat, float* const* d_lambda,
                         float* const* d_components_out, void* d_workspace,
                         size_t workspace_bytes, void* stream);

/* ------------------------------------------------------------------------
 * Classical template matching with rotations (Algorithm 1), the comparator of
 * TTM: for every rotation j of d_quats the template is rotated, masked and
 * S-normalised (exactly as in ttm_build_tensor_template), transformed, and
 * correlated with the volume through the FFT of the plan's problem; the NCC
 * c(x, R_j) = w(x) (f * S(t)_{R_j})(x) is reduced to its maximum over j,
 *   d_best[x] = max_j c(x, R_j),   d_best_index[x] = the first j attaining it.
 * Outside the interior both are 0.  Rotations run in batches of 32.
 *   problem      a problem of the plan that uses the FFT path.
 *   d_template   s^3 float32 raw template (s of the problem's template).
 *   d_quats      n_rot x 4 float32 unit quaternions.
 *   d_vol, d_w   the problem's volume and its w from ttm_local_stats.
 *   d_best       X*Y*Z float32 output; d_best_index X*Y*Z int32 output.
 * Errors: TTM_ERR_INVALID_ARG, TTM_ERR_UNSUPPORTED (direct-path problem),
 * TTM_ERR_WORKSPACE, TTM_ERR_NUMERIC (a rotated copy has zero variance),
 * TTM_ERR_CUDA.
 * ---------------------------------------------------------------------- */
ttm_status ttm_classical_workspace_size(ttm_plan_t plan, int problem, size_t* bytes);
ttm_status ttm_classical_ncc(ttm_plan_t plan, int problem, const float* d_template,
                             const float* d_quats, int n_rot, const float* d_vol,
                             const float* d_w, float* d_best, int* d_best_index,
                             void* d_workspace, size_t workspace_bytes, void* stream);

/* ------------------------------------------------------------------------
 * Peaks of the position score (Sec. 3.4).  A voxel is a peak when its score
 * exceeds threshold and beats every other voxel of the (2*radius+1)^3 cube
 * around it (equal scores: the lower linear index wins).  Up to max_peaks
 * peaks, highest score first (equal scores: lower index first), are written
 * to h_out with their lambda and quaternion; *n_out receives the count.
 * d_lambda may be NULL (lambda reported as 0).  Synchronises the stream.
 * Errors: TTM_ERR_INVALID_ARG (radius < 0 or > 32, max_peaks < 0),
 * TTM_ERR_WORKSPACE, TTM_ERR_CUDA.
 * ---------------------------------------------------------------------- */
ttm_status ttm_extract_peaks(ttm_plan_t plan, int problem, const float* d_score,
                             const float* d_quat, const float* d_lambda, float threshold,
                             int radius, int max_peaks, ttm_peak* h_out, int* n_out,
                             void* d_workspace, size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * ttm_lowpass -- the optional isotropic prefilter h of Sec. 2 (t' = h * t,
 * f' = h * f, h * 1 = 1): a sampled Gaussian of unit sum, radius
 * int(4 sigma + 0.5) <= 32, applied along x, y and z in turn as a linear
 * convolution with zero outside the X*Y*Z array (as scipy's gaussian_filter
 * with mode "constant" and truncate 4).  d_in, d_tmp (scratch) and d_out are
 * distinct device arrays of X*Y*Z floats.  Use it on a template before
 * ttm_build_tensor_template when the plan's lowpass_sigma is set; the plan
 * filters the volumes itself.  Asynchronous.  TTM_ERR_INVALID_ARG for a bad
 * pointer, size or sigma.
 * ------------------------------------------------------------------------ */
ttm_status ttm_lowpass(const float* d_in, int X, int Y, int Z, float sigma, float* d_tmp,
                       float* d_out, void* stream);

/* ---------------------------------------------------------------------------
 * ttm_match_peaks -- the score map and the rotations at its peaks only (the
 * paper's own use of the two outputs, Sec. 3.4: the Frobenius norm locates
 * candidate positions, the dominant Z-eigenvector is computed there).
 *
 * For problem p: the K correlations of d_vol (as ttm_correlate, using the w
 * map d_w from ttm_local_stats), the score map into d_score (X*Y*Z floats,
 * 0 outside the interior), its local maxima exactly as ttm_extract_peaks
 * (score > threshold, largest in the (2 nms_radius + 1)^3 cube, equal scores
 * to the lower linear index), and then the rotation search and refinement of
 * ttm_correlate at those voxels only.  Up to max_peaks records sorted by
 * score go to h_out (host); *n_out is their number.  q and lambda of a record
 * are bit-identical to the maps ttm_correlate writes at that voxel.  No
 * rotation or lambda map is written.  Synchronises the stream.  Errors: as
 * ttm_extract_peaks, and a device status (TTM_ERR_TIMEOUT) of this call.
 * ------------------------------------------------------------------------ */
ttm_status ttm_match_peaks(ttm_plan_t plan, int problem, const float* d_vol, const float* d_w,
                           float* d_score, float threshold, int nms_radius, int max_peaks,
                           ttm_peak* h_out, int* n_out, void* d_workspace, size_t workspace_bytes,
                           void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TTM_H_ */
