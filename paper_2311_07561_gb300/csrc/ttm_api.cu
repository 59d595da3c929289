// C ABI of the engine (declared in include/ttm.h): argument validation, plan
// construction (mask runs, tap-major template tables, rotation search grid),
// workspace layout and dispatch of the kernels.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "ttm_internal.h"

namespace ttm {

namespace {
thread_local char g_last_error[256] = {0};
}

void note_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%s:%d)", what, cudaGetErrorString(e),
             file, line);
}

ttm_status after_launch(long long* counter) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        note_cuda_error(e, "kernel launch", __FILE__, __LINE__);
        return TTM_ERR_CUDA;
    }
    if (counter) ++*counter;
    return TTM_OK;
}

namespace {

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

// Super-Fibonacci spiral on S^3 (Alexa, CVPR 2022): point i uses s = i + 1/2,
// radii sqrt(s/n), sqrt(1 - s/n) and angles 2 pi s / sqrt(2), 2 pi s / psi
// with psi^4 = psi + 4.  Every point is flipped to the half sphere a >= 0.
void half_sphere_points(int n, std::vector<double>& q) {
    const double psi = 1.533751168755204288118041;
    const double phi = std::sqrt(2.0);
    const double two_pi = 6.283185307179586476925287;
    q.assign((size_t)4 * n, 0.0);
    for (int i = 0; i < n; ++i) {
        double s = i + 0.5;
        double r = std::sqrt(s / n), R = std::sqrt(1.0 - s / n);
        double al = two_pi * s / phi, be = two_pi * s / psi;
        double v[4] = {r * std::sin(al), r * std::cos(al), R * std::sin(be), R * std::cos(be)};
        double nn = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2] + v[3] * v[3]);
        double sg = v[0] < 0 ? -1.0 : 1.0;
        for (int k = 0; k < 4; ++k) q[4 * i + k] = sg * v[k] / nn;
    }
}

// Exponent vectors and multinomial weights of S^n(R^4) in C-ABI order
// (host-side enumeration for the tables built at plan time).
void sym_table(int n, std::vector<int>& e, std::vector<double>& mu) {
    e.clear();
    mu.clear();
    std::vector<int> t(n, 0);
    auto fact = [](int k) { double r = 1; for (int i = 2; i <= k; ++i) r *= i; return r; };
    while (true) {
        int ex[4] = {0, 0, 0, 0};
        for (int p = 0; p < n; ++p) ex[t[p]]++;
        for (int i = 0; i < 4; ++i) e.push_back(ex[i]);
        mu.push_back(fact(n) / (fact(ex[0]) * fact(ex[1]) * fact(ex[2]) * fact(ex[3])));
        int p = n - 1;
        while (p >= 0 && t[p] == 3) --p;
        if (p < 0) break;
        t[p]++;
        for (int k = p + 1; k < n; ++k) t[k] = t[p];
    }
}

template <typename T>
ttm_status dev_upload(T** dst, const std::vector<T>& src) {
    *dst = nullptr;
    if (src.empty()) return TTM_OK;
    cudaError_t e = cudaMalloc((void**)dst, src.size() * sizeof(T));
    if (e != cudaSuccess) {
        note_cuda_error(e, "cudaMalloc", __FILE__, __LINE__);
        cudaGetLastError();
        return TTM_ERR_OUT_OF_MEMORY;
    }
    TTM_CUDA_TRY(cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
    return TTM_OK;
}

ttm_status build_grid(ttm_plan_s* P) {
    RotGrid& g = P->grid;
    // mixed precision searches 1024 points (64 regions of 16): the FP64 model
    // of the search and refinement gives a largest lambda shortfall of 6.2e-5
    // at order 6 (4.2e-5 with 2048 points) and 8.4e-5 at order 4 (1.7e-5),
    // inside that mode's 5e-3 tolerance; FP32 keeps 2048 for its 1e-4
    const int n_def = P->opts.precision == TTM_PREC_MIXED ? 1024 : 2048;
    const int n = P->opts.n_grid > 0 ? P->opts.n_grid : n_def;
    const int nc = P->opts.n_cells > 0 ? P->opts.n_cells : n / 16;
    // refinement budget: at order 6 the maxima of phi are sharper and the
    // grid search lands closer; an FP64 model of the search and refinement
    // (the unit tests' model, on 400 voxels of the 928 x 928 x 464 workload's
    // template) gives the same largest lambda shortfall (4.2e-5 with 2048
    // grid points, 6.2e-5 with 1024: grid misses) with 2 candidates x 2
    // refined x 2 Newton steps as with 8 x 4 x 3.  At order 4 the FP64 model
    // allows 3 x 2 x 3 as well, but the FP16 grid search ranks near-tied
    // regions differently (2.4e-4 key resolution of the normalised phi): at
    // a peak of a 200-rotation template the GPU then refined the wrong
    // maximum (lambda 2.1e-5 short), so order 4 keeps 8 x 4 x 3
    const bool o6 = P->n_order == 6;
    const int cand = P->opts.n_candidates > 0 ? P->opts.n_candidates : (o6 ? 2 : 8);
    const int newton = P->opts.newton_steps > 0 ? P->opts.newton_steps : (o6 ? 2 : 3);
    const int refine = P->opts.n_refined > 0 ? P->opts.n_refined : (o6 ? 2 : 4);
    if (n > 65535 || nc > n || n % nc != 0 || cand > 8 || newton > 64 || refine > 4)
        return TTM_ERR_INVALID_ARG;
    std::vector<double> pts, ctr;
    half_sphere_points(n, pts);
    half_sphere_points(nc, ctr);
    std::vector<int> label(n);
    for (int i = 0; i < n; ++i) {
        double best = -1.0;
        int bl = 0;
        for (int c = 0; c < nc; ++c) {
            double d = std::fabs(pts[4 * i] * ctr[4 * c] + pts[4 * i + 1] * ctr[4 * c + 1] +
                                 pts[4 * i + 2] * ctr[4 * c + 2] + pts[4 * i + 3] * ctr[4 * c + 3]);
            if (d > best) { best = d; bl = c; }
        }
        label[i] = bl;
    }
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return label[a] < label[b]; });
    std::vector<int> e;
    std::vector<double> mu;
    sym_table(P->n_order, e, mu);
    const int K = (int)mu.size();
    const int K4 = rotation_row_stride(P->n_order);
    std::vector<float> hq((size_t)4 * n), hm((size_t)K4 * n, 0.f);
    std::vector<int> ends(n);
    for (int g_i = 0; g_i < n; ++g_i) {
        const double* q = &pts[4 * order[g_i]];
        for (int k = 0; k < 4; ++k) hq[4 * g_i + k] = (float)q[k];
        for (int a = 0; a < K; ++a) {
            double v = mu[a];
            for (int i = 0; i < 4; ++i)
                for (int r = 0; r < e[4 * a + i]; ++r) v *= q[i];
            hm[(size_t)g_i * K4 + a] = (float)v;
        }
        // regions: consecutive groups of n / nc points in nearest-centre order
        ends[g_i] = ((g_i + 1) % (n / nc) == 0) ? 1 : 0;
    }
    g.n_grid = n;
    g.n_cells = nc;
    g.n_cand = cand;
    g.newton = newton;
    g.n_refine = refine;
    TTM_TRY(dev_upload(&g.d_q, hq));
    TTM_TRY(dev_upload(&g.d_m, hm));
    TTM_TRY(dev_upload(&g.d_cell_end, ends));
    if (search_tc_supported(P->n_order, n, nc)) {
        std::vector<uint16_t> tab;
        build_grid_fp16(hm.data(), K, K4, n, tab);
        std::vector<uint32_t> bits(n / 32, 0u);
        for (int i = 0; i < n; ++i)
            if (ends[i]) bits[i / 32] |= 1u << (i % 32);
        TTM_TRY(dev_upload(&g.d_gtab, tab));
        TTM_TRY(dev_upload(&g.d_endbits, bits));
    }
    return TTM_OK;
}

// Mask -> x-runs and tap-major component table.
ttm_status prepare_template(ttm_plan_s* P, TemplateData& T, const float* d_mask) {
    const int s = T.desc.s, c = T.desc.centre, K = T.desc.K;
    const size_t s3 = (size_t)s * s * s;
    std::vector<float> m(s3), comp((size_t)K * s3);
    TTM_CUDA_TRY(cudaMemcpy(m.data(), d_mask, s3 * sizeof(float), cudaMemcpyDeviceToHost));
    TTM_CUDA_TRY(cudaMemcpy(comp.data(), T.d_comp, comp.size() * sizeof(float),
                            cudaMemcpyDeviceToHost));
    bool any = false;
    T.soft = false;
    for (float v : m) {
        if (!(v >= 0.f && v <= 1.f)) return TTM_ERR_INVALID_ARG;      // also NaN
        if (v != 0.f && v != 1.f) T.soft = true;
        any = any || v > 0.f;
    }
    if (!any) return TTM_ERR_INVALID_ARG;
    for (float v : comp)
        if (!std::isfinite(v)) return TTM_ERR_NUMERIC;
    if (T.soft) {
        // a soft (weighting) mask: the correlations and the window sums run
        // through the FFT only; no runs or taps for the direct paths
        (void)P;
        TTM_TRY(dev_upload(&T.d_mask, m));
        return TTM_OK;
    }
    std::vector<MaskRun> runs;
    std::vector<int> tap0;
    std::vector<float> taps;
    int ntap = 0;
    for (int uz = 0; uz < s; ++uz)
        for (int uy = 0; uy < s; ++uy) {
            int ux = 0;
            while (ux < s) {
                if (m[((size_t)uz * s + uy) * s + ux] != 1.f) { ++ux; continue; }
                int u1 = ux;
                while (u1 + 1 < s && m[((size_t)uz * s + uy) * s + u1 + 1] == 1.f) ++u1;
                MaskRun r{uy - c, uz - c, ux - c, u1 - c};
                runs.push_back(r);
                tap0.push_back(ntap);
                for (int xx = ux; xx <= u1; ++xx) {
                    for (int a = 0; a < K; ++a)
                        taps.push_back(comp[(size_t)a * s3 + ((size_t)uz * s + uy) * s + xx]);
                    ++ntap;
                }
                ux = u1 + 1;
            }
        }
    if (runs.empty()) return TTM_ERR_INVALID_ARG;
    T.runs = runs;
    T.n_taps = ntap;
    T.dz_min = T.dy_min = T.x_min = 1 << 30;
    T.dz_max = T.dy_max = T.x_max = -(1 << 30);
    for (const MaskRun& r : runs) {
        T.dz_min = std::min(T.dz_min, r.dz); T.dz_max = std::max(T.dz_max, r.dz);
        T.dy_min = std::min(T.dy_min, r.dy); T.dy_max = std::max(T.dy_max, r.dy);
        T.x_min = std::min(T.x_min, r.x0); T.x_max = std::max(T.x_max, r.x1);
    }
    std::vector<int> dz0(T.dz_max - T.dz_min + 2, 0);
    {
        size_t k = 0;
        for (int dz = T.dz_min; dz <= T.dz_max; ++dz) {
            dz0[dz - T.dz_min] = (int)k;
            while (k < runs.size() && runs[k].dz == dz) ++k;
        }
        dz0[T.dz_max - T.dz_min + 1] = (int)runs.size();
    }
    (void)P;
    TTM_TRY(dev_upload(&T.d_mask, m));
    TTM_TRY(dev_upload(&T.d_runs, runs));
    TTM_TRY(dev_upload(&T.d_run_tap0, tap0));
    TTM_TRY(dev_upload(&T.d_dz_run0, dz0));
    TTM_TRY(dev_upload(&T.d_taps, taps));
    if (direct_tc_supported(K, ntap)) {
        // tensor-core direct path: FP16 component table and per-tap offsets
        std::vector<uint16_t> tab;
        build_direct_tc_table(taps, ntap, K, tab, &T.tc_scale);
        const int ntp = (int)(tab.size() / (size_t)direct_tc_columns(K));
        std::vector<int> dxyz(ntp, 64 | (64 << 8) | (64 << 16));      // padded taps: offset 0
        int t_i = 0;
        for (const MaskRun& r : runs)
            for (int dx = r.x0; dx <= r.x1; ++dx)
                dxyz[t_i++] = (dx + 64) | ((r.dy + 64) << 8) | ((r.dz + 64) << 16);
        TTM_TRY(dev_upload(&T.d_tc_tab, tab));
        TTM_TRY(dev_upload(&T.d_tap_dxyz, dxyz));
    }
    return TTM_OK;
}

const float2* twiddle_table(ttm_plan_s* P, int L, ttm_status* err) {
    for (auto& t : P->twiddles)
        if (t.first == L) return t.second;
    std::vector<float2> h(L);
    const double two_pi = 6.283185307179586476925287;
    for (int k = 0; k < L; ++k) {
        double a = -two_pi * (double)k / (double)L;
        h[k] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    float2* d = nullptr;
    *err = dev_upload(&d, h);
    if (*err != TTM_OK) return nullptr;
    P->twiddles.push_back({L, d});
    return d;
}

// Cost model of the two correlation paths (ns per voxel): the FFT path moves
// ~40 bytes per component per padded voxel at ~5 TB/s, the direct path does
// 2 K n_taps FLOP at ~30 TFLOP/s on the CUDA cores, or 2 N n_taps FLOP (N = K
// padded to 16) at ~150 TFLOP/s effective on the tensor cores.
double model_ratio(const ttm_plan_s* P, const ProblemData& pr, const TemplateData& T) {
    const double pad = (double)pr.fft.Xp * pr.fft.Yp * pr.fft.Zp / (double)pr.nvox();
    const double fft_ns = pad * (40.0 * P->K + 40.0) / 5000.0;
    double direct_ns = 2.0 * P->K * T.n_taps / 30000.0;
    if (P->opts.precision == TTM_PREC_MIXED && T.d_tc_tab)      // tensor cores, FP16 operands
        direct_ns = 2.0 * direct_tc_columns(P->K) * T.n_taps / 150000.0;
    return direct_ns / fft_ns;          // > 1: the FFT path is expected to win
}

bool prefer_fft(const ttm_plan_s* P, const ProblemData& pr, const TemplateData& T) {
    return model_ratio(P, pr, T) > 1.0;
}

// The autotuner times both paths only where the model leaves them within
// this factor of each other.
constexpr double kTuneRange = 8.0;

ttm_status prepare_fft(ttm_plan_s* P, ProblemData& pr, cudaStream_t st) {
    ttm_status err = TTM_OK;
    pr.fft.Xp = fft_good_length(pr.X);
    pr.fft.Yp = fft_good_length(pr.Y);
    pr.fft.Zp = fft_good_length(pr.Z);
    if (!fft_length_ok(pr.fft.Xp) || !fft_length_ok(pr.fft.Yp) || !fft_length_ok(pr.fft.Zp))
        return TTM_ERR_UNSUPPORTED;
    pr.fft.d_tw_x = twiddle_table(P, pr.fft.Xp, &err); TTM_TRY(err);
    pr.fft.d_tw_y = twiddle_table(P, pr.fft.Yp, &err); TTM_TRY(err);
    pr.fft.d_tw_z = twiddle_table(P, pr.fft.Zp, &err); TTM_TRY(err);
    for (size_t i = 0; i < P->specs.size(); ++i) {
        const SpecSet& sp = P->specs[i];
        if (sp.tmpl == pr.tmpl && sp.Xp == pr.fft.Xp && sp.Yp == pr.fft.Yp && sp.Zp == pr.fft.Zp &&
            sp.mixed == pr.mixed) {
            pr.spec_index = (int)i;
            return TTM_OK;
        }
    }
    const TemplateData& T = P->tmpl[pr.tmpl];
    SpecSet sp;
    sp.tmpl = pr.tmpl; sp.Xp = pr.fft.Xp; sp.Yp = pr.fft.Yp; sp.Zp = pr.fft.Zp; sp.mixed = pr.mixed;
    const size_t nspec = pr.fft.nspec();
    const size_t nreal = (size_t)pr.fft.Xp * pr.fft.Yp * pr.fft.Zp;
    const size_t s3 = (size_t)T.desc.s * T.desc.s * T.desc.s;
    bool oom = cudaMalloc((void**)&sp.d_mask_spec, nspec * sizeof(float2)) != cudaSuccess;
    if (!oom) {
        if (pr.mixed)
            oom = cudaMalloc(&sp.d_spec_bf, (size_t)P->K * nspec * 4) != cudaSuccess;
        else
            oom = cudaMalloc((void**)&sp.d_spec, (size_t)P->K * nspec * sizeof(float2)) != cudaSuccess;
    }
    P->specs.push_back(sp);   // freed with the plan, also on failure
    if (oom) { cudaGetLastError(); return TTM_ERR_OUT_OF_MEMORY; }
    pr.spec_index = (int)P->specs.size() - 1;
    float* pad = nullptr;
    float2* tmp = nullptr;
    if (cudaMalloc((void**)&pad, nreal * sizeof(float)) != cudaSuccess ||
        (pr.mixed && cudaMalloc((void**)&tmp, nspec * sizeof(float2)) != cudaSuccess)) {
        cudaGetLastError();
        cudaFree(pad);
        return TTM_ERR_OUT_OF_MEMORY;
    }
    ttm_status s = launch_template_spectra(T.d_mask, 1, T.desc.s, pr.fft, pad, sp.d_mask_spec, st,
                                           &P->launches);
    if (!pr.mixed) {
        if (s == TTM_OK)
            s = launch_template_spectra(T.d_comp, P->K, T.desc.s, pr.fft, pad, sp.d_spec, st,
                                        &P->launches);
    } else {
        for (int k = 0; k < P->K && s == TTM_OK; ++k) {
            s = launch_template_spectra(T.d_comp + (size_t)k * s3, 1, T.desc.s, pr.fft, pad, tmp,
                                        st, &P->launches);
            if (s == TTM_OK)
                s = launch_spectra_to_bf16(tmp, (char*)sp.d_spec_bf + (size_t)k * nspec * 4, nspec,
                                           st, &P->launches);
        }
    }
    cudaError_t e = cudaStreamSynchronize(st);
    cudaFree(pad);
    cudaFree(tmp);
    if (s != TTM_OK) return s;
    if (e != cudaSuccess) { cudaGetLastError(); return TTM_ERR_CUDA; }
    return TTM_OK;
}

cudaEvent_t pool_event(ttm_plan_s* P) {
    if (!P->event_pool.empty()) {
        cudaEvent_t e = P->event_pool.back();
        P->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

// Runs fn (which queues kernels on st); with timing on, brackets it with an
// event pair attributed to kernel class cls.
template <typename F>
ttm_status timed(ttm_plan_s* P, int cls, cudaStream_t st, F&& fn) {
    if (!P->timing) return fn();
    cudaEvent_t a = pool_event(P), b = pool_event(P);
    if (!a || !b) return TTM_ERR_CUDA;
    TTM_CUDA_TRY(cudaEventRecord(a, st));
    const long long before = P->launches;
    ttm_status s = fn();
    TTM_CUDA_TRY(cudaEventRecord(b, st));
    P->timed.push_back(TimedLaunch{cls, a, b, P->launches - before});
    return s;
}

void free_plan(ttm_plan_s* P) {
    for (TimedLaunch& t : P->timed) {
        cudaEventDestroy(t.start);
        cudaEventDestroy(t.stop);
    }
    for (cudaEvent_t e : P->event_pool) cudaEventDestroy(e);
    for (cudaEvent_t e : P->ev_chunk) cudaEventDestroy(e);
    if (P->ev_fork) cudaEventDestroy(P->ev_fork);
    if (P->ev_join) cudaEventDestroy(P->ev_join);
    if (P->s_hi) cudaStreamDestroy(P->s_hi);
    if (P->s_lo) cudaStreamDestroy(P->s_lo);
    for (TemplateData& T : P->tmpl) {
        cudaFree(T.d_runs);
        cudaFree(T.d_mask);
        cudaFree(T.d_run_tap0);
        cudaFree(T.d_dz_run0);
        cudaFree(T.d_taps);
        cudaFree(T.d_tc_tab);
        cudaFree(T.d_tap_dxyz);
        cudaFree(T.d_spec);
    }
    for (SpecSet& sp : P->specs) {
        cudaFree(sp.d_spec);
        cudaFree(sp.d_spec_bf);
        cudaFree(sp.d_mask_spec);
    }
    for (auto& t : P->twiddles) cudaFree(t.second);
    cudaFree(P->grid.d_q);
    cudaFree(P->grid.d_m);
    cudaFree(P->grid.d_cell_end);
    cudaFree(P->grid.d_gtab);
    cudaFree(P->grid.d_endbits);
    delete P;
}

// Streams and events of the pipelined rotation stage (rotation_chunks > 1).
ttm_status make_rotation_streams(ttm_plan_s* P) {
    const int nch = P->opts.rotation_chunks > 0 ? P->opts.rotation_chunks : 8;
    if (nch > 64) return TTM_ERR_INVALID_ARG;
    P->rot_chunks = nch;
    if (nch == 1) return TTM_OK;
    int least = 0, greatest = 0;
    TTM_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    TTM_CUDA_TRY(cudaStreamCreateWithPriority(&P->s_hi, cudaStreamNonBlocking, greatest));
    TTM_CUDA_TRY(cudaStreamCreateWithPriority(&P->s_lo, cudaStreamNonBlocking, least));
    TTM_CUDA_TRY(cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming));
    TTM_CUDA_TRY(cudaEventCreateWithFlags(&P->ev_join, cudaEventDisableTiming));
    P->ev_chunk.assign(nch, nullptr);
    for (int c = 0; c < nch; ++c)
        TTM_CUDA_TRY(cudaEventCreateWithFlags(&P->ev_chunk[c], cudaEventDisableTiming));
    return TTM_OK;
}

// workspace layout: [0, 256) header (moments, counters); [256, ...) scratch
constexpr size_t kHeader = 256;
constexpr int kPeakCapMax = 1 << 22;

size_t peak_cap(size_t nvox) { return std::min(nvox, (size_t)kPeakCapMax); }

// Correlation maps first (both paths), then for the FFT path the image
// spectrum and the K product spectra, then 8 candidate grid indices per voxel.
// Components per inverse-FFT group: the product spectra of one group live in
// the workspace at a time (all K while they fit in 8 GiB, fewer for large
// boxes), so the workspace holds the K correlation maps plus one group.
constexpr size_t kProdBudget = (size_t)8 << 30;

int comp_group(const ttm_plan_s* P, const ProblemData& pr) {
    const size_t per = pr.fft.nspec() * 2 * (pr.mixed ? 2 : 4);
    const size_t g = per ? kProdBudget / per : (size_t)P->K;
    return (int)std::max<size_t>(1, std::min<size_t>(g, (size_t)P->K));
}

size_t corr_region_bytes(const ttm_plan_s* P, const ProblemData& pr) {
    const size_t es = pr.mixed ? 2 : 4;          // bytes per stored real (corr maps)
    size_t b = align256((size_t)P->K * pr.nvox() * es);
    if (pr.path == TTM_PATH_FFT)
        b += align256(pr.fft.nspec() * sizeof(float2)) +
             align256((size_t)comp_group(P, pr) * pr.fft.nspec() * 2 * es);
    return b;
}

size_t scratch_bytes(const ttm_plan_s* P, const ProblemData& pr) {
    const size_t nv = pr.nvox();
    size_t corr = corr_region_bytes(P, pr) + align256(nv * 16);
    if (pr.path == TTM_PATH_FFT)
        corr = std::max(corr, 4 * pr.fft.nspec() * sizeof(float2) + 2 * nv * sizeof(float) + 256);
    size_t peaks = 2 * align256(nv * sizeof(float)) + align256(peak_cap(nv) * peak_record_bytes());
    // ttm_match_peaks keeps the correlation maps and candidates while it finds peaks
    const size_t corr_peaks = corr_region_bytes(P, pr) + align256(nv * 16) + peaks;
    return std::max(std::max(corr, peaks), corr_peaks);
}

// Where one problem's correlation stage keeps its data in the workspace: the
// K maps, the image spectrum and one group of product spectra (FFT path),
// and the search candidates.  One problem at a time, everything sits at the
// start of the scratch; with resident waves (plan option batch_mib) each
// problem of a wave has its own maps and candidates, and the spectra sit in
// a scratch area after the wave's maps.
struct CorrLayout {
    char* corr = nullptr;
    char* spec = nullptr;
    char* prod = nullptr;
    uint16_t* cand = nullptr;
};

CorrLayout corr_layout(const ttm_plan_s* P, const ProblemData& pr, void* ws, bool resident) {
    CorrLayout L;
    const size_t es = pr.mixed ? 2 : 4;
    char* base = (char*)ws;
    if (resident) {
        L.corr = base + pr.res_corr_off;
        L.cand = (uint16_t*)(base + pr.res_cand_off);
        L.spec = base + P->wave_scratch_off;
    } else {
        L.corr = base + kHeader;
        L.cand = (uint16_t*)(L.corr + corr_region_bytes(P, pr));
        L.spec = L.corr + align256((size_t)P->K * pr.nvox() * es);
    }
    L.prod = L.spec + align256(pr.fft.nspec() * sizeof(float2));
    return L;
}

// Resident waves: consecutive problems with the same map type whose maps
// and candidates fit in batch_mib MiB together (a problem larger than that
// is a wave of its own).  Offsets from kHeader; the spectra scratch of the
// FFT problems follows the largest wave.
size_t resident_bytes(const ttm_plan_s* P, const ProblemData& pr, size_t* cand_off) {
    const size_t es = pr.mixed ? 2 : 4;
    const size_t maps = align256((size_t)P->K * pr.nvox() * es);
    const VoxBox box = interior_box(pr.X, pr.Y, pr.Z, P->tmpl[pr.tmpl].desc.s);
    if (cand_off) *cand_off = maps;
    return maps + align256(box.count() * 16);
}

size_t wave_scratch_bytes(const ttm_plan_s* P) {
    size_t b = 0;
    for (const ProblemData& pr : P->prob)
        if (pr.path == TTM_PATH_FFT)
            b = std::max(b, align256(pr.fft.nspec() * sizeof(float2)) +
                                align256((size_t)comp_group(P, pr) * pr.fft.nspec() * 2 *
                                         (pr.mixed ? 2 : 4)));
    return b;
}

void plan_waves(ttm_plan_s* P) {
    const size_t budget = (size_t)P->opts.batch_mib << 20;
    const int np = (int)P->prob.size();
    P->waves.clear();
    size_t acc = 0, largest = 0;
    int w0 = 0;
    for (int p = 0; p < np; ++p) {
        ProblemData& pr = P->prob[p];
        size_t cand_off = 0;
        const size_t need = resident_bytes(P, pr, &cand_off);
        if (p > w0 && (acc + need > budget || pr.mixed != P->prob[w0].mixed)) {
            P->waves.emplace_back(w0, p);
            w0 = p;
            acc = 0;
        }
        pr.res_corr_off = kHeader + acc;
        pr.res_cand_off = kHeader + acc + cand_off;
        acc += need;
        largest = std::max(largest, acc);
    }
    P->waves.emplace_back(w0, np);
    P->wave_scratch_off = kHeader + largest;
}

ttm_status check_ws(const ttm_plan_s* P, void* ws, size_t bytes) {
    if (!ws || bytes < P->ws_bytes) return TTM_ERR_WORKSPACE;
    if (!aligned(ws, 256)) return TTM_ERR_INVALID_ARG;
    return TTM_OK;
}

// ---- per-problem steps (shared by the C ABI and the plan-time tuner) ----

// The volume the method works on: vol itself, or h * vol (the plan's
// Gaussian prefilter, Sec. 2) in the problem's workspace slot.
ttm_status prefilter(ttm_plan_s* plan, const ProblemData& pr, const float* vol, void* d_workspace,
                     cudaStream_t st, const float** out) {
    if (!(plan->opts.lowpass_sigma > 0.f)) {
        *out = vol;
        return TTM_OK;
    }
    float* dst = (float*)((char*)d_workspace + pr.lp_off);
    float* tmp = (float*)((char*)dst + align256(pr.nvox() * sizeof(float)));
    TTM_TRY(launch_lowpass(vol, pr.X, pr.Y, pr.Z, plan->opts.lowpass_sigma, tmp, dst, st,
                           &plan->launches));
    *out = dst;
    return TTM_OK;
}

// problems a and b read the same volume (same pointer, no prefilter, same
// extents and FFT box)
bool same_volume(const ttm_plan_s* P, int a, int b, const float* const* d_vols) {
    const ProblemData &x = P->prob[a], &y = P->prob[b];
    return d_vols[a] == d_vols[b] && !(P->opts.lowpass_sigma > 0.f) && x.X == y.X &&
           x.Y == y.Y && x.Z == y.Z && x.fft.Xp == y.fft.Xp && x.fft.Yp == y.fft.Yp &&
           x.fft.Zp == y.fft.Zp;
}

bool stats_on_fft(const ProblemData& pr) {
    return pr.path == TTM_PATH_FFT && fft_template_length(pr.fft.Xp);
}

// What the previous problem of a ttm_local_stats call left in the workspace
// for this one (same volume): nothing, the volume's moments, or the moments
// and the spectra of f - mean and (f - mean)^2 (same FFT box, FFT sums).
enum StatsReuse { kReuseNone = 0, kReuseMoments = 1, kReuseSpectra = 2 };

// w for one problem (Algorithm 1, image block): FFT window sums when the
// problem takes the FFT path with a compile-time x length, else run sums.
ttm_status stats_problem(ttm_plan_s* plan, const ProblemData& pr, const float* vol, float* w,
                         void* d_workspace, cudaStream_t st, int reuse = kReuseNone) {
    // header: sum f, sum f^2, sum (f - mean)^4, flagged-window counter
    double* d_mom = (double*)d_workspace;
    unsigned int* d_flagged = (unsigned int*)((char*)d_workspace + 24);
    if (reuse == kReuseNone) {
        TTM_CUDA_TRY(cudaMemsetAsync(d_mom, 0, 4 * sizeof(double), st));
        TTM_TRY(timed(plan, KC_MOMENTS, st, [&] {
            return launch_volume_moments(vol, pr.nvox(), d_mom, st, &plan->launches);
        }));
    } else if (reuse == kReuseMoments) {
        // the fourth moment comes with the spectra: zero it and the counter
        TTM_CUDA_TRY(cudaMemsetAsync(d_mom + 2, 0, 2 * sizeof(double), st));
    } else {
        TTM_CUDA_TRY(cudaMemsetAsync(d_flagged, 0, sizeof(unsigned int), st));
    }
    const TemplateData& T = plan->tmpl[pr.tmpl];
    if (stats_on_fft(pr)) {
        // window sums of (f - mean) and (f - mean)^2 as correlations with the mask
        const size_t nspec = pr.fft.nspec();
        char* base = (char*)d_workspace + kHeader;
        float2* F1 = (float2*)base;
        float2* F2 = F1 + nspec;
        float2* prod = F2 + nspec;                       // two product spectra
        float* sums = (float*)(prod + 2 * nspec);        // S1, S2 maps
        const float2* mspec = plan->specs[pr.spec_index].d_mask_spec;
        return timed(plan, KC_LOCAL_STATS, st, [&] {
            if (reuse != kReuseSpectra) {
                TTM_TRY(launch_fft_forward(vol, pr.X, pr.Y, pr.Z, pr.fft, F1, st,
                                           &plan->launches, 1, d_mom));
                TTM_TRY(launch_fft_forward(vol, pr.X, pr.Y, pr.Z, pr.fft, F2, st,
                                           &plan->launches, 2, d_mom));
            }
            // the sums are read on the interior only
            const FftKeep keep = fft_keep_interior(pr.X, pr.Y, pr.Z, T.desc.s);
            TTM_TRY(launch_fft_spectrum_inverse_z(F1, mspec, 1, pr.fft, prod, keep, st,
                                                  &plan->launches));
            TTM_TRY(launch_fft_spectrum_inverse_z(F2, mspec, 1, pr.fft, prod + nspec, keep, st,
                                                  &plan->launches));
            TTM_TRY(launch_fft_inverse_yx(prod, 2, pr.X, pr.Y, pr.Z, pr.fft, sums,
                                          (int*)((char*)d_workspace + 32), keep, st,
                                          &plan->launches));
            TTM_TRY(launch_stats_from_sums(sums, sums + pr.nvox(), w, pr.X, pr.Y, pr.Z, T.desc.s,
                                           T.desc.mask_sum, d_mom, d_flagged, st,
                                           &plan->launches));
            // windows whose FP32 sums are not accurate enough: exact FP64 sums
            return launch_exact_stats(vol, w, pr.X, pr.Y, pr.Z, T, d_mom, d_flagged, st,
                                      &plan->launches);
        });
    }
    return timed(plan, KC_LOCAL_STATS, st, [&] {
        return launch_local_stats(vol, pr.X, pr.Y, pr.Z, T, d_mom, w, st, &plan->launches);
    });
}

// The K correlation maps of one problem into the workspace (FFT or direct).
// With spec_ready the image spectrum is already in place: the previous
// problem of the call took the same volume through the same FFT box.
ttm_status corr_problem(ttm_plan_s* plan, const ProblemData& pr, const float* vol,
                        void* d_workspace, cudaStream_t st, bool resident = false,
                        bool spec_ready = false) {
    const CorrLayout L = corr_layout(plan, pr, d_workspace, resident);
    float* corr = (float*)L.corr;
    if (pr.path == TTM_PATH_FFT) {
        float2* spec = (float2*)L.spec;
        void* prod = L.prod;
        const SpecSet& sp = plan->specs[pr.spec_index];
        if (!spec_ready)
            TTM_TRY(timed(plan, KC_FFT_FORWARD, st, [&] {
                return launch_fft_forward(vol, pr.X, pr.Y, pr.Z, pr.fft, spec, st,
                                          &plan->launches);
            }));
        const int G = comp_group(plan, pr);
        const size_t nspec = pr.fft.nspec();
        // the score, rotation and component outputs read the interior only
        const FftKeep keep = fft_keep_interior(pr.X, pr.Y, pr.Z, plan->tmpl[pr.tmpl].desc.s);
        for (int k0 = 0; k0 < plan->K; k0 += G) {
            const int g = std::min(G, plan->K - k0);
            TTM_TRY(timed(plan, KC_FFT_SPECTRUM, st, [&] {
                return pr.mixed ? launch_fft_spectrum_inverse_z_bf16(
                                      spec, (const char*)sp.d_spec_bf + (size_t)k0 * nspec * 4, g,
                                      pr.fft, prod, keep, st, &plan->launches)
                                : launch_fft_spectrum_inverse_z(spec, sp.d_spec + (size_t)k0 * nspec,
                                                                g, pr.fft, (float2*)prod, keep, st,
                                                                &plan->launches);
            }));
            TTM_TRY(timed(plan, KC_FFT_INVERSE, st, [&] {
                int* d_status = (int*)((char*)d_workspace + 32);
                return pr.mixed ? launch_fft_inverse_yx_bf16(
                                      prod, g, pr.X, pr.Y, pr.Z, pr.fft,
                                      (char*)corr + (size_t)k0 * pr.nvox() * 2, d_status, keep,
                                      st, &plan->launches)
                                : launch_fft_inverse_yx((float2*)prod, g, pr.X, pr.Y, pr.Z, pr.fft,
                                                        corr + (size_t)k0 * pr.nvox(), d_status,
                                                        keep, st, &plan->launches);
            }));
        }
        return TTM_OK;
    }
    const TemplateData& T = plan->tmpl[pr.tmpl];
    if (pr.tc_direct) {
        // the volume's moments (mean and spread condition the FP16 operand)
        double* d_mom = (double*)((char*)d_workspace + 64);
        TTM_CUDA_TRY(cudaMemsetAsync(d_mom, 0, 2 * sizeof(double), st));
        TTM_TRY(timed(plan, KC_MOMENTS, st, [&] {
            return launch_volume_moments(vol, pr.nvox(), d_mom, st, &plan->launches);
        }));
        return timed(plan, KC_DIRECT_CORR, st, [&] {
            return launch_direct_tc(vol, pr.X, pr.Y, pr.Z, T, plan->K, d_mom, corr,
                                    (int*)((char*)d_workspace + 32), st, &plan->launches);
        });
    }
    return timed(plan, KC_DIRECT_CORR, st, [&] {
        return launch_direct_corr(vol, pr.X, pr.Y, pr.Z, T, plan->K, corr, st, &plan->launches);
    });
}

// Score, rotation search and refinement of one problem from its correlation
// maps (Sec. 3.3-3.4); exterior voxels get the exterior values.  With more
// than one chunk the interior is split into rot_chunks ranges: the searches
// run in order on the plan's high-priority stream, and the refinement of
// chunk i starts on the low-priority stream once its search is done, so the
// tensor-core search (integer-ALU bound) and the refinement (FMA bound) share
// the SMs.  Both streams fork from and join back into st (capturable).
ttm_status rotation_problem(ttm_plan_s* plan, const ProblemData& pr, const float* w, float* score,
                            float* quat, float* lam, float* comp_out, void* d_workspace,
                            cudaStream_t st) {
    const CorrLayout L = corr_layout(plan, pr, d_workspace, false);
    float* corr = (float*)L.corr;
    uint16_t* cand = L.cand;
    int* d_status = (int*)((char*)d_workspace + 32);
    const TemplateData& T = plan->tmpl[pr.tmpl];
    const VoxBox box = interior_box(pr.X, pr.Y, pr.Z, T.desc.s);
    const size_t units = box.count();
    if (units > 0xFFFFFFFFull) return TTM_ERR_UNSUPPORTED;
    TTM_TRY(timed(plan, KC_EXTERIOR, st, [&] {
        return launch_exterior_fill(pr.Z, box, plan->K, score, quat, lam, comp_out, st,
                                    &plan->launches);
    }));
    int nch = plan->rot_chunks;
    if ((size_t)nch * 128 * 152 > units) nch = 1;        // too small to split
    if (nch <= 1 || !plan->s_hi) {
        TTM_TRY(timed(plan, KC_ROTATION, st, [&] {
            return launch_rotation_search(plan->n_order, corr, pr.mixed, w, pr.nvox(), box, 0,
                                          (uint32_t)units, plan->grid, cand, d_status, score, st,
                                          &plan->launches);
        }));
        return timed(plan, KC_POLISH, st, [&] {
            return launch_rotation_polish(plan->n_order, corr, pr.mixed, w, pr.nvox(), box, 0,
                                          (uint32_t)units, plan->grid, cand, score, quat, lam,
                                          comp_out, st, &plan->launches);
        });
    }
    // chunk bounds in whole 128-voxel tiles
    const size_t tiles = (units + 127) / 128;
    auto bound = [&](int c) {
        return (uint32_t)std::min(units, (tiles * (size_t)c / (size_t)nch) * 128);
    };
    TTM_CUDA_TRY(cudaEventRecord(plan->ev_fork, st));
    TTM_CUDA_TRY(cudaStreamWaitEvent(plan->s_hi, plan->ev_fork, 0));
    TTM_CUDA_TRY(cudaStreamWaitEvent(plan->s_lo, plan->ev_fork, 0));
    for (int c = 0; c < nch; ++c) {
        const uint32_t u0 = bound(c), u1 = c + 1 == nch ? (uint32_t)units : bound(c + 1);
        TTM_TRY(timed(plan, KC_ROTATION, plan->s_hi, [&] {
            return launch_rotation_search(plan->n_order, corr, pr.mixed, w, pr.nvox(), box, u0,
                                          u1, plan->grid, cand, d_status, score, plan->s_hi,
                                          &plan->launches);
        }));
        TTM_CUDA_TRY(cudaEventRecord(plan->ev_chunk[c], plan->s_hi));
        TTM_CUDA_TRY(cudaStreamWaitEvent(plan->s_lo, plan->ev_chunk[c], 0));
        TTM_TRY(timed(plan, KC_POLISH, plan->s_lo, [&] {
            return launch_rotation_polish(plan->n_order, corr, pr.mixed, w, pr.nvox(), box, u0,
                                          u1, plan->grid, cand, score, quat, lam, comp_out,
                                          plan->s_lo, &plan->launches);
        }));
    }
    TTM_CUDA_TRY(cudaEventRecord(plan->ev_join, plan->s_lo));
    TTM_CUDA_TRY(cudaStreamWaitEvent(st, plan->ev_join, 0));
    return TTM_OK;
}

// Score, rotation search and refinement of the problems [p0, p1) of one
// resident wave (their correlation maps all in the workspace).  The interior
// units of the wave, problem after problem in tiles of 128, are split into
// rot_chunks ranges; each range is one search launch and one refinement
// launch over a table of (problem, units) segments in the kernels'
// parameters (a range that spans more than kMaxRotSegs problems takes one
// more launch per kMaxRotSegs), pipelined on the rotation streams as in
// rotation_problem.  The problems of a wave share the map type.
ttm_status rotation_wave(ttm_plan_s* plan, int p0, int p1, const float* const* d_w,
                         float* const* d_score, float* const* d_quat, float* const* d_lambda,
                         float* const* d_comp, void* d_workspace, cudaStream_t st) {
    const int n = p1 - p0;
    int* d_status = (int*)((char*)d_workspace + 32);
    const bool mixed = plan->prob[p0].mixed;
    std::vector<RotSeg> segs((size_t)n);
    std::vector<size_t> tile0((size_t)n + 1, 0);
    for (int j = 0; j < n; ++j) {
        const int p = p0 + j;
        const ProblemData& pr = plan->prob[p];
        if (pr.mixed != mixed) return TTM_ERR_UNSUPPORTED;
        const CorrLayout L = corr_layout(plan, pr, d_workspace, true);
        const VoxBox box = interior_box(pr.X, pr.Y, pr.Z, plan->tmpl[pr.tmpl].desc.s);
        const size_t units = box.count();
        if (units > 0xFFFFFFFFull) return TTM_ERR_UNSUPPORTED;
        float* lam = d_lambda ? d_lambda[p] : nullptr;
        float* comp = d_comp ? d_comp[p] : nullptr;
        TTM_TRY(timed(plan, KC_EXTERIOR, st, [&] {
            return launch_exterior_fill(pr.Z, box, plan->K, d_score[p], d_quat[p], lam, comp, st,
                                        &plan->launches);
        }));
        RotSeg& sg = segs[(size_t)j];
        sg.corr = L.corr; sg.w = d_w[p]; sg.score = d_score[p]; sg.cand = L.cand;
        sg.quat = d_quat[p]; sg.lambda = lam; sg.comp_out = comp;
        sg.nvox = pr.nvox(); sg.box = box; sg.u0 = 0; sg.u1 = (uint32_t)units;
        tile0[(size_t)j + 1] = tile0[(size_t)j] + (units + kRotTile - 1) / kRotTile;
    }
    const size_t tiles = tile0[(size_t)n];
    if (tiles == 0) return TTM_OK;
    // the launches of the tile range [a, b)
    std::vector<RotBatch> bl;
    auto batches = [&](size_t a, size_t b) {
        bl.clear();
        RotBatch cur;
        for (int j = 0; j < n; ++j) {
            const size_t lo = std::max(a, tile0[(size_t)j]), hi = std::min(b, tile0[(size_t)j + 1]);
            if (lo >= hi) continue;
            RotSeg sg = segs[(size_t)j];
            sg.u0 = (uint32_t)((lo - tile0[(size_t)j]) * kRotTile);
            sg.u1 = (uint32_t)std::min<size_t>(segs[(size_t)j].u1, (hi - tile0[(size_t)j]) * kRotTile);
            if (!cur.add(sg)) {
                bl.push_back(cur);
                cur = RotBatch();
                cur.add(sg);
            }
        }
        if (cur.n) bl.push_back(cur);
    };
    auto search = [&](cudaStream_t s) {
        for (const RotBatch& b : bl)
            TTM_TRY(timed(plan, KC_ROTATION, s, [&] {
                return launch_rotation_search(plan->n_order, b, mixed, plan->grid, d_status, s,
                                              &plan->launches);
            }));
        return TTM_OK;
    };
    auto polish = [&](cudaStream_t s) {
        for (const RotBatch& b : bl)
            TTM_TRY(timed(plan, KC_POLISH, s, [&] {
                return launch_rotation_polish(plan->n_order, b, mixed, plan->grid, s,
                                              &plan->launches);
            }));
        return TTM_OK;
    };
    int nch = plan->rot_chunks;
    if ((size_t)nch * 152 > tiles) nch = 1;               // too small to split
    if (nch <= 1 || !plan->s_hi) {
        batches(0, tiles);
        TTM_TRY(search(st));
        return polish(st);
    }
    TTM_CUDA_TRY(cudaEventRecord(plan->ev_fork, st));
    TTM_CUDA_TRY(cudaStreamWaitEvent(plan->s_hi, plan->ev_fork, 0));
    TTM_CUDA_TRY(cudaStreamWaitEvent(plan->s_lo, plan->ev_fork, 0));
    for (int c = 0; c < nch; ++c) {
        batches(tiles * (size_t)c / (size_t)nch, tiles * (size_t)(c + 1) / (size_t)nch);
        TTM_TRY(search(plan->s_hi));
        TTM_CUDA_TRY(cudaEventRecord(plan->ev_chunk[c], plan->s_hi));
        TTM_CUDA_TRY(cudaStreamWaitEvent(plan->s_lo, plan->ev_chunk[c], 0));
        TTM_TRY(polish(plan->s_lo));
    }
    TTM_CUDA_TRY(cudaEventRecord(plan->ev_join, plan->s_lo));
    TTM_CUDA_TRY(cudaStreamWaitEvent(st, plan->ev_join, 0));
    return TTM_OK;
}

// Copies the device peak list to the host: records sorted by score
// (descending; equal scores by voxel index), the first max_peaks kept.
// Synchronises the stream.
ttm_status copy_peaks_to_host(const ProblemData& pr, const int* d_count, const void* list, int cap,
                              int max_peaks, ttm_peak* h_out, int* n_out, cudaStream_t st) {
    int count = 0;
    TTM_CUDA_TRY(cudaMemcpyAsync(&count, d_count, sizeof(int), cudaMemcpyDeviceToHost, st));
    TTM_CUDA_TRY(cudaStreamSynchronize(st));
    if (count > cap) return TTM_ERR_WORKSPACE;
    struct Rec { int idx; float score, lambda, q[4]; int pad; };
    static_assert(sizeof(Rec) == 32, "peak record layout");
    if (peak_record_bytes() != sizeof(Rec)) return TTM_ERR_CUDA;
    std::vector<Rec> recs(count);
    if (count > 0) {
        TTM_CUDA_TRY(cudaMemcpyAsync(recs.data(), list, (size_t)count * sizeof(Rec),
                                     cudaMemcpyDeviceToHost, st));
        TTM_CUDA_TRY(cudaStreamSynchronize(st));
    }
    std::sort(recs.begin(), recs.end(), [](const Rec& a, const Rec& b) {
        if (a.score != b.score) return a.score > b.score;
        return a.idx < b.idx;
    });
    const int nout = std::min(count, max_peaks);
    for (int i = 0; i < nout; ++i) {
        const Rec& r = recs[i];
        ttm_peak& o = h_out[i];
        o.x = (int)(r.idx % pr.X);
        o.y = (int)((r.idx / pr.X) % pr.Y);
        o.z = (int)(r.idx / ((size_t)pr.X * pr.Y));
        o.score = r.score;
        o.lambda = r.lambda;
        for (int k = 0; k < 4; ++k) o.q[k] = r.q[k];
    }
    *n_out = nout;
    return TTM_OK;
}

// ---- autotuner (TTM_PATH_TUNE) ----

// A problem moved to the direct path: tensor cores in mixed precision where
// the template has their table, CUDA cores otherwise.
void to_direct(const ttm_plan_s* P, ProblemData& pr) {
    pr.path = TTM_PATH_DIRECT;
    pr.mixed = false;
    pr.tc_direct = P->opts.precision == TTM_PREC_MIXED && P->tmpl[pr.tmpl].d_tc_tab != nullptr;
}

// Device time of local statistics + K correlations of one problem: one
// warm-up run, then the best of two timed runs (ms), or -1 on failure.
double time_paths_once(ttm_plan_s* P, const ProblemData& pr, const float* vol, float* w, void* ws,
                       cudaStream_t st) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        cudaGetLastError();
        if (a) cudaEventDestroy(a);
        return -1.0;
    }
    double best = -1.0;
    for (int rep = 0; rep < 3; ++rep) {
        if (cudaEventRecord(a, st) != cudaSuccess) break;
        if (stats_problem(P, pr, vol, w, ws, st) != TTM_OK) break;
        if (corr_problem(P, pr, vol, ws, st) != TTM_OK) break;
        if (cudaEventRecord(b, st) != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess) break;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) break;
        if (rep > 0 && (best < 0.0 || ms < best)) best = ms;
    }
    cudaGetLastError();
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return best;
}

// Times the direct and the FFT path of every distinct problem shape that can
// take both (problems arrive here on the FFT path) and keeps the faster.
// Problems with the same template, extents and precision share a decision.
// Template spectra no FFT problem uses any more are freed.
ttm_status tune_paths(ttm_plan_s* P, cudaStream_t st) {
    const int np = (int)P->prob.size();
    for (int p = 0; p < np; ++p) {
        ProblemData& pr = P->prob[p];
        if (pr.path != TTM_PATH_FFT || P->tmpl[pr.tmpl].soft) continue;
        bool shared = false;
        for (int q = 0; q < p && !shared; ++q) {
            const ProblemData& o = P->prob[q];
            if (o.tmpl != pr.tmpl || o.X != pr.X || o.Y != pr.Y || o.Z != pr.Z) continue;
            if (o.tune_ms[0] < 0.0 && o.tune_ms[1] < 0.0) continue;     // not timed
            pr.tune_ms[0] = o.tune_ms[0];
            pr.tune_ms[1] = o.tune_ms[1];
            if (o.path == TTM_PATH_DIRECT) {
                pr.path = TTM_PATH_DIRECT;
                pr.mixed = false;
                pr.tc_direct = o.tc_direct;
            }
            shared = true;
        }
        if (shared) continue;
        const double ratio = model_ratio(P, pr, P->tmpl[pr.tmpl]);
        if (ratio > kTuneRange) continue;                          // FFT, clearly
        if (ratio < 1.0 / kTuneRange) { to_direct(P, pr); continue; }
        ProblemData dpr = pr;
        dpr.path = TTM_PATH_DIRECT;
        dpr.mixed = false;
        dpr.tc_direct = P->opts.precision == TTM_PREC_MIXED && P->tmpl[pr.tmpl].d_tc_tab != nullptr;
        const size_t nv = pr.nvox();
        const size_t wsb = kHeader + std::max(scratch_bytes(P, pr), scratch_bytes(P, dpr));
        float* vol = nullptr;
        float* w = nullptr;
        void* ws = nullptr;
        if (cudaMalloc((void**)&vol, nv * sizeof(float)) != cudaSuccess ||
            cudaMalloc((void**)&w, nv * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&ws, wsb) != cudaSuccess) {
            // not enough memory to tune: keep the planner's estimate
            cudaGetLastError();
            cudaFree(vol); cudaFree(w); cudaFree(ws);
            if (!prefer_fft(P, pr, P->tmpl[pr.tmpl])) to_direct(P, pr);
            continue;
        }
        ttm_status s = launch_fill_random(vol, nv, 0x5eedu + (uint32_t)p, st, &P->launches);
        if (s == TTM_OK) {
            pr.tune_ms[0] = time_paths_once(P, dpr, vol, w, ws, st);
            pr.tune_ms[1] = time_paths_once(P, pr, vol, w, ws, st);
        }
        cudaError_t e = cudaStreamSynchronize(st);
        cudaFree(vol); cudaFree(w); cudaFree(ws);
        if (s != TTM_OK) return s;
        if (e != cudaSuccess) return TTM_ERR_CUDA;
        if (pr.tune_ms[1] < 0.0 || (pr.tune_ms[0] >= 0.0 && pr.tune_ms[0] < pr.tune_ms[1])) {
            pr.path = TTM_PATH_DIRECT;
            pr.mixed = false;
            pr.tc_direct = dpr.tc_direct;
        }
    }
    for (size_t i = 0; i < P->specs.size(); ++i) {
        bool used = false;
        for (const ProblemData& pr : P->prob) used = used || (pr.path == TTM_PATH_FFT && pr.spec_index == (int)i);
        if (used) continue;
        SpecSet& sp = P->specs[i];
        cudaFree(sp.d_spec); cudaFree(sp.d_spec_bf); cudaFree(sp.d_mask_spec);
        sp.d_spec = nullptr; sp.d_spec_bf = nullptr; sp.d_mask_spec = nullptr;
    }
    return TTM_OK;
}

}  // namespace
}  // namespace ttm

using namespace ttm;

extern "C" {

const char* ttm_status_string(ttm_status s) {
    switch (s) {
        case TTM_OK: return "TTM_OK";
        case TTM_ERR_INVALID_ARG: return "TTM_ERR_INVALID_ARG";
        case TTM_ERR_UNSUPPORTED: return "TTM_ERR_UNSUPPORTED";
        case TTM_ERR_OUT_OF_MEMORY: return "TTM_ERR_OUT_OF_MEMORY";
        case TTM_ERR_CUDA: return "TTM_ERR_CUDA";
        case TTM_ERR_TIMEOUT: return "TTM_ERR_TIMEOUT";
        case TTM_ERR_NUMERIC: return "TTM_ERR_NUMERIC";
        case TTM_ERR_WORKSPACE: return "TTM_ERR_WORKSPACE";
        default: return "TTM_ERR_UNKNOWN";
    }
}

int ttm_device_count(void) {
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

// quadrature nodes rotated per chunk: 128 MiB of rotated copies, at least
// two per SM (one CTA rotates one node), at most 1 GiB
static int build_chunk(int s, int n_rot) {
    const size_t s3 = (size_t)s * s * s;
    size_t nj = ((size_t)128 << 20) / (s3 * sizeof(float));
    nj = std::max<size_t>(nj, 304);
    nj = std::min<size_t>(nj, ((size_t)1 << 30) / (s3 * sizeof(float)));
    if (nj < 1) nj = 1;
    if (nj > (size_t)n_rot) nj = (size_t)n_rot;
    return (int)nj;
}

ttm_status ttm_build_workspace_size(int s, int n_order, int n_rot, size_t* bytes) {
    if (!bytes || s < 3 || s > 128 || n_rot < 1) return TTM_ERR_INVALID_ARG;
    if (n_order < 2 || n_order > 8 || (n_order & 1)) return TTM_ERR_UNSUPPORTED;
    const size_t s3 = (size_t)s * s * s;
    *bytes = kHeader + align256((size_t)build_chunk(s, n_rot) * s3 * sizeof(float));
    return TTM_OK;
}

ttm_status ttm_build_tensor_template(const float* d_template, const float* d_mask, int s,
                                     int n_order, const float* d_quats, const float* d_weights,
                                     int n_rot, float* d_components, void* d_workspace,
                                     size_t workspace_bytes, ttm_tt_desc* desc, void* stream) {
    if (!d_template || !d_mask || !d_quats || !d_components || !desc) return TTM_ERR_INVALID_ARG;
    size_t need = 0;
    TTM_TRY(ttm_build_workspace_size(s, n_order, n_rot, &need));
    if (!d_workspace || workspace_bytes < need) return TTM_ERR_WORKSPACE;
    if (!aligned(d_workspace, 256) || !aligned(d_template, 4) || !aligned(d_mask, 4) ||
        !aligned(d_quats, 4) || !aligned(d_components, 4) || !aligned(d_weights, 4))
        return TTM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    long long cnt = 0;
    char* ws = (char*)d_workspace;
    double* d_msum = (double*)ws;
    int* d_bad = (int*)(ws + 8);
    float* rot = (float*)(ws + kHeader);
    TTM_CUDA_TRY(cudaMemsetAsync(ws, 0, kHeader, st));
    TTM_TRY(launch_mask_sum(d_mask, s, d_msum, st, &cnt));
    double msum = 0.0;
    TTM_CUDA_TRY(cudaMemcpyAsync(&msum, d_msum, sizeof(double), cudaMemcpyDeviceToHost, st));
    TTM_CUDA_TRY(cudaStreamSynchronize(st));
    if (!(msum > 0.0)) return TTM_ERR_INVALID_ARG;
    const int nj = build_chunk(s, n_rot);
    const int s3 = s * s * s;
    for (int j0 = 0; j0 < n_rot; j0 += nj) {
        const int cnt_j = std::min(nj, n_rot - j0);
        TTM_TRY(launch_rotate_normalise(d_template, d_mask, s, d_quats, j0, cnt_j, rot, msum, d_bad,
                                        st, &cnt));
        TTM_TRY(launch_fold_components(n_order, d_quats, d_weights, n_rot, j0, cnt_j, rot, s3,
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

ttm_status ttm_plan(ttm_plan_t* out, int n_problems, const int* vol_dims, const int* tmpl_index,
                    int n_templates, const ttm_tt_desc* descs, const float* const* d_components,
                    const float* const* d_masks, const ttm_plan_opts* opts, void* stream) {
    if (!out) return TTM_ERR_INVALID_ARG;
    *out = nullptr;
    if (n_problems < 1 || n_templates < 1 || !vol_dims || !tmpl_index || !descs ||
        !d_components || !d_masks)
        return TTM_ERR_INVALID_ARG;
    const int n_order = descs[0].n_order;
    for (int k = 0; k < n_templates; ++k) {
        const ttm_tt_desc& d = descs[k];
        if (d.n_order != n_order) return TTM_ERR_UNSUPPORTED;  // one order per plan
        if (d.n_order < 2 || d.n_order > 8 || (d.n_order & 1)) return TTM_ERR_UNSUPPORTED;
        if (d.K != n_comp(d.n_order) || d.s < 3 || d.s > 128 || d.centre != d.s / 2 ||
            !(d.mask_sum > 0.0) || !d_components[k] || !d_masks[k])
            return TTM_ERR_INVALID_ARG;
    }
    for (int p = 0; p < n_problems; ++p) {
        const int X = vol_dims[3 * p], Y = vol_dims[3 * p + 1], Z = vol_dims[3 * p + 2];
        if (tmpl_index[p] < 0 || tmpl_index[p] >= n_templates) return TTM_ERR_INVALID_ARG;
        const int s = descs[tmpl_index[p]].s;
        if (X < s || Y < s || Z < s) return TTM_ERR_INVALID_ARG;
        if ((size_t)X * Y * Z >= ((size_t)1 << 31)) return TTM_ERR_UNSUPPORTED;
    }
    if (opts && opts->lowpass_sigma != 0.f && !lowpass_sigma_ok(opts->lowpass_sigma))
        return TTM_ERR_INVALID_ARG;
    if (opts) {
        // plan options, checked before any device work
        const ttm_plan_opts& o = *opts;
        if (o.path < TTM_PATH_AUTO || o.path > TTM_PATH_TUNE) return TTM_ERR_INVALID_ARG;
        if (o.precision != TTM_PREC_FP32 && o.precision != TTM_PREC_MIXED) return TTM_ERR_INVALID_ARG;
        if (o.n_grid < 0 || o.n_cells < 0 || o.n_candidates < 0 || o.newton_steps < 0 ||
            o.rotation_chunks < 0 || o.n_refined < 0 || o.batch_mib < 0 || o.batch_mib > (1 << 20))
            return TTM_ERR_INVALID_ARG;
        const int n = o.n_grid > 0 ? o.n_grid : 2048, nc = o.n_cells > 0 ? o.n_cells : n / 16;
        if (n > 65535 || nc > n || n % nc != 0 || o.n_candidates > 8 || o.newton_steps > 64 ||
            o.n_refined > 4)
            return TTM_ERR_INVALID_ARG;
    }
    ttm_plan_s* P = new (std::nothrow) ttm_plan_s();
    if (!P) return TTM_ERR_OUT_OF_MEMORY;
    if (opts) P->opts = *opts;
    P->n_order = n_order;
    P->K = n_comp(n_order);
    cudaStream_t st = (cudaStream_t)stream;
    ttm_status s_ = TTM_OK;
    if (cudaStreamSynchronize(st) != cudaSuccess) { cudaGetLastError(); free_plan(P); return TTM_ERR_CUDA; }
    P->tmpl.resize(n_templates);
    for (int k = 0; k < n_templates && s_ == TTM_OK; ++k) {
        P->tmpl[k].desc = descs[k];
        P->tmpl[k].d_comp = d_components[k];
        s_ = prepare_template(P, P->tmpl[k], d_masks[k]);
    }
    if (s_ == TTM_OK) s_ = build_grid(P);
    if (s_ == TTM_OK) s_ = make_rotation_streams(P);
    if (s_ != TTM_OK) { free_plan(P); return s_; }
    P->prob.resize(n_problems);
    size_t ws = 0;
    for (int p = 0; p < n_problems; ++p) {
        ProblemData& pr = P->prob[p];
        pr.X = vol_dims[3 * p]; pr.Y = vol_dims[3 * p + 1]; pr.Z = vol_dims[3 * p + 2];
        pr.tmpl = tmpl_index[p];
        const TemplateData& T = P->tmpl[pr.tmpl];
        pr.fft.Xp = fft_good_length(pr.X);
        pr.fft.Yp = fft_good_length(pr.Y);
        pr.fft.Zp = fft_good_length(pr.Z);
        const bool fft_ok = fft_length_ok(pr.fft.Xp) && fft_length_ok(pr.fft.Yp) &&
                            fft_length_ok(pr.fft.Zp);
        int path = P->opts.path;
        if (T.soft) {
            // soft masks: FFT correlations and FFT window sums only
            if (path == TTM_PATH_DIRECT || !fft_ok || !fft_template_length(pr.fft.Xp)) {
                free_plan(P);
                return TTM_ERR_UNSUPPORTED;
            }
            path = TTM_PATH_FFT;
        }
        if (path == TTM_PATH_TUNE) path = fft_ok ? TTM_PATH_FFT : TTM_PATH_DIRECT;
        if (path == TTM_PATH_AUTO) path = (fft_ok && prefer_fft(P, pr, T)) ? TTM_PATH_FFT : TTM_PATH_DIRECT;
        if (path == TTM_PATH_FFT && !fft_ok) { free_plan(P); return TTM_ERR_UNSUPPORTED; }
        if (path != TTM_PATH_FFT && path != TTM_PATH_DIRECT) { free_plan(P); return TTM_ERR_INVALID_ARG; }
        pr.path = path;
        pr.mixed = path == TTM_PATH_FFT && P->opts.precision == TTM_PREC_MIXED &&
                   fft_template_length(pr.fft.Xp) && fft_template_length(pr.fft.Yp) &&
                   fft_template_length(pr.fft.Zp);
        pr.tc_direct = path == TTM_PATH_DIRECT && P->opts.precision == TTM_PREC_MIXED &&
                       T.d_tc_tab != nullptr;
        if (P->opts.precision != TTM_PREC_FP32 && P->opts.precision != TTM_PREC_MIXED) {
            free_plan(P);
            return TTM_ERR_INVALID_ARG;
        }
        if (path == TTM_PATH_FFT) {
            s_ = prepare_fft(P, pr, st);
            if (s_ != TTM_OK) { free_plan(P); return s_; }
        }
    }
    if (P->opts.path == TTM_PATH_TUNE) {
        s_ = tune_paths(P, st);
        if (s_ != TTM_OK) { free_plan(P); return s_; }
    }
    const bool lp = P->opts.lowpass_sigma > 0.f;
    if (P->opts.batch_mib > 0 && n_problems > 1) {
        plan_waves(P);
        // the prefiltered volume and its scratch sit after every problem's
        // scratch and the resident waves
        size_t end = P->wave_scratch_off + wave_scratch_bytes(P);
        size_t lpb = 0;
        for (const ProblemData& pr : P->prob) {
            end = std::max(end, kHeader + align256(scratch_bytes(P, pr)));
            lpb = std::max(lpb, lp ? 2 * align256(pr.nvox() * sizeof(float)) : 0);
        }
        for (ProblemData& pr : P->prob) pr.lp_off = end;
        P->ws_bytes = end + lpb;
        *out = P;
        return TTM_OK;
    }
    for (ProblemData& pr : P->prob) {
        // the prefiltered volume and its scratch sit after the problem's scratch
        const size_t sb = align256(scratch_bytes(P, pr));
        pr.lp_off = kHeader + sb;
        ws = std::max(ws, sb + (lp ? 2 * align256(pr.nvox() * sizeof(float)) : 0));
    }
    P->ws_bytes = kHeader + ws;
    *out = P;
    return TTM_OK;
}

ttm_status ttm_plan_workspace_size(ttm_plan_t plan, size_t* bytes) {
    if (!plan || !bytes) return TTM_ERR_INVALID_ARG;
    *bytes = plan->ws_bytes;
    return TTM_OK;
}

ttm_status ttm_plan_problem_path(ttm_plan_t plan, int problem, int* path) {
    if (!plan || !path || problem < 0 || problem >= (int)plan->prob.size())
        return TTM_ERR_INVALID_ARG;
    *path = plan->prob[problem].path;
    return TTM_OK;
}

ttm_status ttm_plan_problem_tuning(ttm_plan_t plan, int problem, double* ms) {
    if (!plan || !ms || problem < 0 || problem >= (int)plan->prob.size())
        return TTM_ERR_INVALID_ARG;
    ms[0] = plan->prob[problem].tune_ms[0];
    ms[1] = plan->prob[problem].tune_ms[1];
    return TTM_OK;
}

ttm_status ttm_plan_problem_tensor_direct(ttm_plan_t plan, int problem, int* on) {
    if (!plan || !on || problem < 0 || problem >= (int)plan->prob.size())
        return TTM_ERR_INVALID_ARG;
    *on = plan->prob[problem].tc_direct ? 1 : 0;
    return TTM_OK;
}

ttm_status ttm_plan_problem_fft_box(ttm_plan_t plan, int problem, int* box) {
    if (!plan || !box || problem < 0 || problem >= (int)plan->prob.size())
        return TTM_ERR_INVALID_ARG;
    const ProblemData& pr = plan->prob[problem];
    const bool fft = pr.path == TTM_PATH_FFT;
    box[0] = fft ? pr.fft.Xp : 0;
    box[1] = fft ? pr.fft.Yp : 0;
    box[2] = fft ? pr.fft.Zp : 0;
    return TTM_OK;
}

ttm_status ttm_plan_launch_count(ttm_plan_t plan, long long* launches) {
    if (!plan || !launches) return TTM_ERR_INVALID_ARG;
    *launches = plan->launches;
    return TTM_OK;
}

ttm_status ttm_probe_bounded_wait(long long polls, int arrive, int* status_out, void* stream) {
    if (polls < 1 || polls > (1LL << 24) || !status_out) return TTM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int* d = nullptr;
    TTM_CUDA_TRY(cudaMalloc((void**)&d, sizeof(int)));
    long long cnt = 0;
    ttm_status s = launch_wait_probe((long)polls, arrive ? 1 : 0, d, st, &cnt);
    int h = TTM_ERR_CUDA;
    if (s == TTM_OK &&
        (cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
         cudaStreamSynchronize(st) != cudaSuccess)) {
        cudaGetLastError();
        s = TTM_ERR_CUDA;
    }
    cudaFree(d);
    if (s != TTM_OK) return s;
    *status_out = h;
    return TTM_OK;
}

ttm_status ttm_plan_waves(ttm_plan_t plan, int* n_waves, int* first) {
    if (!plan || !n_waves) return TTM_ERR_INVALID_ARG;
    *n_waves = (int)plan->waves.size();
    if (first)
        for (size_t i = 0; i < plan->waves.size(); ++i) first[i] = plan->waves[i].first;
    return TTM_OK;
}

ttm_status ttm_plan_device_status(ttm_plan_t plan, void* d_workspace, size_t workspace_bytes,
                                  void* stream) {
    if (!plan) return TTM_ERR_INVALID_ARG;
    TTM_TRY(check_ws(plan, d_workspace, workspace_bytes));
    cudaStream_t st = (cudaStream_t)stream;
    int v = 0;
    TTM_CUDA_TRY(cudaMemcpyAsync(&v, (char*)d_workspace + 32, sizeof(int), cudaMemcpyDeviceToHost, st));
    TTM_CUDA_TRY(cudaStreamSynchronize(st));
    return v == 0 ? TTM_OK : (ttm_status)v;
}

ttm_status ttm_plan_enable_timing(ttm_plan_t plan, int enable) {
    if (!plan) return TTM_ERR_INVALID_ARG;
    plan->timing = enable != 0;
    return TTM_OK;
}

ttm_status ttm_plan_timing(ttm_plan_t plan, double* ms, long long* launches, int n_classes) {
    if (!plan || n_classes < 0) return TTM_ERR_INVALID_ARG;
    for (int c = 0; c < n_classes; ++c) {
        if (ms) ms[c] = 0.0;
        if (launches) launches[c] = 0;
    }
    ttm_status st = TTM_OK;
    for (TimedLaunch& t : plan->timed) {
        float e = 0.f;
        if (cudaEventSynchronize(t.stop) != cudaSuccess ||
            cudaEventElapsedTime(&e, t.start, t.stop) != cudaSuccess) {
            cudaGetLastError();
            st = TTM_ERR_CUDA;
        }
        if (t.cls >= 0 && t.cls < n_classes) {
            if (ms) ms[t.cls] += e;
            if (launches) launches[t.cls] += t.n;
        }
        plan->event_pool.push_back(t.start);
        plan->event_pool.push_back(t.stop);
    }
    plan->timed.clear();
    return st;
}

const char* ttm_kernel_class_name(int c) {
    static const char* names[TTM_KERNEL_CLASSES] = {
        "volume_moments", "local_stats", "direct_corr", "rotation_search", "fft_forward",
        "fft_spectrum_inverse", "fft_inverse", "peaks", "template", "fft_plan", "rotation_polish",
        "exterior_fill", "rotation_stage"};
    if (c < 0 || c >= TTM_KERNEL_CLASSES) return "unknown";
    return names[c];
}

void ttm_plan_destroy(ttm_plan_t plan) {
    if (plan) free_plan(plan);
}

ttm_status ttm_local_stats(ttm_plan_t plan, const float* const* d_vols, float* const* d_w,
                           void* d_workspace, size_t workspace_bytes, void* stream) {
    if (!plan || !d_vols || !d_w) return TTM_ERR_INVALID_ARG;
    TTM_TRY(check_ws(plan, d_workspace, workspace_bytes));
    const int np = (int)plan->prob.size();
    for (int p = 0; p < np; ++p)
        if (!d_vols[p] || !d_w[p] || !aligned(d_vols[p], 4) || !aligned(d_w[p], 4))
            return TTM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    TTM_CUDA_TRY(cudaMemsetAsync((char*)d_workspace + 32, 0, sizeof(int), st));  // status word
    for (int p = 0; p < np; ++p) {
        const ProblemData& pr = plan->prob[p];
        // consecutive problems of one volume share its moments and, on one
        // FFT box, the spectra of its window sums
        int reuse = kReuseNone;
        if (p > 0 && same_volume(plan, p - 1, p, d_vols))
            reuse = stats_on_fft(plan->prob[p - 1]) && stats_on_fft(pr) ? kReuseSpectra
                                                                         : kReuseMoments;
        const float* vol = nullptr;
        TTM_TRY(prefilter(plan, pr, d_vols[p], d_workspace, st, &vol));
        TTM_TRY(stats_problem(plan, pr, vol, d_w[p], d_workspace, st, reuse));
    }
    return TTM_OK;
}

ttm_status ttm_correlate(ttm_plan_t plan, const float* const* d_vols, const float* const* d_w,
                         float* const* d_score, float* const* d_quat, float* const* d_lambda,
                         float* const* d_components_out, void* d_workspace,
                         size_t workspace_bytes, void* stream) {
    if (!plan || !d_vols || !d_w || !d_score || !d_quat) return TTM_ERR_INVALID_ARG;
    TTM_TRY(check_ws(plan, d_workspace, workspace_bytes));
    const int np = (int)plan->prob.size();
    for (int p = 0; p < np; ++p) {
        if (!d_vols[p] || !d_w[p] || !d_score[p] || !d_quat[p]) return TTM_ERR_INVALID_ARG;
        if (!aligned(d_quat[p], 16) || !aligned(d_vols[p], 4) || !aligned(d_score[p], 4))
            return TTM_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    TTM_CUDA_TRY(cudaMemsetAsync((char*)d_workspace + 32, 0, sizeof(int), st));
    // the image spectrum of the previous problem serves the next one when
    // both take the same volume through the same FFT box
    auto spec_ready = [&](int p) {
        if (p == 0 || !same_volume(plan, p - 1, p, d_vols)) return false;
        const ProblemData &a = plan->prob[p - 1], &b = plan->prob[p];
        return a.path == TTM_PATH_FFT && b.path == TTM_PATH_FFT && a.mixed == b.mixed;
    };
    if (!plan->waves.empty()) {
        for (const auto& wv : plan->waves) {
            for (int p = wv.first; p < wv.second; ++p) {
                const float* vol = nullptr;
                TTM_TRY(prefilter(plan, plan->prob[p], d_vols[p], d_workspace, st, &vol));
                TTM_TRY(corr_problem(plan, plan->prob[p], vol, d_workspace, st, true,
                                     spec_ready(p)));
            }
            TTM_TRY(timed(plan, KC_ROT_STAGE, st, [&] {
                return rotation_wave(plan, wv.first, wv.second, d_w, d_score, d_quat, d_lambda,
                                     d_components_out, d_workspace, st);
            }));
        }
        return TTM_OK;
    }
    for (int p = 0; p < np; ++p) {
        const ProblemData& pr = plan->prob[p];
        const float* vol = nullptr;
        TTM_TRY(prefilter(plan, pr, d_vols[p], d_workspace, st, &vol));
        TTM_TRY(corr_problem(plan, pr, vol, d_workspace, st, false, spec_ready(p)));
        TTM_TRY(timed(plan, KC_ROT_STAGE, st, [&] {
            return rotation_problem(plan, pr, d_w[p], d_score[p], d_quat[p],
                                    d_lambda ? d_lambda[p] : nullptr,
                                    d_components_out ? d_components_out[p] : nullptr,
                                    d_workspace, st);
        }));
    }
    return TTM_OK;
}

static constexpr int kClassicalBatch = 32;

struct ClassicalLayout {
    size_t spec, tspec, prod, maps, rot, pad, total;
};

static ClassicalLayout classical_layout(const ttm_plan_s* P, const ProblemData& pr) {
    const TemplateData& T = P->tmpl[pr.tmpl];
    const size_t nspec = pr.fft.nspec();
    const size_t nreal = (size_t)pr.fft.Xp * pr.fft.Yp * pr.fft.Zp;
    const size_t s3 = (size_t)T.desc.s * T.desc.s * T.desc.s;
    ClassicalLayout L;
    size_t off = kHeader;
    L.spec = off;  off += align256(nspec * sizeof(float2));
    L.tspec = off; off += align256((size_t)kClassicalBatch * nspec * sizeof(float2));
    L.prod = off;  off += align256((size_t)kClassicalBatch * nspec * sizeof(float2));
    L.maps = off;  off += align256((size_t)kClassicalBatch * pr.nvox() * sizeof(float));
    L.rot = off;   off += align256((size_t)kClassicalBatch * s3 * sizeof(float));
    L.pad = off;   off += align256(nreal * sizeof(float));
    L.total = off;
    return L;
}

ttm_status ttm_classical_workspace_size(ttm_plan_t plan, int problem, size_t* bytes) {
    if (!plan || !bytes || problem < 0 || problem >= (int)plan->prob.size())
        return TTM_ERR_INVALID_ARG;
    const ProblemData& pr = plan->prob[problem];
    if (pr.path != TTM_PATH_FFT) return TTM_ERR_UNSUPPORTED;
    *bytes = classical_layout(plan, pr).total;
    return TTM_OK;
}

ttm_status ttm_classical_ncc(ttm_plan_t plan, int problem, const float* d_template,
                             const float* d_quats, int n_rot, const float* d_vol,
                             const float* d_w, float* d_best, int* d_best_index,
                             void* d_workspace, size_t workspace_bytes, void* stream) {
    if (!plan || problem < 0 || problem >= (int)plan->prob.size() || !d_template || !d_quats ||
        n_rot < 1 || !d_vol || !d_w || !d_best || !d_best_index)
        return TTM_ERR_INVALID_ARG;
    const ProblemData& pr = plan->prob[problem];
    if (pr.path != TTM_PATH_FFT) return TTM_ERR_UNSUPPORTED;
    const ClassicalLayout Lay = classical_layout(plan, pr);
    if (!d_workspace || workspace_bytes < Lay.total) return TTM_ERR_WORKSPACE;
    if (!aligned(d_workspace, 256)) return TTM_ERR_INVALID_ARG;
    const TemplateData& T = plan->tmpl[pr.tmpl];
    const int s = T.desc.s;
    cudaStream_t st = (cudaStream_t)stream;
    char* ws = (char*)d_workspace;
    int* d_bad = (int*)(ws + 40);
    float2* spec = (float2*)(ws + Lay.spec);
    float2* tspec = (float2*)(ws + Lay.tspec);
    float2* prod = (float2*)(ws + Lay.prod);
    float* maps = (float*)(ws + Lay.maps);
    float* rot = (float*)(ws + Lay.rot);
    float* pad = (float*)(ws + Lay.pad);
    TTM_CUDA_TRY(cudaMemsetAsync(d_bad, 0, sizeof(int), st));
    TTM_TRY(timed(plan, KC_FFT_FORWARD, st, [&] {
        return launch_fft_forward(d_vol, pr.X, pr.Y, pr.Z, pr.fft, spec, st, &plan->launches);
    }));
    for (int j0 = 0; j0 < n_rot; j0 += kClassicalBatch) {
        const int nb = std::min(kClassicalBatch, n_rot - j0);
        TTM_TRY(timed(plan, KC_TEMPLATE, st, [&] {
            TTM_TRY(launch_rotate_normalise(d_template, T.d_mask, s, d_quats, j0, nb, rot,
                                            T.desc.mask_sum, d_bad, st, &plan->launches));
            return launch_template_spectra(rot, nb, s, pr.fft, pad, tspec, st, &plan->launches);
        }));
        TTM_TRY(timed(plan, KC_FFT_SPECTRUM, st, [&] {
            return launch_fft_spectrum_inverse_z(spec, tspec, nb, pr.fft, prod,
                                                 fft_keep_all(pr.X, pr.Y, pr.Z), st,
                                                 &plan->launches);
        }));
        TTM_TRY(timed(plan, KC_FFT_INVERSE, st, [&] {
            return launch_fft_inverse_yx(prod, nb, pr.X, pr.Y, pr.Z, pr.fft, maps,
                                         (int*)(ws + 32), fft_keep_all(pr.X, pr.Y, pr.Z), st,
                                         &plan->launches);
        }));
        TTM_TRY(timed(plan, KC_PEAKS, st, [&] {
            return launch_best_rotation(maps, nb, j0, d_w, pr.nvox(), d_best, d_best_index, j0 == 0,
                                        st, &plan->launches);
        }));
    }
    int bad = 0;
    TTM_CUDA_TRY(cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    TTM_CUDA_TRY(cudaStreamSynchronize(st));
    return bad ? TTM_ERR_NUMERIC : TTM_OK;
}

ttm_status ttm_extract_peaks(ttm_plan_t plan, int problem, const float* d_score,
                             const float* d_quat, const float* d_lambda, float threshold,
                             int radius, int max_peaks, ttm_peak* h_out, int* n_out,
                             void* d_workspace, size_t workspace_bytes, void* stream) {
    if (!plan || problem < 0 || problem >= (int)plan->prob.size() || !d_score || !d_quat ||
        !n_out || radius < 0 || radius > 32 || max_peaks < 0 || (max_peaks > 0 && !h_out))
        return TTM_ERR_INVALID_ARG;
    if (!aligned(d_quat, 16)) return TTM_ERR_INVALID_ARG;
    TTM_TRY(check_ws(plan, d_workspace, workspace_bytes));
    const ProblemData& pr = plan->prob[problem];
    const size_t nv = pr.nvox();
    cudaStream_t st = (cudaStream_t)stream;
    char* ws = (char*)d_workspace;
    int* d_count = (int*)(ws + 16);
    float* tmp_a = (float*)(ws + kHeader);
    float* tmp_b = (float*)(ws + kHeader + align256(nv * sizeof(float)));
    void* list = ws + kHeader + 2 * align256(nv * sizeof(float));
    const int cap = (int)peak_cap(nv);
    TTM_CUDA_TRY(cudaMemsetAsync(d_count, 0, sizeof(int), st));
    TTM_TRY(timed(plan, KC_PEAKS, st, [&] {
        return launch_peak_candidates_full(d_score, d_quat, d_lambda, pr.X, pr.Y, pr.Z, threshold,
                                           radius, tmp_a, tmp_b, list, cap, d_count, st,
                                           &plan->launches);
    }));
    return copy_peaks_to_host(pr, d_count, list, cap, max_peaks, h_out, n_out, st);
}

ttm_status ttm_lowpass(const float* d_in, int X, int Y, int Z, float sigma, float* d_tmp,
                       float* d_out, void* stream) {
    if (!d_in || !d_tmp || !d_out || X < 1 || Y < 1 || Z < 1) return TTM_ERR_INVALID_ARG;
    if (d_in == d_out || d_in == d_tmp || d_tmp == d_out) return TTM_ERR_INVALID_ARG;
    if (!aligned(d_in, 4) || !aligned(d_tmp, 4) || !aligned(d_out, 4)) return TTM_ERR_INVALID_ARG;
    if (!lowpass_sigma_ok(sigma)) return TTM_ERR_INVALID_ARG;
    long long cnt = 0;
    return launch_lowpass(d_in, X, Y, Z, sigma, d_tmp, d_out, (cudaStream_t)stream, &cnt);
}

ttm_status ttm_match_peaks(ttm_plan_t plan, int problem, const float* d_vol, const float* d_w,
                           float* d_score, float threshold, int radius, int max_peaks,
                           ttm_peak* h_out, int* n_out, void* d_workspace, size_t workspace_bytes,
                           void* stream) {
    if (!plan || problem < 0 || problem >= (int)plan->prob.size() || !d_vol || !d_w || !d_score ||
        !n_out || radius < 0 || radius > 32 || max_peaks < 0 || (max_peaks > 0 && !h_out))
        return TTM_ERR_INVALID_ARG;
    if (!aligned(d_vol, 4) || !aligned(d_w, 4) || !aligned(d_score, 4)) return TTM_ERR_INVALID_ARG;
    TTM_TRY(check_ws(plan, d_workspace, workspace_bytes));
    const ProblemData& pr = plan->prob[problem];
    const TemplateData& T = plan->tmpl[pr.tmpl];
    const size_t nv = pr.nvox();
    cudaStream_t st = (cudaStream_t)stream;
    char* ws = (char*)d_workspace;
    int* d_count = (int*)(ws + 16);
    int* d_status = (int*)(ws + 32);
    // workspace: correlation maps and candidates as in ttm_correlate, then the
    // peak pass's two maps and its list
    float* corr = (float*)(ws + kHeader);
    uint16_t* cand = (uint16_t*)((char*)corr + corr_region_bytes(plan, pr));
    char* pk = (char*)cand + align256(nv * 16);
    float* tmp_a = (float*)pk;
    float* tmp_b = (float*)(pk + align256(nv * sizeof(float)));
    char* list = pk + 2 * align256(nv * sizeof(float));
    const int cap = (int)peak_cap(nv);
    const VoxBox box = interior_box(pr.X, pr.Y, pr.Z, T.desc.s);
    TTM_CUDA_TRY(cudaMemsetAsync(ws + 16, 0, 32, st));       // peak count, status word
    const float* vol = nullptr;
    TTM_TRY(prefilter(plan, pr, d_vol, d_workspace, st, &vol));
    TTM_TRY(corr_problem(plan, pr, vol, d_workspace, st));
    TTM_TRY(timed(plan, KC_ROTATION, st, [&] {
        return launch_score_only(plan->n_order, corr, pr.mixed, d_w, pr.X, pr.Y, pr.Z, box,
                                 d_score, st, &plan->launches);
    }));
    TTM_TRY(timed(plan, KC_PEAKS, st, [&] {
        return launch_peak_candidates_full(d_score, nullptr, nullptr, pr.X, pr.Y, pr.Z, threshold,
                                           radius, tmp_a, tmp_b, list, cap, d_count, st,
                                           &plan->launches);
    }));
    // rotations at the peaks only: the record list is the unit list (voxel
    // index first, 8 words per record), q and lambda go into the records
    UnitList ul;
    ul.idx = (const int*)list;
    ul.stride = 8;
    ul.count = d_count;
    ul.out_stride = 8;
    TTM_TRY(timed(plan, KC_ROTATION, st, [&] {
        return launch_rotation_search(plan->n_order, corr, pr.mixed, d_w, nv, box, 0,
                                      (uint32_t)cap, plan->grid, cand, d_status, d_score, st,
                                      &plan->launches, ul);
    }));
    TTM_TRY(timed(plan, KC_POLISH, st, [&] {
        return launch_rotation_polish(plan->n_order, corr, pr.mixed, d_w, nv, box, 0,
                                      (uint32_t)cap, plan->grid, cand, d_score,
                                      (float*)list + 3, (float*)list + 2, nullptr, st,
                                      &plan->launches, ul);
    }));
    TTM_TRY(copy_peaks_to_host(pr, d_count, list, cap, max_peaks, h_out, n_out, st));
    int dev_status = 0;
    TTM_CUDA_TRY(cudaMemcpy(&dev_status, d_status, sizeof(int), cudaMemcpyDeviceToHost));
    return dev_status == 0 ? TTM_OK : (ttm_status)dev_status;
}

}  // extern "C"
