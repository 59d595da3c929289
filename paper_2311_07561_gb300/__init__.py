"""GB300 (sm_103a) tensorial template matching.

Hot path of Almira, Phelippeau & Martinez-Sanchez, "Fast Normalized
Cross-Correlation for Template Matching with Rotations" (arXiv 2311.07561):
tensor-template build (Sec. 3.2), local NCC statistics (Sec. 2, Algorithm 1),
correlation with the K tensor components, the Frobenius position score and the
dominant Z-eigenvector rotation per voxel (Sec. 3.3-3.4), and peak extraction.

The engine is ``libttm.so`` (C ABI in ``include/ttm.h``); this package is its
ctypes binding plus a small convenience layer.  PyTorch provides device memory
and streams only.
"""

from ._binding import (  # noqa: F401
    EXPORTED,
    LIB_PATH,
    PEAK_DTYPE,
    TTM_PATH_AUTO,
    TTM_PATH_DIRECT,
    TTM_PATH_FFT,
    TTM_PATH_TUNE,
    TTM_PREC_FP32,
    TTM_PREC_MIXED,
    TTM_NOALLOC_SCRATCH_BYTES,
    PlanOpts,
    TTDesc,
    TTMError,
    load_library,
    ttm_build_tensor_template,
    ttm_build_tensor_template_noalloc,
    ttm_build_workspace_size,
    ttm_classical_ncc,
    ttm_classical_workspace_size,
    ttm_correlate,
    ttm_device_count,
    ttm_extract_peaks,
    ttm_match_peaks,
    ttm_lowpass,
    ttm_kernel_class_name,
    ttm_local_stats,
    ttm_plan,
    ttm_plan_destroy,
    ttm_plan_device_status,
    ttm_plan_enable_timing,
    ttm_plan_launch_count,
    ttm_plan_waves,
    ttm_probe_bounded_wait,
    ttm_plan_problem_path,
    ttm_plan_problem_fft_box,
    ttm_plan_problem_tuning,
    ttm_plan_problem_tensor_direct,
    ttm_plan_timing,
    ttm_plan_workspace_size,
    ttm_status_string,
)
from .engine import HostPipeline, HostStream, Matcher, build_template  # noqa: F401
