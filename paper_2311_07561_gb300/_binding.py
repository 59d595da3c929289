"""ctypes binding of libttm.so (the C ABI declared in include/ttm.h).

Argument marshalling only: every function has the name of the C entry point
it calls, turns torch tensors into device pointers, lists into pointer arrays
and a non-zero status into :class:`TTMError`.  All arithmetic runs in the
library's CUDA kernels; there is no fallback of any kind.
"""

from __future__ import annotations

import ctypes
import os
from typing import Any, List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libttm.so")

TTM_OK = 0
STATUS_NAMES = {
    0: "TTM_OK", -1: "TTM_ERR_INVALID_ARG", -2: "TTM_ERR_UNSUPPORTED",
    -3: "TTM_ERR_OUT_OF_MEMORY", -4: "TTM_ERR_CUDA", -5: "TTM_ERR_TIMEOUT",
    -6: "TTM_ERR_NUMERIC", -7: "TTM_ERR_WORKSPACE",
}
TTM_PATH_AUTO, TTM_PATH_DIRECT, TTM_PATH_FFT, TTM_PATH_TUNE = 0, 1, 2, 3
TTM_PREC_FP32, TTM_PREC_MIXED = 0, 1

# Every symbol include/ttm.h declares.
EXPORTED = (
    "ttm_status_string", "ttm_device_count", "ttm_build_workspace_size",
    "ttm_build_tensor_template", "ttm_plan", "ttm_plan_workspace_size",
    "ttm_plan_problem_path", "ttm_plan_problem_fft_box", "ttm_plan_problem_tuning",
    "ttm_plan_problem_tensor_direct",
    "ttm_plan_launch_count", "ttm_plan_waves", "ttm_probe_bounded_wait", "ttm_plan_destroy",
    "ttm_local_stats", "ttm_correlate", "ttm_extract_peaks", "ttm_match_peaks", "ttm_lowpass",
    "ttm_plan_enable_timing",
    "ttm_plan_timing", "ttm_kernel_class_name", "ttm_build_tensor_template_noalloc",
    "ttm_plan_device_status", "ttm_classical_workspace_size", "ttm_classical_ncc",
)
TTM_NOALLOC_SCRATCH_BYTES = 8388608
TTM_KERNEL_CLASSES = 13


class TTMError(RuntimeError):
    def __init__(self, status: int, call: str):
        self.status = status
        super().__init__(f"{call} failed: {STATUS_NAMES.get(status, status)}")


class TTDesc(ctypes.Structure):
    _fields_ = [("n_order", ctypes.c_int), ("K", ctypes.c_int), ("s", ctypes.c_int),
                ("centre", ctypes.c_int), ("n_rot", ctypes.c_int), ("reserved", ctypes.c_int),
                ("mask_sum", ctypes.c_double)]


class Peak(ctypes.Structure):
    _fields_ = [("x", ctypes.c_int), ("y", ctypes.c_int), ("z", ctypes.c_int),
                ("score", ctypes.c_float), ("lambda_", ctypes.c_float),
                ("q", ctypes.c_float * 4)]


class PlanOpts(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int), ("precision", ctypes.c_int), ("n_grid", ctypes.c_int),
                ("n_cells", ctypes.c_int), ("n_candidates", ctypes.c_int),
                ("newton_steps", ctypes.c_int), ("rotation_chunks", ctypes.c_int),
                ("lowpass_sigma", ctypes.c_float), ("n_refined", ctypes.c_int),
                ("batch_mib", ctypes.c_int)]


_lib: Optional[ctypes.CDLL] = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libttm.so (built by ``__graft_entry__.build()``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: the CUDA engine has not been built "
                           "(run `python -c 'import __graft_entry__ as g; g.build()'`)")
    lib = ctypes.CDLL(path)
    P, I, L, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_size_t
    PP = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "ttm_status_string": (ctypes.c_char_p, [I]),
        "ttm_device_count": (I, []),
        "ttm_build_workspace_size": (I, [I, I, I, ctypes.POINTER(S)]),
        "ttm_build_tensor_template": (I, [P, P, I, I, P, P, I, P, P, S, ctypes.POINTER(TTDesc), P]),
        "ttm_plan": (I, [ctypes.POINTER(P), I, ctypes.POINTER(I), ctypes.POINTER(I), I,
                         ctypes.POINTER(TTDesc), PP, PP, ctypes.POINTER(PlanOpts), P]),
        "ttm_plan_workspace_size": (I, [P, ctypes.POINTER(S)]),
        "ttm_plan_problem_path": (I, [P, I, ctypes.POINTER(I)]),
        "ttm_plan_problem_fft_box": (I, [P, I, ctypes.POINTER(I)]),
        "ttm_plan_problem_tensor_direct": (I, [P, I, ctypes.POINTER(I)]),
        "ttm_plan_problem_tuning": (I, [P, I, ctypes.POINTER(ctypes.c_double)]),
        "ttm_plan_launch_count": (I, [P, ctypes.POINTER(L)]),
        "ttm_plan_waves": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I)]),
        "ttm_probe_bounded_wait": (I, [L, I, ctypes.POINTER(I), P]),
        "ttm_plan_destroy": (None, [P]),
        "ttm_local_stats": (I, [P, PP, PP, P, S, P]),
        "ttm_correlate": (I, [P, PP, PP, PP, PP, PP, PP, P, S, P]),
        "ttm_extract_peaks": (I, [P, I, P, P, P, ctypes.c_float, I, I, ctypes.POINTER(Peak),
                                  ctypes.POINTER(I), P, S, P]),
        "ttm_match_peaks": (I, [P, I, P, P, P, ctypes.c_float, I, I, ctypes.POINTER(Peak),
                                ctypes.POINTER(I), P, S, P]),
        "ttm_lowpass": (I, [P, I, I, I, ctypes.c_float, P, P, P]),
        "ttm_plan_enable_timing": (I, [P, I]),
        "ttm_plan_timing": (I, [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(L), I]),
        "ttm_kernel_class_name": (ctypes.c_char_p, [I]),
        "ttm_plan_device_status": (I, [P, P, S, P]),
        "ttm_classical_workspace_size": (I, [P, I, ctypes.POINTER(S)]),
        "ttm_classical_ncc": (I, [P, I, P, P, I, P, P, P, P, P, S, P]),
        "ttm_build_tensor_template_noalloc": (I, [P, P, I, I, P, P, I, P,
                                                  ctypes.POINTER(TTDesc), P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------

def _ptr(x: Any) -> Optional[int]:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    raise TypeError(f"cannot pass {type(x)} as a device pointer")


def _ptrs(xs: Optional[Sequence[Any]]):
    if xs is None:
        return None
    arr = (ctypes.c_void_p * len(xs))()
    for i, x in enumerate(xs):
        arr[i] = _ptr(x)
    return arr


def _stream(stream: Any) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _nbytes(t: Any) -> int:
    return t.numel() * t.element_size()


def _check(status: int, call: str) -> None:
    if status != TTM_OK:
        raise TTMError(status, call)


# ---------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ---------------------------------------------------------------------------

def ttm_status_string(status: int) -> str:
    return load_library().ttm_status_string(status).decode()


def ttm_device_count() -> int:
    return load_library().ttm_device_count()


def ttm_build_workspace_size(s: int, n_order: int, n_rot: int) -> int:
    out = ctypes.c_size_t()
    _check(load_library().ttm_build_workspace_size(s, n_order, n_rot, ctypes.byref(out)),
           "ttm_build_workspace_size")
    return out.value


def ttm_build_tensor_template(template, mask, s: int, n_order: int, quats, weights, n_rot: int,
                              components, workspace, stream=None) -> TTDesc:
    desc = TTDesc()
    st = load_library().ttm_build_tensor_template(
        _ptr(template), _ptr(mask), s, n_order, _ptr(quats), _ptr(weights), n_rot,
        _ptr(components), _ptr(workspace), _nbytes(workspace) if workspace is not None else 0,
        ctypes.byref(desc), _stream(stream))
    _check(st, "ttm_build_tensor_template")
    return desc


def ttm_build_tensor_template_noalloc(template, mask, s: int, n_order: int, quats, weights,
                                      n_rot: int, components, stream=None) -> TTDesc:
    """Same result as ttm_build_tensor_template without any workspace: the
    library's fixed scratch array is used (for callers that cannot allocate)."""
    desc = TTDesc()
    st = load_library().ttm_build_tensor_template_noalloc(
        _ptr(template), _ptr(mask), s, n_order, _ptr(quats), _ptr(weights), n_rot,
        _ptr(components), ctypes.byref(desc), _stream(stream))
    _check(st, "ttm_build_tensor_template_noalloc")
    return desc


def ttm_plan(vol_dims: Sequence[Sequence[int]], tmpl_index: Sequence[int],
             descs: Sequence[TTDesc], components: Sequence[Any], masks: Sequence[Any],
             opts: Optional[PlanOpts] = None, stream=None) -> int:
    """Create a plan; vol_dims holds (X, Y, Z) per problem.  Returns the handle."""
    n = len(vol_dims)
    dims = (ctypes.c_int * (3 * n))(*[int(v) for d in vol_dims for v in d])
    tix = (ctypes.c_int * n)(*[int(k) for k in tmpl_index])
    darr = (TTDesc * len(descs))(*descs)
    handle = ctypes.c_void_p()
    st = load_library().ttm_plan(ctypes.byref(handle), n, dims, tix, len(descs), darr,
                                 _ptrs(components), _ptrs(masks),
                                 ctypes.byref(opts) if opts is not None else None,
                                 _stream(stream))
    _check(st, "ttm_plan")
    return handle.value


def ttm_plan_workspace_size(plan: int) -> int:
    out = ctypes.c_size_t()
    _check(load_library().ttm_plan_workspace_size(plan, ctypes.byref(out)),
           "ttm_plan_workspace_size")
    return out.value


def ttm_plan_problem_path(plan: int, problem: int) -> int:
    out = ctypes.c_int()
    _check(load_library().ttm_plan_problem_path(plan, problem, ctypes.byref(out)),
           "ttm_plan_problem_path")
    return out.value


def ttm_plan_problem_fft_box(plan: int, problem: int) -> tuple:
    out = (ctypes.c_int * 3)()
    _check(load_library().ttm_plan_problem_fft_box(plan, problem, out),
           "ttm_plan_problem_fft_box")
    return tuple(out)


def ttm_plan_problem_tuning(plan: int, problem: int) -> tuple:
    """(direct ms, FFT ms) the autotuner measured for a problem; -1 = not timed."""
    out = (ctypes.c_double * 2)()
    _check(load_library().ttm_plan_problem_tuning(plan, problem, out), "ttm_plan_problem_tuning")
    return tuple(out)


def ttm_plan_problem_tensor_direct(plan: int, problem: int) -> bool:
    out = ctypes.c_int()
    _check(load_library().ttm_plan_problem_tensor_direct(plan, problem, ctypes.byref(out)),
           "ttm_plan_problem_tensor_direct")
    return bool(out.value)


def ttm_plan_launch_count(plan: int) -> int:
    out = ctypes.c_longlong()
    _check(load_library().ttm_plan_launch_count(plan, ctypes.byref(out)), "ttm_plan_launch_count")
    return out.value


def ttm_plan_waves(plan: int) -> list:
    """First problem of each resident wave (empty: one problem at a time)."""
    lib = load_library()
    n = ctypes.c_int()
    _check(lib.ttm_plan_waves(plan, ctypes.byref(n), None), "ttm_plan_waves")
    first = (ctypes.c_int * max(n.value, 1))()
    _check(lib.ttm_plan_waves(plan, ctypes.byref(n), first), "ttm_plan_waves")
    return list(first)[:n.value]


def ttm_probe_bounded_wait(polls: int, arrive: bool, stream=None) -> int:
    """Status of one bounded device-side wait on an mbarrier phase that the
    probe completes itself (arrive) or that nothing completes: TTM_OK or
    TTM_ERR_TIMEOUT."""
    out = ctypes.c_int()
    _check(load_library().ttm_probe_bounded_wait(polls, 1 if arrive else 0, ctypes.byref(out),
                                                 _stream(stream)), "ttm_probe_bounded_wait")
    return out.value


def ttm_plan_destroy(plan: Optional[int]) -> None:
    if plan:
        load_library().ttm_plan_destroy(plan)


def ttm_plan_enable_timing(plan: int, enable: bool = True) -> None:
    _check(load_library().ttm_plan_enable_timing(plan, 1 if enable else 0),
           "ttm_plan_enable_timing")


def ttm_plan_device_status(plan: int, workspace, stream=None) -> int:
    """Status the kernels recorded since the last ttm_correlate (0 = fine)."""
    return load_library().ttm_plan_device_status(plan, _ptr(workspace), _nbytes(workspace),
                                                   _stream(stream))


def ttm_kernel_class_name(kernel_class: int) -> str:
    return load_library().ttm_kernel_class_name(kernel_class).decode()


def ttm_plan_timing(plan: int) -> dict:
    """{class name: (milliseconds, launches)} accumulated since the last call."""
    ms = (ctypes.c_double * TTM_KERNEL_CLASSES)()
    n = (ctypes.c_longlong * TTM_KERNEL_CLASSES)()
    _check(load_library().ttm_plan_timing(plan, ms, n, TTM_KERNEL_CLASSES), "ttm_plan_timing")
    return {ttm_kernel_class_name(c): (ms[c], n[c]) for c in range(TTM_KERNEL_CLASSES) if n[c]}


def ttm_local_stats(plan: int, vols: Sequence[Any], w: Sequence[Any], workspace,
                    stream=None) -> None:
    st = load_library().ttm_local_stats(plan, _ptrs(vols), _ptrs(w), _ptr(workspace),
                                        _nbytes(workspace), _stream(stream))
    _check(st, "ttm_local_stats")


def ttm_correlate(plan: int, vols: Sequence[Any], w: Sequence[Any], score: Sequence[Any],
                  quat: Sequence[Any], lam: Optional[Sequence[Any]] = None,
                  components_out: Optional[Sequence[Any]] = None, workspace=None,
                  stream=None) -> None:
    st = load_library().ttm_correlate(plan, _ptrs(vols), _ptrs(w), _ptrs(score), _ptrs(quat),
                                      _ptrs(lam), _ptrs(components_out), _ptr(workspace),
                                      _nbytes(workspace) if workspace is not None else 0,
                                      _stream(stream))
    _check(st, "ttm_correlate")


def ttm_classical_workspace_size(plan: int, problem: int) -> int:
    out = ctypes.c_size_t()
    _check(load_library().ttm_classical_workspace_size(plan, problem, ctypes.byref(out)),
           "ttm_classical_workspace_size")
    return out.value


def ttm_classical_ncc(plan: int, problem: int, template, quats, n_rot: int, vol, w, best,
                      best_index, workspace, stream=None) -> None:
    st = load_library().ttm_classical_ncc(plan, problem, _ptr(template), _ptr(quats), n_rot,
                                          _ptr(vol), _ptr(w), _ptr(best), _ptr(best_index),
                                          _ptr(workspace), _nbytes(workspace), _stream(stream))
    _check(st, "ttm_classical_ncc")


PEAK_DTYPE = np.dtype([("x", np.int32), ("y", np.int32), ("z", np.int32), ("score", np.float32),
                       ("lambda", np.float32), ("q", np.float32, 4)])


def ttm_extract_peaks(plan: int, problem: int, score, quat, lam, threshold: float, radius: int,
                      max_peaks: int, workspace, stream=None) -> np.ndarray:
    buf = (Peak * max(max_peaks, 1))()
    n = ctypes.c_int()
    st = load_library().ttm_extract_peaks(plan, problem, _ptr(score), _ptr(quat), _ptr(lam),
                                          float(threshold), radius, max_peaks, buf,
                                          ctypes.byref(n), _ptr(workspace), _nbytes(workspace),
                                          _stream(stream))
    _check(st, "ttm_extract_peaks")
    raw = np.frombuffer(bytes(buf), dtype=PEAK_DTYPE, count=max(max_peaks, 1))
    return raw[: n.value].copy()


def ttm_match_peaks(plan: int, problem: int, vol, w, score, threshold: float, radius: int,
                    max_peaks: int, workspace, stream=None) -> np.ndarray:
    """Score map into `score`, then the rotation only at its peaks; returns the
    peak records (x, y, z, score, lambda, q) sorted by score."""
    buf = (Peak * max(max_peaks, 1))()
    n = ctypes.c_int()
    st = load_library().ttm_match_peaks(plan, problem, _ptr(vol), _ptr(w), _ptr(score),
                                        float(threshold), radius, max_peaks, buf,
                                        ctypes.byref(n), _ptr(workspace), _nbytes(workspace),
                                        _stream(stream))
    _check(st, "ttm_match_peaks")
    raw = np.frombuffer(bytes(buf), dtype=PEAK_DTYPE, count=max(max_peaks, 1))
    return raw[: n.value].copy()


def ttm_lowpass(x, sigma: float, tmp=None, out=None, stream=None):
    """Gaussian prefilter of a float32 cuda array (Z, Y, X) or (s, s, s);
    returns the filtered array (allocated with torch unless out is given)."""
    import torch
    if out is None:
        out = torch.empty_like(x)
    if tmp is None:
        tmp = torch.empty_like(x)
    Z, Y, X = x.shape
    _check(load_library().ttm_lowpass(_ptr(x), X, Y, Z, float(sigma), _ptr(tmp), _ptr(out),
                                      _stream(stream)), "ttm_lowpass")
    return out
