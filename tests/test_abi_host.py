"""Host-side checks of the C ABI: the library loads, exports every symbol the
header declares, and rejects bad arguments before touching the GPU.  No
compute call is made, so these run without a GPU."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ttm.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ttm_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import paper_2311_07561_gb300 as ttm
    if not os.path.exists(ttm.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return ttm.load_library()


def test_header_declarations_match_binding():
    import paper_2311_07561_gb300 as ttm
    assert _declared() == sorted(ttm.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name
    # exported with C linkage (no C++ mangling)
    out = os.popen(f"nm -D --defined-only {lib._name}").read()
    for name in _declared():
        assert re.search(rf"\bT {name}$", out, flags=re.M), name


def test_status_strings(lib):
    import paper_2311_07561_gb300 as ttm
    for code, name in ttm._binding.STATUS_NAMES.items():
        assert ttm.ttm_status_string(code) == name
    assert ttm.ttm_status_string(-99) == "TTM_ERR_UNKNOWN"


def test_workspace_size_validation(lib):
    import paper_2311_07561_gb300 as ttm
    out = ctypes.c_size_t()
    assert lib.ttm_build_workspace_size(15, 3, 100, ctypes.byref(out)) == -2   # odd order
    assert lib.ttm_build_workspace_size(15, 10, 100, ctypes.byref(out)) == -2  # order too high
    assert lib.ttm_build_workspace_size(2, 4, 100, ctypes.byref(out)) == -1    # box too small
    assert lib.ttm_build_workspace_size(15, 4, 0, ctypes.byref(out)) == -1     # no rotations
    assert lib.ttm_build_workspace_size(15, 4, 100, None) == -1
    assert lib.ttm_build_workspace_size(15, 4, 100, ctypes.byref(out)) == 0
    assert out.value >= 256 + 100 * 15 ** 3 * 4
    assert ttm.ttm_build_workspace_size(32, 4, 10000) >= 256 + 1024 * 32 ** 3 * 4


def test_null_and_invalid_arguments_are_rejected_on_host(lib):
    import paper_2311_07561_gb300 as ttm
    desc = ttm.TTDesc()
    # null pointers
    assert lib.ttm_build_tensor_template(None, None, 15, 4, None, None, 10, None, None, 0,
                                         ctypes.byref(desc), None) == -1
    # missing workspace is reported as a workspace error
    assert lib.ttm_build_tensor_template(16, 16, 15, 4, 16, None, 10, 16, None, 0,
                                         ctypes.byref(desc), None) == -7
    handle = ctypes.c_void_p()
    assert lib.ttm_plan(None, 1, None, None, 1, None, None, None, None, None) == -1
    assert lib.ttm_plan(ctypes.byref(handle), 0, None, None, 1, None, None, None, None, None) == -1
    # bad descriptor: odd order
    d = ttm.TTDesc(n_order=3, K=20, s=15, centre=7, n_rot=10, reserved=0, mask_sum=100.0)
    dims = (ctypes.c_int * 3)(64, 64, 64)
    tix = (ctypes.c_int * 1)(0)
    ptrs = (ctypes.c_void_p * 1)(16)
    assert lib.ttm_plan(ctypes.byref(handle), 1, dims, tix, 1, ctypes.byref(d), ptrs, ptrs,
                        None, None) == -2
    # volume smaller than the box
    d = ttm.TTDesc(n_order=4, K=35, s=15, centre=7, n_rot=10, reserved=0, mask_sum=100.0)
    small = (ctypes.c_int * 3)(14, 64, 64)
    assert lib.ttm_plan(ctypes.byref(handle), 1, small, tix, 1, ctypes.byref(d), ptrs, ptrs,
                        None, None) == -1
    # template index out of range
    bad = (ctypes.c_int * 1)(1)
    assert lib.ttm_plan(ctypes.byref(handle), 1, dims, bad, 1, ctypes.byref(d), ptrs, ptrs,
                        None, None) == -1
    # plan options out of range, rejected before any device work
    dims = (ctypes.c_int * 3)(64, 64, 64)
    for field, value in (("path", 4), ("path", -1), ("precision", 2), ("n_grid", 70000),
                         ("n_grid", 1000), ("n_cells", 3000), ("n_candidates", 9),
                         ("newton_steps", 65), ("rotation_chunks", -1), ("n_cells", -4),
                         ("lowpass_sigma", 9.0), ("n_refined", 5), ("batch_mib", -1),
                         ("batch_mib", (1 << 20) + 1)):
        o_ = ttm.PlanOpts()
        setattr(o_, field, value)
        assert lib.ttm_plan(ctypes.byref(handle), 1, dims, tix, 1, ctypes.byref(d), ptrs, ptrs,
                            ctypes.byref(o_), None) == -1, (field, value)
    # calls on a null plan
    n = ctypes.c_int()
    assert lib.ttm_plan_waves(None, ctypes.byref(n), None) == -1
    # the bounded-wait probe: poll limit 1 .. 2^24, a status pointer
    assert lib.ttm_probe_bounded_wait(0, 0, ctypes.byref(n), None) == -1
    assert lib.ttm_probe_bounded_wait((1 << 24) + 1, 0, ctypes.byref(n), None) == -1
    assert lib.ttm_probe_bounded_wait(100, 0, None, None) == -1
    assert lib.ttm_local_stats(None, None, None, None, 0, None) == -1
    assert lib.ttm_correlate(None, None, None, None, None, None, None, None, 0, None) == -1
    assert lib.ttm_extract_peaks(None, 0, None, None, None, 0.0, 1, 1, None, ctypes.byref(n),
                                 None, 0, None) == -1
    lib.ttm_plan_destroy(None)


def test_no_gpu_here_means_cuda_error_not_fallback(lib):
    """Without a device the library reports TTM_ERR_CUDA; it has no CPU path."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    assert lib.ttm_device_count() == 0
    import paper_2311_07561_gb300 as ttm
    d = ttm.TTDesc(n_order=4, K=35, s=15, centre=7, n_rot=10, reserved=0, mask_sum=100.0)
    dims = (ctypes.c_int * 3)(64, 64, 64)
    tix = (ctypes.c_int * 1)(0)
    ptrs = (ctypes.c_void_p * 1)(256)
    handle = ctypes.c_void_p()
    assert lib.ttm_plan(ctypes.byref(handle), 1, dims, tix, 1, ctypes.byref(d), ptrs, ptrs,
                        None, None) == -4
