"""The allocation-free tensor-template build.

ttm_build_tensor_template_noalloc serves callers that cannot allocate device
memory (a host application that owns all GPU memory through its own pool or
budget, or a pipeline that cannot take cudaMalloc's implicit synchronisation):
it takes its scratch from a fixed array inside the library instead of a
workspace.  These tests call it through the C ABI twice in a row, on different
inputs so that leftovers of the first call in the shared array would show, and
check each result against the regular entry point on the same inputs.  This
file is collected last so that a run stopping at the first failure has already
run every other test.
"""

import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ttm():
    import os
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2311_07561_gb300 as ttm
    if not os.path.exists(ttm.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    ttm.load_library()
    return ttm


def _inputs(s, r, n_rot, seed):
    import torch
    t = torch.from_numpy(synth.blob_template(s, 5, seed=seed)).cuda()
    m = torch.from_numpy(synth.ball_mask(s, r)).cuda()
    q = torch.from_numpy(synth.shoemake_quaternions(n_rot, seed).astype(np.float32)).cuda()
    return t, m, q


def _both(ttm, s, r, n, n_rot, seed):
    import torch
    t, m, q = _inputs(s, r, n_rot, seed)
    K = (n + 1) * (n + 2) * (n + 3) // 6
    ref = torch.empty((K, s, s, s), dtype=torch.float32, device="cuda")
    ws = torch.empty(ttm.ttm_build_workspace_size(s, n, n_rot), dtype=torch.uint8, device="cuda")
    d_ref = ttm.ttm_build_tensor_template(t, m, s, n, q, None, n_rot, ref, ws)
    got = torch.full((K, s, s, s), float("nan"), dtype=torch.float32, device="cuda")
    d_got = ttm.ttm_build_tensor_template_noalloc(t, m, s, n, q, None, n_rot, got)
    torch.cuda.synchronize()
    return ref.cpu().numpy(), got.cpu().numpy(), d_ref, d_got


def test_noalloc_build_matches_regular_build_twice_in_a_row(ttm):
    # a large first call (many chunks through the fixed array), then a
    # smaller, different one
    for (s, r, n, n_rot, seed) in [(32, 15, 4, 700, 1), (15, 7, 6, 300, 2)]:
        ref, got, d_ref, d_got = _both(ttm, s, r, n, n_rot, seed)
        assert np.all(np.isfinite(got))
        err = np.abs(got - ref).max()
        assert err <= 2e-5 * np.abs(ref).max(), (s, err)
        assert (d_got.K, d_got.s, d_got.centre, d_got.n_rot) == (d_ref.K, d_ref.s, d_ref.centre, d_ref.n_rot)
        assert d_got.mask_sum == d_ref.mask_sum


def test_noalloc_build_rejects_boxes_beyond_its_scratch(ttm):
    lib = ttm.load_library()
    desc = ttm.TTDesc()
    # s = 128 needs 8 MiB for one rotated copy plus the header: more than the array
    st = lib.ttm_build_tensor_template_noalloc(256, 256, 128, 4, 256, None, 10, 256,
                                               ctypes.byref(desc), None)
    assert st == -7
    assert lib.ttm_build_tensor_template_noalloc(None, None, 32, 4, None, None, 10, None,
                                                 ctypes.byref(desc), None) == -1
    # a float array that is not 4-byte aligned is refused on the host, before
    # the scratch address is looked up or anything is queued
    for bad in range(4):
        ptrs = [256, 256, 256, 256, None]
        ptrs[bad] = 257
        t, m, q, out, wts = ptrs
        assert lib.ttm_build_tensor_template_noalloc(t, m, 32, 4, q, wts, 10, out,
                                                     ctypes.byref(desc), None) == -1
    assert lib.ttm_build_tensor_template_noalloc(256, 256, 32, 4, 256, 258, 10, 256,
                                                 ctypes.byref(desc), None) == -1


def test_noalloc_build_allocates_no_device_memory(ttm):
    """Once the library's kernels are loaded (the calls above, or a first
    call here), a further call leaves the device's free memory unchanged: the
    outputs are the caller's and the scratch is the library's fixed array."""
    import torch
    s, r, n, n_rot = 24, 11, 4, 500
    t, m, q = _inputs(s, r, n_rot, 3)
    K = (n + 1) * (n + 2) * (n + 3) // 6
    out = torch.empty((K, s, s, s), dtype=torch.float32, device="cuda")
    ttm.ttm_build_tensor_template_noalloc(t, m, s, n, q, None, n_rot, out)
    torch.cuda.synchronize()
    first = out.clone()
    free0, _ = torch.cuda.mem_get_info()
    ttm.ttm_build_tensor_template_noalloc(t, m, s, n, q, None, n_rot, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.equal(out, first)
