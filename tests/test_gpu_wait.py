"""Bounded device-side waits: the poll loop every tensor-core kernel waits
on its mbarriers with ends, and reports TTM_ERR_TIMEOUT, when the phase it
waits for never completes.  The wait here is on a phase that nothing
completes (a barrier no thread arrives on), with a short host-given poll
limit; no fault, trap or endless loop is involved, and the context stays
usable afterwards."""

import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TTM_ERR_TIMEOUT = -5          # include/ttm.h


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


def test_wait_on_a_completed_phase_returns_ok(ttm):
    assert ttm.ttm_probe_bounded_wait(1000, True) == 0


@pytest.mark.parametrize("polls", [1, 100, 1000])
def test_wait_that_nothing_completes_runs_out(ttm, polls):
    import torch
    t0 = time.perf_counter()
    assert ttm.ttm_probe_bounded_wait(polls, False) == TTM_ERR_TIMEOUT
    elapsed = time.perf_counter() - t0
    print(f"{polls} polls ran out in {elapsed * 1e3:.2f} ms")
    assert elapsed < 30.0
    # the context still runs work: a device computation right after
    x = torch.arange(1000, dtype=torch.float32, device="cuda")
    assert float(x.sum()) == pytest.approx(499500.0)
    assert ttm.ttm_probe_bounded_wait(10, True) == 0


def test_the_kernels_wait_limit_ends_within_seconds(ttm):
    """The tensor-core kernels give up after 2^18 polls: about a second."""
    t0 = time.perf_counter()
    assert ttm.ttm_probe_bounded_wait(1 << 18, False) == TTM_ERR_TIMEOUT
    elapsed = time.perf_counter() - t0
    print(f"2^18 polls ran out in {elapsed:.2f} s")
    assert elapsed < 10.0
