"""Host-side checks of HostStream's volume sharing (no GPU): a problem ->
volume map must give one index per problem, indices 0 .. n-1, and one size
per volume; the checks run before any device memory is touched."""

import pytest

import paper_2311_07561_gb300 as ttm


class _FakeMatcher:
    def __init__(self, problems):
        self.problems = problems

    def new_outputs(self):            # reached only when the checks pass
        raise AssertionError("device memory requested")


PROBLEMS = [((40, 30, 20), 0), ((40, 30, 20), 1), ((50, 30, 20), 0), ((50, 30, 20), 1)]


@pytest.mark.parametrize("volume_of, message", [
    ([0, 0, 1], "one volume index per problem"),
    ([0, 0, 2, 2], "0 .. n-1"),
    ([0, 0, 0, 1], "differ in size"),
])
def test_volume_map_is_checked_first(volume_of, message):
    with pytest.raises(ValueError, match=message):
        ttm.HostStream(matcher=_FakeMatcher(PROBLEMS), volume_of=volume_of)


def test_a_valid_map_reaches_the_device_allocations():
    # past the checks: the device step (no CUDA device here: the package
    # says so; with one, the fake matcher's allocation guard fires)
    with pytest.raises((AssertionError, RuntimeError), match="device"):
        ttm.HostStream(matcher=_FakeMatcher(PROBLEMS), volume_of=[0, 0, 1, 1])


def test_depth_is_checked():
    with pytest.raises(ValueError, match="depth"):
        ttm.HostStream(matcher=_FakeMatcher(PROBLEMS), depth=0)
