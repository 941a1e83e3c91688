"""Runs last: no bounded wait of the signature kernel's warp pairs gave up
during the GPU tests (every hand-over between a pair's control and math warps
completed)."""
import pytest

pytestmark = pytest.mark.gpu


def test_no_bounded_wait_gave_up(cuda):
    assert cuda.device_faults() == 0
