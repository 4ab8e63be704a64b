"""Read-only clock queries against the real NVML on a GPU: the SM clocks it
supports at the running memory clock, and the current/maximum SM clock.  Nothing
here locks or changes a clock."""
import pytest

import paper_2505_06022_gb300 as sy

from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu


def test_supported_and_current_clocks():
    torch_cuda()
    idx = sy.sy_clock_nvml_index(0)
    mem, clocks = sy.sy_clock_supported(idx)
    cur, mx = sy.sy_clock_current(idx)
    assert mem > 0 and len(clocks) > 0
    assert all(a > b for a, b in zip(clocks, clocks[1:]))  # highest first, no repeats
    assert 0 < cur <= mx and min(clocks) <= mx
    print(f"memory {mem} MHz; {len(clocks)} SM clocks {clocks[0]}..{clocks[-1]} MHz; current {cur}, max {mx}")
