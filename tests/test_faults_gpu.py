"""Failure paths, injected on the host (nothing faults or hangs the GPU):
NVML missing (SY_FAULT=nvml_missing) turns every energy query into
SY_ERR_NVML_UNAVAILABLE while timing keeps working; bad device indices and
misuse of metering windows are reported as status codes."""
import os

import pytest

import paper_2505_06022_gb300 as sy

from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture
def nvml_missing():
    old = os.environ.get("SY_FAULT")
    os.environ["SY_FAULT"] = "nvml_missing"
    yield
    if old is None:
        del os.environ["SY_FAULT"]
    else:
        os.environ["SY_FAULT"] = old


def test_energy_queries_report_nvml_unavailable(nvml_missing):
    torch = torch_cuda()
    with sy.Queue(0) as q:
        with pytest.raises(sy.SyError) as e:
            sy.sy_energy_read(q.handle)
        assert e.value.name == "SY_ERR_NVML_UNAVAILABLE"
        with pytest.raises(sy.SyError) as e:
            sy.sy_device_energy(q.handle)
        assert e.value.name == "SY_ERR_NVML_UNAVAILABLE"
        a, b, c = (torch.zeros(64, 128, device="cuda") for _ in range(3))
        p = sy.stencil_params(64, 128, 1, 0.25, "f32")
        sy.sy_meter_begin(q.handle)  # the window opens; it just has no energy reading
        evs = sy.sy_stencil_step(q.handle, p, a, b, c, [(0, 64)], 1, want_events=True)
        with pytest.raises(sy.SyError) as e:
            sy.sy_meter_end(q.handle)
        assert e.value.name == "SY_ERR_NVML_UNAVAILABLE"
        with pytest.raises(sy.SyError) as e:
            sy.sy_kernel_energy(q.handle, evs[0])
        assert e.value.name == "SY_ERR_NVML_UNAVAILABLE"
        assert sy.sy_event_elapsed(q.handle, evs[0]) > 0  # timing does not depend on NVML


def test_queue_and_window_misuse():
    torch_cuda()
    with pytest.raises(sy.SyError) as e:
        sy.sy_queue_create(1 << 20)
    assert e.value.name == "SY_ERR_INVALID_ARGUMENT"
    with sy.Queue(0) as q:
        with pytest.raises(sy.SyError) as e:
            sy.sy_meter_end(q.handle)  # no window open
        assert e.value.name == "SY_ERR_INVALID_ARGUMENT"
        try:
            sy.sy_meter_begin(q.handle)
        except sy.SyError:
            pass
        with pytest.raises(sy.SyError) as e:
            sy.sy_meter_begin(q.handle)  # already open
        assert e.value.name == "SY_ERR_INVALID_ARGUMENT"
        try:
            sy.sy_meter_end(q.handle)
        except sy.SyError as err:
            assert err.name == "SY_ERR_NVML_UNAVAILABLE"
        with pytest.raises(sy.SyError) as e:
            sy.sy_event_elapsed(q.handle, 123456789)
        assert e.value.name == "SY_ERR_INVALID_ARGUMENT"
