"""Checkpoint and resume: stepping on from a saved (u^{n-1}, u^n, n) gives the bits of the
uninterrupted run, also into a buffer with another pitch; foreign files are refused."""
import numpy as np
import pytest

import oracle
import paper_2505_06022_gb300 as sy
from paper_2505_06022_gb300 import inputs

from gpu_helpers import to_device, to_host, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    torch_cuda()
    with sy.Queue(0) as queue:
        yield queue.handle


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_resume_equals_uninterrupted_run(q, tmp_path, dtype):
    torch = torch_cuda()
    ny, nx, r = 96, 250, 2
    u0 = inputs.to_storage(inputs.gaussian_pulse(ny, nx, 9.0), dtype)
    p = sy.stencil_params(ny, nx, r, 0.25, dtype)
    chunks = sy.sy_split_rows(ny, 3)
    cur = to_device(u0)
    prev = torch.empty_like(cur)
    sy.sy_stencil_start(q, p, cur, prev, chunks, r)
    for _ in range(7):
        sy.sy_stencil_step(q, p, prev, cur, prev, chunks, r)
        prev, cur = cur, prev
    path = str(tmp_path / "ck.bin")
    sy.sy_checkpoint_save(q, path, p, prev, cur, 7)
    # resume into buffers with a wider pitch
    pitch = 264
    pp = sy.stencil_params(ny, nx, r, 0.25, dtype, pitch=pitch)
    tdt = torch.float32 if dtype == "f32" else torch.int16
    rp, rc = (torch.full((ny, pitch), 0, dtype=tdt, device="cuda") for _ in range(2))
    assert sy.sy_checkpoint_load(q, path, pp, rp, rc) == 7
    for _ in range(5):
        sy.sy_stencil_step(q, p, prev, cur, prev, chunks, r)
        prev, cur = cur, prev
        sy.sy_stencil_step(q, pp, rp, rc, rp, chunks, r)
        rp, rc = rc, rp
    torch.cuda.synchronize()
    st = np.float32 if dtype == "f32" else np.uint16
    a, b = to_host(cur, (ny, nx), st), to_host(rc, (ny, nx), st)
    assert np.array_equal(a.view(np.uint8), np.ascontiguousarray(b).view(np.uint8))
    _, want = oracle.wave_run_mirror(oracle.DTYPES[dtype], u0, 12, r, 0.25)
    assert np.array_equal(a.view(np.uint8), want.view(np.uint8))


def test_checkpoint_refuses_foreign_files(q, tmp_path):
    torch = torch_cuda()
    a, b = (torch.zeros(16, 32, device="cuda") for _ in range(2))
    p = sy.stencil_params(16, 32, 1, 0.25, "f32")
    path = str(tmp_path / "ck.bin")
    sy.sy_checkpoint_save(q, path, p, a, b, 3)
    other = sy.stencil_params(16, 32, 2, 0.25, "f32")
    with pytest.raises(sy.SyError) as e:
        sy.sy_checkpoint_load(q, path, other, a, b)
    assert e.value.name == "SY_ERR_INVALID_ARGUMENT"
    bad = tmp_path / "bad.bin"
    bad.write_bytes(b"not a checkpoint at all, just bytes" * 4)
    with pytest.raises(sy.SyError) as e:
        sy.sy_checkpoint_load(q, str(bad), p, a, b)
    assert e.value.name == "SY_ERR_IO"
    with pytest.raises(sy.SyError) as e:
        sy.sy_checkpoint_load(q, str(tmp_path / "missing.bin"), p, a, b)
    assert e.value.name == "SY_ERR_IO"
