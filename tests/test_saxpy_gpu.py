"""SAXPY on the GPU (paper §2 Listing 1; §3 Listing 2 split form) against the oracle:
bit-exact, since both sides compute fl(fl(alpha*x) + y) without FMA."""
import numpy as np
import pytest

import oracle
import paper_2505_06022_gb300 as sy
from paper_2505_06022_gb300 import inputs

from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    torch_cuda()
    with sy.Queue(0) as queue:
        yield queue.handle


def run(q, alpha, x, y, off=(0, 0, 0), inplace=None):
    torch = torch_cuda()
    n = x.size
    bufs = [torch.zeros(n + 8, dtype=torch.float32, device="cuda") for _ in range(3)]
    xs = bufs[0][off[0]: off[0] + n]
    ys = bufs[1][off[1]: off[1] + n]
    xs.copy_(torch.from_numpy(x))
    ys.copy_(torch.from_numpy(y))
    zs = bufs[2][off[2]: off[2] + n] if inplace is None else (xs if inplace == "x" else ys)
    sy.sy_saxpy(q, n, alpha, xs, ys, zs)
    torch.cuda.synchronize()
    return zs.cpu().numpy()


def test_config0_bit_exact(q):
    # SAXPY z = alpha*x + y, FP32, N = 2^20, alpha = 2.5, x, y uniform in [-1, 1) from seed 0
    n = 1 << 20
    x, y = inputs.saxpy_inputs(n, seed=0)
    z = run(q, 2.5, x, y)
    assert np.array_equal(z.view(np.uint32), oracle.saxpy_f32(2.5, x, y).view(np.uint32))


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 31, 1023, 4097, 65537])
@pytest.mark.parametrize("off", [(0, 0, 0), (1, 1, 1), (3, 3, 3), (1, 0, 2), (0, 2, 0)])
def test_ragged_and_misaligned(q, n, off):
    x, y = inputs.saxpy_inputs(n, seed=7)
    z = run(q, -1.75, x, y, off)
    assert np.array_equal(z.view(np.uint32), oracle.saxpy_f32(-1.75, x, y).view(np.uint32))


@pytest.mark.parametrize("which", ["x", "y"])
def test_in_place(q, which):
    n = 10007
    x, y = inputs.saxpy_inputs(n, seed=2)
    z = run(q, 3.0, x, y, inplace=which)
    assert np.array_equal(z.view(np.uint32), oracle.saxpy_f32(3.0, x, y).view(np.uint32))


def test_split_one_to_one_chunks(q):
    torch = torch_cuda()
    n = (1 << 16) + 13
    x, y = inputs.saxpy_inputs(n, seed=4)
    want = oracle.saxpy_f32(0.5, x, y)
    for chunks in [sy.sy_split_rows(n, 4), [(0, 1), (1, 2), (2, n)], [(0, n - 3), (n - 3, n)],
                   sy.sy_split_rows(n, 37)]:
        xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
        zd = torch.full_like(xd, float("nan"))
        evs = sy.sy_saxpy_split(q, n, 0.5, xd, yd, zd, chunks, want_events=True)
        torch.cuda.synchronize()
        assert np.array_equal(zd.cpu().numpy().view(np.uint32), want.view(np.uint32))
        assert len(evs) == len(chunks) and all(sy.sy_event_elapsed(q, e) >= 0 for e in evs)


def test_large_sampled(q):
    # N = 2^26 (768 MiB of traffic): every element checked against the oracle.
    torch = torch_cuda()
    n = 1 << 26
    x, y = inputs.saxpy_inputs(n, seed=0)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    zd = torch.empty_like(xd)
    sy.sy_saxpy(q, n, 2.5, xd, yd, zd)
    torch.cuda.synchronize()
    assert np.array_equal(zd.cpu().numpy().view(np.uint32), oracle.saxpy_f32(2.5, x, y).view(np.uint32))


def test_errors(q):
    torch = torch_cuda()
    buf = torch.zeros(100, device="cuda")
    with pytest.raises(sy.SyError) as e:
        sy.sy_saxpy(q, 50, 1.0, buf[0:50], buf[0:50], buf[10:60])
    assert e.value.name == "SY_ERR_ALIAS"
    with pytest.raises(sy.SyError) as e:
        sy.sy_saxpy(q, -1, 1.0, buf, buf, buf)
    assert e.value.name == "SY_ERR_INVALID_ARGUMENT"
    with pytest.raises(sy.SyError) as e:
        sy.sy_saxpy_split(q, 100, 1.0, buf, buf, buf, [(0, 40), (50, 100)])
    assert e.value.name == "SY_ERR_BAD_CHUNKS"
    sy.sy_saxpy(q, 0, 1.0, None, None, None)  # n == 0 is a no-op
    before = sy.sy_queue_launch_count(q)
    with pytest.raises(sy.SyError):
        sy.sy_saxpy(q, 50, 1.0, buf[0:50], buf[0:50], buf[1:51])
    assert sy.sy_queue_launch_count(q) == before  # a rejected call launches nothing
