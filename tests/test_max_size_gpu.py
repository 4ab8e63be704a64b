"""Fields past 2^31 elements: every element offset and byte offset the kernels form
needs 64 bits.  SAXPY, the 2D whole run and the 3D whole run are checked bit for bit
against the oracle.

Inputs are a small block from the seeded generator repeated across the field on the
device, so the oracle works on small host arrays: SAXPY's result repeats with the
block's period (every element is compared on the device), and a stencil point after a
few steps depends only on the box of its light cone, which the host builds from the
block by modular indexing."""
import numpy as np
import pytest

import oracle
import paper_2505_06022_gb300 as sy
from paper_2505_06022_gb300 import inputs

from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu

TWO31 = 1 << 31


@pytest.fixture(scope="module")
def q():
    torch_cuda()
    with sy.Queue(0) as queue:
        yield queue.handle


def _free(torch):
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def test_saxpy_past_2_31_elements(q):
    torch = torch_cuda()
    period = 1 << 20
    n = TWO31 + 77  # the last vector ends past element 2^31; a ragged scalar tail follows
    xp, yp = inputs.saxpy_inputs(period, seed=9)
    want = torch.from_numpy(oracle.saxpy_f32(2.5, xp, yp).view(np.int32)).cuda()
    reps = -(-n // period)
    xd = torch.from_numpy(xp).cuda().repeat(reps)[:n]
    yd = torch.from_numpy(yp).cuda().repeat(reps)[:n]
    zd = torch.empty(n, dtype=torch.float32, device="cuda")
    sy.sy_saxpy(q, n, 2.5, xd, yd, zd)
    torch.cuda.synchronize()
    got = zd.view(torch.int32)
    whole = (n // period) * period
    assert torch.equal(got[:whole].view(-1, period), want.expand(n // period, period))
    assert torch.equal(got[whole:], want[: n - whole])
    del xd, yd, zd, got
    _free(torch)


def _tiled_2d(torch, block, ny, nx):
    """Device field (ny, nx) with element (i, j) = block[i % by, j % bx]."""
    by, bx = block.shape
    band = torch.from_numpy(block).cuda().repeat(1, -(-nx // bx))[:, :nx].contiguous()
    return band.repeat(-(-ny // by), 1)[:ny]


def test_wave_run_past_2_31_points(q):
    torch = torch_cuda()
    ny, nx = 32771, 65552  # 2.148e9 points; 16-byte rows; 4 chunks of ~8192 rows
    steps, r, c2 = 3, 1, 0.25
    block = inputs.random_field(21, 61, 1040)
    u0 = _tiled_2d(torch, block, ny, nx)
    ua, ub = torch.empty_like(u0), torch.empty_like(u0)
    p = sy.stencil_params(ny, nx, r, c2, "f32")
    chunks = sy.sy_split_rows(ny, 4)
    _, cv, _ = sy.sy_wave_run(q, p, u0, ua, ub, steps, chunks, r)
    torch.cuda.synchronize()
    cur = {u0.data_ptr(): u0, ua.data_ptr(): ua, ub.data_ptr(): ub}[cv]
    row31 = TWO31 // nx  # the row holding element 2^31
    col31 = TWO31 - row31 * nx
    samples = [(row31, col31), (row31, col31 - 1), (row31 + 1, 0), (row31 - 1, nx - 1), (0, 0), (ny - 1, nx - 1),
               (ny - 1, 0), (0, nx - 1), (chunks[1][0], 5), (chunks[1][0] - 1, 777), (chunks[3][0], nx - 2),
               (chunks[3][1] - 1, 40000), (20000, 32768)]
    h = (steps + 1) * r + 1
    for i, j in samples:
        rows = np.arange(max(0, i - h), min(ny, i + h + 1))
        cols = np.arange(max(0, j - h), min(nx, j + h + 1))
        box = np.ascontiguousarray(block[np.ix_(rows % block.shape[0], cols % block.shape[1])])
        _, m = oracle.wave_run_mirror(oracle.F32, box, steps, r, c2)
        got = np.float32(cur[i, j].item())
        assert got.view(np.uint32) == m[i - rows[0], j - cols[0]].view(np.uint32), (i, j)
    del u0, ua, ub, cur
    _free(torch)


def test_wave3d_run_past_2_31_points(q):
    torch = torch_cuda()
    nz, ny, nx = 1031, 1040, 2008  # 2.153e9 points; the plane holding element 2^31 is 1028
    steps, r, c2 = 2, 1, 0.125
    block = inputs.random_field_3d(23, 7, 13, 136)
    bz, by, bx = block.shape
    plane = _tiled_2d(torch, np.ascontiguousarray(block.reshape(bz * by, bx)), bz * by, nx)  # (bz*by, nx)
    slab = plane.view(bz, by, nx).repeat(1, -(-ny // by), 1)[:, :ny].contiguous()  # (bz, ny, nx)
    u0 = slab.repeat(-(-nz // bz), 1, 1)[:nz].reshape(-1)
    del plane, slab
    ua, ub = torch.empty_like(u0), torch.empty_like(u0)
    p = sy.stencil3d_params(nz, ny, nx, r, c2, "f32")
    chunks = sy.sy_split_rows(nz, 4)
    _, cv, _ = sy.sy_wave3d_run(q, p, u0, ua, ub, steps, chunks, r)
    torch.cuda.synchronize()
    cur = {u0.data_ptr(): u0, ua.data_ptr(): ua, ub.data_ptr(): ub}[cv].view(nz, ny, nx)
    z31 = TWO31 // (ny * nx)
    rest = TWO31 - z31 * ny * nx
    y31, x31 = rest // nx, rest % nx
    samples = [(z31, y31, x31), (z31, y31, x31 - 1), (z31 + 1, 0, 0), (0, 0, 0), (nz - 1, ny - 1, nx - 1),
               (chunks[2][0], 500, 1000), (chunks[2][0] - 1, ny - 1, 3), (nz - 1, 0, nx - 1), (700, 520, 1999)]
    h = (steps + 1) * r + 1
    for pt in samples:
        ax = [np.arange(max(0, c - h), min(n, c + h + 1)) for c, n in zip(pt, (nz, ny, nx))]
        box = np.ascontiguousarray(block[np.ix_(ax[0] % bz, ax[1] % by, ax[2] % bx)])
        _, m = oracle.wave3d_run_mirror(oracle.F32, box, steps, r, c2)
        got = np.float32(cur[pt].item())
        assert got.view(np.uint32) == m[tuple(c - a[0] for c, a in zip(pt, ax))].view(np.uint32), pt
    del u0, ua, ub, cur
    _free(torch)
