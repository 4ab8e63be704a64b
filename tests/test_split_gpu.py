"""Split-buffer execution on the GPU: every chunk in a buffer of its own, halos
moved by the transfers the range mappers infer (one halo-exchange kernel per step,
launches overlapped by programmatic dependent launch).  Must be bit-identical to the
oracle (and so to the shared-buffer mode), whatever the number of transfers, the
copy unit the row width allows, and with launch overlap turned off."""
import numpy as np
import pytest

import oracle
import paper_2505_06022_gb300 as sy
from paper_2505_06022_gb300 import inputs

from gpu_helpers import bits, torch_cuda

pytestmark = pytest.mark.gpu

DT = {"f32": oracle.F32, "bf16": oracle.BF16, "f16": oracle.F16}


@pytest.fixture(scope="module")
def q():
    torch_cuda()
    with sy.Queue(0) as queue:
        yield queue.handle


def to_local(u, chunks, h, c, pitch, tdt, torch):
    ny = u.shape[0]
    lo, hi, rows = sy.sy_split_layout(ny, chunks, h, c)
    a, b = chunks[c]
    buf = torch.zeros(rows, pitch, dtype=tdt, device="cuda")
    src = u if u.dtype == np.float32 else u.view(np.int16)
    buf[lo: lo + (b - a), : u.shape[1]] = torch.from_numpy(np.ascontiguousarray(src[a:b])).cuda()
    return buf


@pytest.mark.parametrize("dtype,r,h,ny,nx,chunks,variant", [
    ("f32", 1, 1, 64, 300, None, 0),
    ("f32", 2, 3, 37, 129, [(0, 1), (1, 3), (3, 30), (30, 37)], 0),     # chunks shorter than the halo
    ("bf16", 4, 4, 50, 520, [(0, 20), (20, 22), (22, 50)], 0),
    ("f16", 3, 3, 33, 70, [(0, 33)], 0),
    ("bf16", 1, 2, 61, 131, None, 0),                                   # odd row width: 2-byte copy unit
    ("f32", 1, 1, 160, 96, "many", 0),                                  # 38 transfers: two halo launches
    ("f16", 2, 3, 48, 200, [(i, i + 2) for i in range(0, 48, 2)], 0),   # every halo spans two owners
    ("bf16", 4, 4, 50, 520, [(0, 20), (20, 22), (22, 50)], 15),         # the march form in local buffers
    ("f16", 2, 3, 48, 200, [(i, i + 2) for i in range(0, 48, 2)], 15),
])
def test_split_buffers_bit_exact(q, dtype, r, h, ny, nx, chunks, variant):
    torch = torch_cuda()
    chunks = sy.sy_split_rows(ny, 20) if chunks == "many" else (chunks or sy.sy_split_rows(ny, 4))
    u0 = inputs.to_storage(inputs.gaussian_pulse(ny, nx, 6.0) + 0.05 * inputs.random_field(3, ny, nx), dtype)
    tdt = torch.float32 if dtype == "f32" else torch.int16
    pitch = (nx + 7) // 8 * 8
    cur = [to_local(u0, chunks, h, c, pitch, tdt, torch) for c in range(len(chunks))]
    prev = [torch.zeros_like(t) for t in cur]
    p = sy.stencil_params(ny, nx, r, 0.25, dtype, pitch=pitch, variant=variant)
    sy.sy_stencil_start_split(q, p, cur, prev, chunks, h)
    steps = 8
    for _ in range(steps):
        sy.sy_stencil_step_split(q, p, prev, cur, prev, chunks, h)
        prev, cur = cur, prev
    torch.cuda.synchronize()
    got = []
    for c, (a, b) in enumerate(chunks):
        lo, _, _ = sy.sy_split_layout(ny, chunks, h, c)
        part = cur[c][lo: lo + (b - a), :nx].cpu().numpy()
        got.append(part if dtype == "f32" else part.view(np.uint16))
    _, want = oracle.wave_run_mirror(DT[dtype], u0, steps, r, 0.25)
    assert np.array_equal(bits(np.ascontiguousarray(np.concatenate(got))), bits(want))


def test_step_rows_matches_chunked_step(q):
    torch = torch_cuda()
    ny, nx, r = 90, 256, 2
    u0 = inputs.to_storage(inputs.gaussian_pulse(ny, nx, 9.0), "f32")
    cur = torch.from_numpy(u0).cuda()
    prev = torch.empty_like(cur)
    p = sy.stencil_params(ny, nx, r, 0.25, "f32")
    for a, b in [(0, 31), (31, 32), (32, 90)]:  # the same rows as a chunk list, one call each
        sy.sy_stencil_step_rows(q, p, None, cur, prev, a, b, r, start=True)
    nxt = torch.empty_like(cur)
    for a, b in [(0, 45), (45, 90)]:
        sy.sy_stencil_step_rows(q, p, prev, cur, nxt, a, b, r)
    torch.cuda.synchronize()
    op, oc = oracle.wave_run_mirror(oracle.F32, u0, 1, r, 0.25)
    assert np.array_equal(nxt.cpu().numpy().view(np.uint32), oc.view(np.uint32))
    with pytest.raises(sy.SyError) as e:
        sy.sy_stencil_step_rows(q, p, prev, cur, nxt, 10, 91, r)
    assert e.value.name == "SY_ERR_BAD_CHUNKS"
    with pytest.raises(sy.SyError) as e:
        sy.sy_stencil_step_rows(q, p, prev, cur, nxt, 0, 10, 1)
    assert e.value.name == "SY_ERR_HALO_TOO_SMALL"


def test_step_planes_matches_chunked_3d_step(q):
    """sy_stencil3d_step_planes on plane ranges equals the chunked 3D step, and a rank's local
    buffer (its planes plus halo planes) stepped on its own planes equals the whole grid."""
    torch = torch_cuda()
    nz, ny, nx, r = 14, 20, 140, 2
    u0 = inputs.to_storage(inputs.gaussian_pulse_3d(nz, ny, nx, 3.0), "f32")
    cur = torch.from_numpy(u0).cuda()
    prev = torch.empty_like(cur)
    p = sy.stencil3d_params(nz, ny, nx, r, 0.125, "f32")
    for a, b in [(0, 5), (5, 6), (6, 14)]:
        sy.sy_stencil3d_step_planes(q, p, None, cur, prev, a, b, r, start=True)
    nxt = torch.empty_like(cur)
    for a, b in [(0, 7), (7, 14)]:
        sy.sy_stencil3d_step_planes(q, p, prev, cur, nxt, a, b, r)
    torch.cuda.synchronize()
    _, oc = oracle.wave3d_run_mirror(oracle.F32, u0, 1, r, 0.125)
    assert np.array_equal(nxt.cpu().numpy().view(np.uint32), oc.view(np.uint32))
    # a local buffer holding planes [4, 10) plus 2 halo planes each side: stepping its own planes
    lo, hi = 4 - r, 10 + r
    lp, lc = prev[lo:hi].contiguous(), cur[lo:hi].contiguous()
    ln = torch.empty_like(lc)
    pl = sy.stencil3d_params(hi - lo, ny, nx, r, 0.125, "f32")
    sy.sy_stencil3d_step_planes(q, pl, lp, lc, ln, r, r + 6, r)
    torch.cuda.synchronize()
    assert np.array_equal(ln[r: r + 6].cpu().numpy().view(np.uint32), oc[4:10].view(np.uint32))
    with pytest.raises(sy.SyError) as e:
        sy.sy_stencil3d_step_planes(q, p, prev, cur, nxt, 3, 15, r)
    assert e.value.name == "SY_ERR_BAD_CHUNKS"


_NO_OVERLAP = r"""
import sys
import numpy as np
import torch
sys.path[:0] = [sys.argv[1], sys.argv[2]]
import oracle
import paper_2505_06022_gb300 as sy
from paper_2505_06022_gb300 import inputs
ny, nx, r, h = 70, 260, 2, 2
chunks = sy.sy_split_rows(ny, 5)
u0 = inputs.to_storage(inputs.gaussian_pulse(ny, nx, 7.0), "f32")
cur, prev = [], []
for c, (a, b) in enumerate(chunks):
    lo, _, rows = sy.sy_split_layout(ny, chunks, h, c)
    t = torch.zeros(rows, nx, dtype=torch.float32, device="cuda")
    t[lo: lo + (b - a)] = torch.from_numpy(np.ascontiguousarray(u0[a:b])).cuda()
    cur.append(t)
    prev.append(torch.zeros_like(t))
p = sy.stencil_params(ny, nx, r, 0.25, "f32")
with sy.Queue(0) as q:
    sy.sy_stencil_start_split(q.handle, p, cur, prev, chunks, h)
    for _ in range(6):
        sy.sy_stencil_step_split(q.handle, p, prev, cur, prev, chunks, h)
        prev, cur = cur, prev
    torch.cuda.synchronize()
got = np.concatenate([cur[c][sy.sy_split_layout(ny, chunks, h, c)[0]:][: b - a].cpu().numpy()
                      for c, (a, b) in enumerate(chunks)])
_, want = oracle.wave_run_mirror(oracle.F32, u0, 6, r, 0.25)
assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
print("ok")
"""


def test_split_without_launch_overlap():
    """SY_PDL=0: the halo kernel and the chunk kernels run strictly one after another,
    with the same results (a fresh process: the switch is read once)."""
    import os
    import subprocess
    import sys

    torch_cuda()
    here = os.path.dirname(os.path.abspath(__file__))
    env = dict(os.environ, SY_PDL="0")
    out = subprocess.run([sys.executable, "-c", _NO_OVERLAP, os.path.dirname(here), here], env=env,
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0 and out.stdout.strip().endswith("ok"), out.stderr[-2000:]


def test_split_full_size_sampled(q):
    """The benchmark's split-buffer form at full size: 8192^2 FP32 with 0.01 noise on the
    Gaussian, 4 chunks in buffers of their own, halo 1, the Taylor start and 30 steps (one
    halo-exchange kernel and 4 chunk kernels a step); sampled points (corners, chunk
    boundaries on both sides, the centre) equal the precision mirror on the box of their
    light cone, bit for bit."""
    torch = torch_cuda()
    ny = nx = 8192
    steps, r, h = 30, 1, 1
    chunks = sy.sy_split_rows(ny, 4)
    u0 = inputs.to_storage(inputs.gaussian_pulse(ny, nx, 64.0) + 0.01 * inputs.random_field(5, ny, nx), "f32")
    cur = [to_local(u0, chunks, h, c, nx, torch.float32, torch) for c in range(len(chunks))]
    prev = [torch.zeros_like(t) for t in cur]
    p = sy.stencil_params(ny, nx, r, 0.25, "f32")
    sy.sy_stencil_start_split(q, p, cur, prev, chunks, h)
    for _ in range(steps):
        sy.sy_stencil_step_split(q, p, prev, cur, prev, chunks, h)
        prev, cur = cur, prev
    torch.cuda.synchronize()
    samples = [(0, 0), (0, 8191), (8191, 0), (8191, 8191), (2047, 4096), (2048, 4096), (2047, 0),
               (2048, 8191), (4095, 4100), (4096, 4100), (6143, 17), (6144, 17), (4096, 4096), (1000, 7000)]
    for (i, j) in samples:
        c = next(k for k, (a, b) in enumerate(chunks) if a <= i < b)
        lo, _, _ = sy.sy_split_layout(ny, chunks, h, c)
        got = cur[c][lo + i - chunks[c][0], j].item()
        y0, y1 = max(0, i - (steps + 1) * r - 1), min(ny, i + (steps + 1) * r + 2)
        x0, x1 = max(0, j - (steps + 1) * r - 1), min(nx, j + (steps + 1) * r + 2)
        _, m = oracle.wave_run_mirror(oracle.F32, np.ascontiguousarray(u0[y0:y1, x0:x1]), steps, r, 0.25)
        assert np.float32(got).view(np.uint32) == m[i - y0, j - x0].view(np.uint32), (i, j)
