"""Non-finite values in a field spread as IEEE arithmetic says: after a few steps the
kernels and the oracle's precision mirror agree bit for bit on every finite point and
on the class (NaN, +inf, -inf) of every other point.  NaN payloads are not compared
(IEEE leaves them to the implementation).  A kernel that masked lanes by multiplying
with zero, or reordered an addition, would change where NaN and infinity appear."""
import numpy as np
import pytest

import oracle
import paper_2505_06022_gb300 as sy
from paper_2505_06022_gb300 import inputs

from gpu_helpers import torch_cuda, wave_run

pytestmark = pytest.mark.gpu

DT = {"f32": oracle.F32, "bf16": oracle.BF16, "f16": oracle.F16}
# storage bit patterns of +inf, -inf and a quiet NaN
SPECIAL = {"f32": (0x7F800000, 0xFF800000, 0x7FC00000), "bf16": (0x7F80, 0xFF80, 0x7FC0),
           "f16": (0x7C00, 0xFC00, 0x7E00)}


@pytest.fixture(scope="module")
def q():
    torch_cuda()
    with sy.Queue(0) as queue:
        yield queue.handle


def plant(u, dtype, points):
    """Copy of storage array u with +inf, -inf, NaN written at the given flat indices."""
    u = u.copy()
    raw = u.view(np.uint32 if dtype == "f32" else np.uint16).reshape(-1)
    for idx, pattern in zip(points, SPECIAL[dtype]):
        raw[idx] = pattern
    return u


def same_ieee(got, want, dtype):
    g = oracle.storage_to_f64(got, DT[dtype]) if dtype != "f32" else got.astype(np.float64)
    w = oracle.storage_to_f64(want, DT[dtype]) if dtype != "f32" else want.astype(np.float64)
    for cls in (np.isnan, np.isposinf, np.isneginf):
        assert np.array_equal(cls(g), cls(w))
    fin = np.isfinite(w)
    assert np.count_nonzero(~fin) > 0 and np.count_nonzero(fin) > 0
    gb = got.view(np.uint32 if dtype == "f32" else np.uint16)
    wb = want.view(np.uint32 if dtype == "f32" else np.uint16)
    assert np.array_equal(gb[fin], wb[fin])


@pytest.mark.parametrize("dtype,r", [("f32", 1), ("f32", 2), ("bf16", 1), ("f16", 1), ("f16", 4)])
def test_2d_nonfinite_values_spread_as_in_the_oracle(q, dtype, r):
    ny, nx = 40, 260
    u0 = inputs.to_storage(inputs.gaussian_pulse(ny, nx, 6.0) + 0.05 * inputs.random_field(3, ny, nx), dtype)
    # +inf inside a chunk, -inf on a chunk boundary row, NaN at the right edge of a warp span
    u0 = plant(u0, dtype, [12 * nx + 40, 20 * nx + 200, 30 * nx + 127])
    gp, gc = wave_run(q, u0, 3, r, 0.25, dtype, [(0, 20), (20, 33), (33, ny)])
    op, oc = oracle.wave_run_mirror(DT[dtype], u0, 3, r, 0.25)
    same_ieee(gc, oc, dtype)
    same_ieee(gp, op, dtype)


def test_3d_nonfinite_values_spread_as_in_the_oracle(q):
    torch = torch_cuda()
    shape = (10, 20, 140)
    u0 = inputs.to_storage(inputs.gaussian_pulse_3d(*shape, 3.0) + 0.05 * inputs.random_field_3d(4, *shape), "f32")
    nz, ny, nx = shape
    u0 = plant(u0, "f32", [(4 * ny + 10) * nx + 60, (5 * ny + 3) * nx + 127, (9 * ny + 19) * nx + 139])
    d0 = torch.from_numpy(u0).cuda().reshape(-1)
    a, b = torch.empty_like(d0), torch.empty_like(d0)
    p = sy.stencil3d_params(*shape, 1, 0.125, "f32")
    _, cv, _ = sy.sy_wave3d_run(q, p, d0, a, b, 2, [(0, 5), (5, 10)], 1)
    torch.cuda.synchronize()
    got = {d0.data_ptr(): d0, a.data_ptr(): a, b.data_ptr(): b}[cv].cpu().numpy().reshape(shape)
    _, want = oracle.wave3d_run_mirror(oracle.F32, u0, 2, 1, 0.125)
    same_ieee(got, want, "f32")


def test_saxpy_nonfinite_operands(q):
    torch = torch_cuda()
    n = 1031
    x, y = inputs.saxpy_inputs(n, seed=14)
    x, y = x.copy(), y.copy()
    x[[0, 5, 600]] = [np.inf, -np.inf, np.nan]
    y[[5, 9, 1030]] = [np.inf, np.nan, -np.inf]  # -inf + inf at 5
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    zd = torch.empty_like(xd)
    sy.sy_saxpy(q, n, 2.5, xd, yd, zd)
    torch.cuda.synchronize()
    same_ieee(zd.cpu().numpy(), oracle.saxpy_f32(2.5, x, y), "f32")
