"""Memory-safety checks without a sanitizer: every field lives inside a larger
buffer whose row padding and surrounding guard bands hold NaN bit patterns.  A
kernel that read a padding or guard value into a result would not reproduce the
oracle bit for bit, and one that wrote outside the field would change a guard
byte; both are checked after each run, for every kernel family."""
import numpy as np
import pytest

import oracle
import paper_2505_06022_gb300 as sy
from paper_2505_06022_gb300 import inputs

from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu

GUARD = 2048  # elements before and after each field (8 KiB of FP32)
DT = {"f32": oracle.F32, "bf16": oracle.BF16, "f16": oracle.F16}


@pytest.fixture(scope="module")
def q():
    torch_cuda()
    with sy.Queue(0) as queue:
        yield queue.handle


class Guarded:
    """A (rows x pitch) field at offset GUARD of a flat buffer; everything that is not a
    field element (row padding, guard bands) holds a NaN pattern."""

    def __init__(self, rows, cols, pitch, dtype, torch, values=None):
        self.rows, self.cols, self.pitch, self.dtype = rows, cols, pitch, dtype
        self.tdt = torch.float32 if dtype == "f32" else torch.int16
        nan = np.array([0x7FC00001], np.uint32).view(np.int32)[0] if dtype == "f32" else np.int16(0x7E01)
        total = GUARD + rows * pitch + GUARD
        host = np.full(total, nan, np.int32 if dtype == "f32" else np.int16)
        if values is not None:
            v = values.view(np.int32 if dtype == "f32" else np.int16)
            body = host[GUARD: GUARD + rows * pitch].reshape(rows, pitch)
            body[:, :cols] = v.reshape(rows, cols)
        self.initial = host.copy()
        self.buf = torch.from_numpy(host.view(np.float32) if dtype == "f32" else host).cuda()
        self.field = self.buf[GUARD: GUARD + rows * pitch]

    def values(self):
        h = self.buf.cpu().numpy()
        body = h[GUARD: GUARD + self.rows * self.pitch].reshape(self.rows, self.pitch)[:, : self.cols]
        return np.ascontiguousarray(body).view(np.float32 if self.dtype == "f32" else np.uint16)

    def guards_intact(self):
        h = self.buf.cpu().numpy().view(self.initial.dtype)
        body = h[GUARD: GUARD + self.rows * self.pitch].reshape(self.rows, self.pitch)
        init = self.initial[GUARD: GUARD + self.rows * self.pitch].reshape(self.rows, self.pitch)
        return (np.array_equal(h[:GUARD], self.initial[:GUARD]) and np.array_equal(h[-GUARD:], self.initial[-GUARD:])
                and np.array_equal(body[:, self.cols:], init[:, self.cols:]))


def bits(a):
    return a.view(np.uint32) if a.dtype == np.float32 else a


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("r", [1, 2, 4])
@pytest.mark.parametrize("variant", [0, 9, 13])  # default tiles, halo-lane tiles, narrow (16-bit; FP32: 0)
def test_2d_step_reads_and_writes_only_the_field(q, dtype, r, variant):
    torch = torch_cuda()
    ny, nx = 37, 301
    v = 4 if dtype == "f32" else 8
    pitch = (nx + v - 1) // v * v + 2 * v
    u0 = inputs.to_storage(inputs.gaussian_pulse(ny, nx, 6.0) + 0.05 * inputs.random_field(5, ny, nx), dtype)
    cur = Guarded(ny, nx, pitch, dtype, torch, u0)
    prev = Guarded(ny, nx, pitch, dtype, torch)
    p = sy.stencil_params(ny, nx, r, 0.25, dtype, pitch=pitch, variant=variant if (dtype != "f32" or variant < 13)
                          else 0)
    chunks = [(0, 5), (5, 6), (6, 30), (30, 37)]
    sy.sy_stencil_start(q, p, cur.field, prev.field, chunks, r)
    for _ in range(4):
        sy.sy_stencil_step(q, p, prev.field, cur.field, prev.field, chunks, r)
        prev, cur = cur, prev
    torch.cuda.synchronize()
    _, want = oracle.wave_run_mirror(DT[dtype], u0, 4, r, 0.25)
    assert np.array_equal(bits(cur.values()), bits(want))
    assert cur.guards_intact() and prev.guards_intact()


@pytest.mark.parametrize("variant", list(range(0, 11)))
def test_3d_every_variant_reads_and_writes_only_the_field(q, variant):
    torch = torch_cuda()
    nz, ny, nx, r = 7, 19, 150, 2
    pitch, planes = 160, 19 * 160 + 8
    u0 = inputs.to_storage(inputs.gaussian_pulse_3d(nz, ny, nx, 3.0) + 0.05 * inputs.random_field_3d(6, nz, ny, nx),
                           "f32")
    # a 3D field as nz planes of `planes` elements, the rows of a plane at `pitch`; NaN elsewhere
    nanpat = np.array([0x7FC00001], np.uint32).view(np.float32)[0]
    filled = np.full((nz, planes), nanpat, np.float32)
    filled[:, : ny * pitch].reshape(nz, ny, pitch)[:, :, :nx] = u0
    cur = Guarded(nz, planes, planes, "f32", torch, filled.reshape(nz, planes))
    prev = Guarded(nz, planes, planes, "f32", torch, np.full((nz, planes), nanpat, np.float32))
    p = sy.stencil3d_params(nz, ny, nx, r, 0.125, "f32", pitch=pitch, plane=planes, variant=variant)
    chunks = [(0, 3), (3, 7)]
    sy.sy_stencil3d_start(q, p, cur.field, prev.field, chunks, r)
    for _ in range(3):
        sy.sy_stencil3d_step(q, p, prev.field, cur.field, prev.field, chunks, r)
        prev, cur = cur, prev
    torch.cuda.synchronize()
    _, want = oracle.wave3d_run_mirror(oracle.F32, u0, 3, r, 0.125)
    got = cur.buf.cpu().numpy()[GUARD: GUARD + nz * planes].reshape(nz, planes)
    got = np.ascontiguousarray(got[:, : ny * pitch].reshape(nz, ny, pitch)[:, :, :nx])
    assert np.array_equal(bits(got), bits(want))
    for g in (cur, prev):  # guard bands, and every non-field element of a plane, untouched where no step writes
        h = g.buf.cpu().numpy().view(np.int32)
        assert np.array_equal(h[:GUARD], g.initial[:GUARD].view(np.int32))
        assert np.array_equal(h[-GUARD:], g.initial[-GUARD:].view(np.int32))
        body = h[GUARD: GUARD + nz * planes].reshape(nz, planes)
        init = g.initial[GUARD: GUARD + nz * planes].view(np.int32).reshape(nz, planes)
        assert np.array_equal(body[:, ny * pitch:], init[:, ny * pitch:])
        rows = body[:, : ny * pitch].reshape(nz, ny, pitch)
        rows0 = init[:, : ny * pitch].reshape(nz, ny, pitch)
        assert np.array_equal(rows[:, :, nx:], rows0[:, :, nx:])


@pytest.mark.parametrize("T,r", [(2, 1), (4, 1), (2, 2)])
def test_temporal_blocking_reads_and_writes_only_the_field(q, T, r):
    torch = torch_cuda()
    ny, nx = 70, 300
    pitch = 312
    u0 = inputs.to_storage(inputs.gaussian_pulse(ny, nx, 7.0), "f32")
    b = Guarded(ny, nx, pitch, "f32", torch, u0)
    a, c, d = (Guarded(ny, nx, pitch, "f32", torch) for _ in range(3))
    p = sy.stencil_params(ny, nx, r, 0.25, "f32", pitch=pitch)
    chunks = sy.sy_split_rows(ny, 3)
    sy.sy_stencil_start(q, p, b.field, a.field, chunks, T * r)
    sy.sy_stencil_multistep(q, p, T, a.field, b.field, c.field, d.field, chunks, T * r)
    torch.cuda.synchronize()
    _, want = oracle.wave_run_mirror(oracle.F32, u0, T, r, 0.25)
    assert np.array_equal(bits(d.values()), bits(want))
    assert all(g.guards_intact() for g in (a, b, c, d))


def test_batched_reads_and_writes_only_the_fields(q):
    torch = torch_cuda()
    shapes = [(33, 130, 1), (9, 61, 2), (70, 257, 4), (5, 5, 1)]
    fields, host = [], []
    for k, (ny, nx, r) in enumerate(shapes):
        pitch = (nx + 3) // 4 * 4 + 4
        u0 = inputs.to_storage(inputs.gaussian_pulse(ny, nx, 4.0) + 0.05 * inputs.random_field(20 + k, ny, nx), "f32")
        ub = Guarded(ny, nx, pitch, "f32", torch, u0)
        ua = Guarded(ny, nx, pitch, "f32", torch)
        fields.append((ny, nx, pitch, r, ua, ub))
        host.append(u0)
    for tile_rows in (0, 4):
        plan = sy.sy_stencil_batch_plan(q, [(ny, nx, pitch, r, 0.25, ua.field, ub.field)
                                            for ny, nx, pitch, r, ua, ub in fields], "f32", tile_rows)
        try:
            sy.sy_stencil_batch_start(plan)
            sy.sy_stencil_batch_step(plan, 0)
            sy.sy_stencil_batch_step(plan, 1)
            torch.cuda.synchronize()
        finally:
            sy.sy_stencil_batch_destroy(plan)
        for (ny, nx, pitch, r, ua, ub), u0 in zip(fields, host):
            _, want = oracle.wave_run_mirror(oracle.F32, u0, 2, r, 0.25)
            assert np.array_equal(bits(ub.values()), bits(want))
            assert ua.guards_intact() and ub.guards_intact()
        for (ny, nx, pitch, r, ua, ub), u0 in zip(fields, host):  # fresh u0 for the next plan
            ub.buf.copy_(torch.from_numpy(ub.initial.view(np.float32)).cuda())


def test_saxpy_reads_and_writes_only_its_range(q):
    torch = torch_cuda()
    for n in (1, 3, 4097, 100003):
        x, y = inputs.saxpy_inputs(n, seed=3)
        gx, gy = Guarded(1, n, n, "f32", torch, x), Guarded(1, n, n, "f32", torch, y)
        gz = Guarded(1, n, n, "f32", torch)
        sy.sy_saxpy(q, n, 2.5, gx.field, gy.field, gz.field)
        torch.cuda.synchronize()
        assert np.array_equal(bits(gz.values()), bits(oracle.saxpy_f32(2.5, x, y).reshape(1, n)))
        assert gx.guards_intact() and gy.guards_intact() and gz.guards_intact()
