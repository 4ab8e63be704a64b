"""Values in the subnormal ranges of FP32, BF16 and FP16: the kernels must not flush
them to zero (no fast-math, no flush-to-zero anywhere on the path), so every kernel
family reproduces the oracle's precision mirror bit for bit on fields and operands
scaled far below the smallest normal number."""
import numpy as np
import pytest

import oracle
import paper_2505_06022_gb300 as sy
from paper_2505_06022_gb300 import inputs

from gpu_helpers import bits, to_host, torch_cuda, wave_run

pytestmark = pytest.mark.gpu

DT = {"f32": oracle.F32, "bf16": oracle.BF16, "f16": oracle.F16}
# Scales that put a [-1, 1) field wholly below the storage type's smallest normal:
# FP32 2^-126, BF16 2^-126 (same exponent range), FP16 2^-14.
SCALE = {"f32": 2.0 ** -134, "bf16": 2.0 ** -129, "f16": 2.0 ** -17}
TINY = {"f32": 2.0 ** -126, "bf16": 2.0 ** -126, "f16": 2.0 ** -14}


@pytest.fixture(scope="module")
def q():
    torch_cuda()
    with sy.Queue(0) as queue:
        yield queue.handle


def subnormal_field(seed, shape, dtype):
    u = inputs.to_storage(inputs.random_field(seed, *shape).astype(np.float64) * SCALE[dtype], dtype)
    vals = np.abs(oracle.storage_to_f64(u, DT[dtype]) if dtype != "f32" else u.astype(np.float64))
    assert np.count_nonzero((vals > 0) & (vals < TINY[dtype])) > 0.9 * vals.size  # nearly all subnormal
    return u


def test_saxpy_subnormal_operands(q):
    torch = torch_cuda()
    n = 4099
    x, y = inputs.saxpy_inputs(n, seed=12)
    x = (x.astype(np.float64) * 2.0 ** -130).astype(np.float32)
    y = (y.astype(np.float64) * 2.0 ** -128).astype(np.float32)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    zd = torch.empty_like(xd)
    sy.sy_saxpy(q, n, 2.5, xd, yd, zd)
    torch.cuda.synchronize()
    want = oracle.saxpy_f32(2.5, x, y)
    assert np.count_nonzero(np.abs(want) < 2.0 ** -126) > 0.9 * n
    assert np.array_equal(zd.cpu().numpy().view(np.uint32), want.view(np.uint32))


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("r", [1, 2, 4])
def test_wave_steps_on_a_subnormal_field(q, dtype, r):
    ny, nx = 50, 300
    u0 = subnormal_field(7, (ny, nx), dtype)
    gp, gc = wave_run(q, u0, 4, r, 0.25, dtype, sy.sy_split_rows(ny, 3))
    op, oc = oracle.wave_run_mirror(DT[dtype], u0, 4, r, 0.25)
    assert np.any(bits(oc) != 0)
    assert np.array_equal(bits(gc), bits(oc)) and np.array_equal(bits(gp), bits(op))


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_temporal_blocking_on_a_subnormal_field(q, dtype):
    torch = torch_cuda()
    ny, nx, T, r = 70, 304, 2, 1
    u0 = subnormal_field(8, (ny, nx), dtype)
    chunks = sy.sy_split_rows(ny, 3)
    tdt = torch.float32 if dtype == "f32" else torch.int16
    B = torch.from_numpy(u0 if dtype == "f32" else u0.view(np.int16)).cuda()
    A, C, D = (torch.zeros(ny, nx, dtype=tdt, device="cuda") for _ in range(3))
    p = sy.stencil_params(ny, nx, r, 0.25, dtype)
    sy.sy_stencil_start(q, p, B, A, chunks, T * r)
    sy.sy_stencil_multistep(q, p, T, A, B, C, D, chunks, T * r)
    sy.sy_queue_sync(q)
    st = np.float32 if dtype == "f32" else np.uint16
    op, oc = oracle.wave_run_mirror(DT[dtype], u0, T, r, 0.25)
    assert np.array_equal(bits(to_host(D, (ny, nx), st)), bits(oc))
    assert np.array_equal(bits(to_host(C, (ny, nx), st)), bits(op))


@pytest.mark.parametrize("dtype,variant", [("f32", 0), ("bf16", 0), ("f32", 9)])
def test_3d_steps_on_a_subnormal_field(q, dtype, variant):
    torch = torch_cuda()
    shape = (9, 21, 140)
    u0 = inputs.to_storage(inputs.random_field_3d(9, *shape).astype(np.float64) * SCALE[dtype], dtype)
    d0 = torch.from_numpy(u0 if dtype == "f32" else u0.view(np.int16)).cuda().reshape(-1)
    a, b = torch.empty_like(d0), torch.empty_like(d0)
    p = sy.stencil3d_params(*shape, 2, 0.125, dtype, variant=variant)
    pv, cv, _ = sy.sy_wave3d_run(q, p, d0, a, b, 3, [(0, 4), (4, 9)], 2)
    torch.cuda.synchronize()
    byptr = {d0.data_ptr(): d0, a.data_ptr(): a, b.data_ptr(): b}
    st = np.float32 if dtype == "f32" else np.uint16
    op, oc = oracle.wave3d_run_mirror(DT[dtype], u0, 3, 2, 0.125)
    got = byptr[cv].cpu().numpy().view(st).reshape(shape)
    assert np.any(bits(oc) != 0)
    assert np.array_equal(bits(got), bits(oc))
