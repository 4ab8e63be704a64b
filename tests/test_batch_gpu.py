"""Batched stencils (many uneven grids, one persistent launch per step, CUDA graph)
against the oracle and against stepping each grid with sy_stencil_step: bit-exact."""
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


def pitch_for(nx, dtype):
    v = 4 if dtype == "f32" else 8
    return (nx + v - 1) // v * v


def make_grids(shapes, dtype, seed=0):
    """shapes: list of (ny, nx, r).  Returns host initial fields and device (u_a, u_b) per grid."""
    torch = torch_cuda()
    host, dev = [], []
    for g, (ny, nx, r) in enumerate(shapes):
        u0 = inputs.to_storage(inputs.gaussian_pulse(ny, nx, max(1.5, min(ny, nx) / 16.0)) +
                               0.02 * inputs.random_field(seed + g, ny, nx), dtype)
        pitch = pitch_for(nx, dtype)
        tdt = torch.float32 if dtype == "f32" else torch.int16
        ub = torch.full((ny, pitch), -1, dtype=tdt, device="cuda")
        ub[:, :nx] = torch.from_numpy(u0 if dtype == "f32" else u0.view(np.int16)).cuda()
        ua = torch.full_like(ub, -1)
        host.append(u0)
        dev.append((ua, ub, pitch))
    return host, dev


def plan_for(q, shapes, dev, dtype, tile_rows=0, c2=0.25):
    return sy.sy_stencil_batch_plan(q, [(ny, nx, pitch, r, c2, ua, ub) for (ny, nx, r), (ua, ub, pitch)
                                        in zip(shapes, dev)], dtype, tile_rows)


def host_of(t, nx, dtype):
    a = t.cpu().numpy()[:, :nx]
    return np.ascontiguousarray(a if dtype == "f32" else a.view(np.uint16))


SMALL = [(8, 8, 1), (1, 1, 2), (37, 300, 4), (64, 129, 3), (5, 1030, 1), (130, 40, 2), (17, 17, 4), (300, 33, 1)]


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("tile_rows", [0, 2, 4, 8])
def test_batch_steps_bit_exact_vs_oracle(q, dtype, tile_rows):
    torch = torch_cuda()
    host, dev = make_grids(SMALL, dtype)
    plan = plan_for(q, SMALL, dev, dtype, tile_rows)
    try:
        tiles, points, blocks = sy.sy_stencil_batch_info(plan)
        assert points == sum(ny * nx for ny, nx, _ in SMALL) and blocks > 0 and tiles > 0
        sy.sy_stencil_batch_start(plan)
        steps = 7
        for s in range(steps):
            sy.sy_stencil_batch_step(plan, s & 1, timed=True)
        torch.cuda.synchronize()
        assert sy.sy_stencil_batch_times(plan, 1)[0] > 0
        for (ny, nx, r), u0, (ua, ub, _) in zip(SMALL, host, dev):
            op, oc = oracle.wave_run_mirror(DT[dtype], u0, steps, r, 0.25)
            newest, older = (ua, ub) if steps % 2 == 1 else (ub, ua)
            assert np.array_equal(bits(host_of(newest, nx, dtype)), bits(oc))
            assert np.array_equal(bits(host_of(older, nx, dtype)), bits(op))
            # padding untouched
            pad = (newest.cpu().numpy()[:, nx:])
            assert (pad.view(np.int32 if dtype == "f32" else np.int16) == (-1 if dtype != "f32" else
                                                                           np.float32(-1).view(np.int32))).all()
    finally:
        sy.sy_stencil_batch_destroy(plan)


def test_graph_run_equals_per_grid_steps(q):
    torch = torch_cuda()
    shapes = [(ny, nx, r) for ny, nx, r in inputs.batch_grids(count=12, seed=5, side_lo=64, side_hi=700)]
    host, dev = make_grids(shapes, "f32")
    plan = plan_for(q, shapes, dev, "f32", 4)
    try:
        sy.sy_stencil_batch_start(plan)
        steps = 10
        sy.sy_stencil_batch_capture(plan, steps)
        sy.sy_stencil_batch_run(plan)
        sy.sy_stencil_batch_run(plan)  # even count: the second replay continues the simulation
        torch.cuda.synchronize()
        ms = sy.sy_stencil_batch_times(plan, steps + 1)
        assert all(m > 0 for m in ms[1:])
        for (ny, nx, r), u0, (ua, ub, pitch) in zip(shapes, host, dev):
            # the same grid stepped alone through sy_stencil_step
            cur = torch.full_like(ub, -1.0)
            cur[:, :nx] = torch.from_numpy(u0).cuda()
            prev = torch.empty_like(cur)
            p = sy.stencil_params(ny, nx, r, 0.25, "f32", pitch=pitch)
            sy.sy_stencil_start(q, p, cur, prev, [(0, ny)], r)
            for _ in range(2 * steps):
                sy.sy_stencil_step(q, p, prev, cur, prev, [(0, ny)], r)
                prev, cur = cur, prev
            torch.cuda.synchronize()
            assert torch.equal(ub[:, :nx].contiguous().view(torch.int32), cur[:, :nx].contiguous().view(torch.int32))
            assert torch.equal(ua[:, :nx].contiguous().view(torch.int32), prev[:, :nx].contiguous().view(torch.int32))
    finally:
        sy.sy_stencil_batch_destroy(plan)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("steps", [7, 10])
def test_cross_step_form_bit_exact_vs_oracle(q, dtype, steps):
    """The whole run as one cooperative launch with a grid barrier between steps."""
    torch = torch_cuda()
    host, dev = make_grids(SMALL, dtype)
    plan = plan_for(q, SMALL, dev, dtype, 0)
    try:
        sy.sy_stencil_batch_start(plan)
        sy.sy_stencil_batch_capture_persistent(plan, steps)
        sy.sy_stencil_batch_run(plan)
        sy.sy_queue_sync(q)
        assert sy.sy_stencil_batch_times(plan, 2)[1] > 0
        for (ny, nx, r), u0, (ua, ub, _) in zip(SMALL, host, dev):
            op, oc = oracle.wave_run_mirror(DT[dtype], u0, steps, r, 0.25)
            newest, older = (ua, ub) if steps % 2 == 1 else (ub, ua)
            assert np.array_equal(bits(host_of(newest, nx, dtype)), bits(oc)), (ny, nx, r)
            assert np.array_equal(bits(host_of(older, nx, dtype)), bits(op)), (ny, nx, r)
    finally:
        sy.sy_stencil_batch_destroy(plan)
    torch.cuda.synchronize()


def test_cross_step_form_equals_class_launches_on_config2(q):
    """64 grids of the batched workload, 100 steps: every point of every grid identical
    between the per-class launches (one graph) and the one-launch form."""
    torch = torch_cuda()
    shapes = inputs.batch_grids()
    runs = []
    for persistent in (False, True):
        dev = []
        for ny, nx, r in shapes:
            pitch = pitch_for(nx, "f32")
            ub = torch.zeros((ny, pitch), dtype=torch.float32, device="cuda")
            ub[:, :nx] = torch.from_numpy(inputs.batch_initial(ny, nx, "f32")).cuda()
            dev.append((torch.empty_like(ub), ub, pitch))
        plan = plan_for(q, shapes, dev, "f32", 0)
        try:
            sy.sy_stencil_batch_start(plan)
            (sy.sy_stencil_batch_capture_persistent if persistent else sy.sy_stencil_batch_capture)(plan, 100)
            sy.sy_stencil_batch_run(plan)
            sy.sy_queue_sync(q)
        finally:
            sy.sy_stencil_batch_destroy(plan)
        runs.append(dev)
    for (ny, nx, _), (a0, b0, _), (a1, b1, _) in zip(shapes, *runs):  # the fields, not their row padding
        assert torch.equal(a0[:, :nx].contiguous().view(torch.int32), a1[:, :nx].contiguous().view(torch.int32))
        assert torch.equal(b0[:, :nx].contiguous().view(torch.int32), b1[:, :nx].contiguous().view(torch.int32))


def test_cross_step_barrier_wait_is_bounded_and_context_survives(q):
    """Host-injected fault: block 0 never arrives at the first step barrier.  Every other
    block's wait gives up after about a second, the run reports SY_ERR_TIMEOUT once, and the
    next capture on the same queue runs correctly."""
    import os

    torch = torch_cuda()
    host, dev = make_grids(SMALL, "f32")
    old = os.environ.get("SY_FAULT")
    os.environ["SY_FAULT"] = "batch_barrier_timeout"
    try:
        plan = plan_for(q, SMALL, dev, "f32", 0)
        sy.sy_stencil_batch_start(plan)
        sy.sy_stencil_batch_capture_persistent(plan, 4)
    finally:
        if old is None:
            del os.environ["SY_FAULT"]
        else:
            os.environ["SY_FAULT"] = old
    try:
        sy.sy_stencil_batch_run(plan)
        with pytest.raises(sy.SyError) as e:
            sy.sy_queue_sync(q)
        assert e.value.name == "SY_ERR_TIMEOUT"
        sy.sy_queue_sync(q)  # reported once, then cleared
    finally:
        sy.sy_stencil_batch_destroy(plan)
    host, dev = make_grids(SMALL, "f32")
    plan = plan_for(q, SMALL, dev, "f32", 0)
    try:
        sy.sy_stencil_batch_start(plan)
        sy.sy_stencil_batch_capture_persistent(plan, 4)
        sy.sy_stencil_batch_run(plan)
        sy.sy_queue_sync(q)
        for (ny, nx, r), u0, (ua, ub, _) in zip(SMALL, host, dev):
            _, oc = oracle.wave_run_mirror(oracle.F32, u0, 4, r, 0.25)
            assert np.array_equal(bits(host_of(ub, nx, "f32")), bits(oc))
    finally:
        sy.sy_stencil_batch_destroy(plan)
    torch.cuda.synchronize()


@pytest.mark.parametrize("tile_rows", [0, 4], ids=["classes", "rows4"])
def test_config2_full_batch_sampled(q, tile_rows):
    """64 grids, sides log-uniform in [256, 4096] (seed 1), radius from {1, 2, 4}, 100 steps in one
    graph, as per-radius-class launches (the timed configuration) and as one launch per step with
    4-row tiles; sampled points of the largest and smallest grids against the oracle (light cone)."""
    torch = torch_cuda()
    shapes = inputs.batch_grids()
    host, dev = [], []
    for g, (ny, nx, r) in enumerate(shapes):
        u0 = inputs.batch_initial(ny, nx, "f32")
        pitch = pitch_for(nx, "f32")
        ub = torch.zeros((ny, pitch), dtype=torch.float32, device="cuda")
        ub[:, :nx] = torch.from_numpy(u0).cuda()
        host.append(u0)
        dev.append((torch.empty_like(ub), ub, pitch))
    plan = plan_for(q, shapes, dev, "f32", tile_rows)
    try:
        sy.sy_stencil_batch_start(plan)
        sy.sy_stencil_batch_capture(plan, 100)
        sy.sy_stencil_batch_run(plan)
        torch.cuda.synchronize()
        areas = [ny * nx for ny, nx, _ in shapes]
        for g in (int(np.argmin(areas)), int(np.argmax(areas)), 7):
            ny, nx, r = shapes[g]
            newest = dev[g][1][:, :nx].cpu().numpy()  # even step count: u_b holds u^100
            h = (100 + 1) * r + 1
            for (pi, pj) in [(0, 0), (ny // 2, nx // 2), (ny - 1, nx - 1), (ny // 3, nx - 2)]:
                y0, y1, x0, x1 = max(0, pi - h), min(ny, pi + h + 1), max(0, pj - h), min(nx, pj + h + 1)
                _, oc = oracle.wave_run_mirror(oracle.F32, np.ascontiguousarray(host[g][y0:y1, x0:x1]), 100, r, 0.25)
                assert newest[pi, pj].view(np.uint32) == oc[pi - y0, pj - x0].view(np.uint32), (g, pi, pj)
    finally:
        sy.sy_stencil_batch_destroy(plan)


@pytest.mark.parametrize("tile_rows", [0, 4])
def test_max_grids_per_plan(q, tile_rows):
    """4096 grids in one plan (the most a plan takes; a work-list entry holds the grid index in
    12 bits), sides from 1 to 300, every radius: two steps bit-exact against the oracle; a
    4097th grid is refused."""
    torch = torch_cuda()
    z = inputs.splitmix64(31, 3 * 4096)
    shapes = [(1 + int(z[3 * g] % np.uint64(40)), 1 + int(z[3 * g + 1] % np.uint64(300)),
               1 + int(z[3 * g + 2] % np.uint64(4))) for g in range(4096)]
    host, dev = [], []
    for g, (ny, nx, r) in enumerate(shapes):
        u0 = inputs.random_field(5000 + g, ny, nx)
        pitch = pitch_for(nx, "f32")
        ub = torch.zeros((ny, pitch), dtype=torch.float32, device="cuda")
        ub[:, :nx] = torch.from_numpy(u0).cuda()
        host.append(u0)
        dev.append((torch.zeros_like(ub), ub, pitch))
    plan = plan_for(q, shapes, dev, "f32", tile_rows)
    try:
        sy.sy_stencil_batch_start(plan)
        sy.sy_stencil_batch_step(plan, 0)
        sy.sy_stencil_batch_step(plan, 1)
        torch.cuda.synchronize()
    finally:
        sy.sy_stencil_batch_destroy(plan)
    for (ny, nx, r), (ua, ub, pitch), u0 in zip(shapes, dev, host):
        _, want = oracle.wave_run_mirror(oracle.F32, u0, 2, r, 0.25)
        assert np.array_equal(bits(host_of(ub, nx, "f32")), bits(want)), (ny, nx, r)
    extra = torch.zeros((1, 4), device="cuda"), torch.zeros((1, 4), device="cuda")
    with pytest.raises(sy.SyError) as e:
        sy.sy_stencil_batch_plan(q, [(ny, nx, pitch, r, 0.25, ua, ub) for (ny, nx, r), (ua, ub, pitch)
                                     in zip(shapes, dev)] + [(1, 1, 4, 1, 0.25, extra[0], extra[1])], "f32", tile_rows)
    assert e.value.name == "SY_ERR_INVALID_ARGUMENT"


def test_batch_errors(q):
    torch = torch_cuda()
    a = torch.zeros(16, 64, device="cuda")
    b = torch.zeros(16, 64, device="cuda")
    with pytest.raises(sy.SyError) as e:
        sy.sy_stencil_batch_plan(q, [(16, 64, 64, 1, 0.25, a, a)])
    assert e.value.name == "SY_ERR_ALIAS"
    with pytest.raises(sy.SyError) as e:
        sy.sy_stencil_batch_plan(q, [(16, 63, 63, 1, 0.25, a, b)])  # 252-byte pitch: not 16-aligned
    assert e.value.name == "SY_ERR_INVALID_ARGUMENT"
    with pytest.raises(sy.SyError) as e:
        sy.sy_stencil_batch_plan(q, [(16, 64, 64, 5, 0.25, a, b)])
    assert e.value.name == "SY_ERR_INVALID_ARGUMENT"
    with pytest.raises(sy.SyError) as e:
        sy.sy_stencil_batch_plan(q, [(16, 64, 64, 1, 0.25, a, b), (8, 64, 64, 1, 0.25, a.view(-1)[512:], b)])
    assert e.value.name == "SY_ERR_ALIAS"
    with pytest.raises(sy.SyError) as e:
        sy.sy_stencil_batch_plan(q, [])
    assert e.value.name == "SY_ERR_INVALID_ARGUMENT"
    plan = sy.sy_stencil_batch_plan(q, [(16, 64, 64, 1, 0.25, a, b)])
    with pytest.raises(sy.SyError) as e:
        sy.sy_stencil_batch_run(plan)  # nothing captured yet
    assert e.value.name == "SY_ERR_INVALID_ARGUMENT"
    sy.sy_stencil_batch_destroy(plan)
