"""The 3D leapfrog step on the GPU, chunked along planes: bit-identical to the
oracle's precision mirror for every storage type, radius and tile variant, on
grids that span several tiles with ragged edges in every dimension, with padded
row and plane strides, on the unaligned (one point per thread) path, through the
captured whole-run graph, and -- at the full 512^3 workload in the launch
configuration the benchmark times -- at sampled points against the oracle on
their light cones."""
import numpy as np
import pytest

import oracle
import paper_2505_06022_gb300 as sy
from paper_2505_06022_gb300 import inputs

from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu

DT = {"f32": oracle.F32, "bf16": oracle.BF16, "f16": oracle.F16}
C2 = 0.125


@pytest.fixture(scope="module")
def q():
    torch_cuda()
    with sy.Queue(0) as queue:
        yield queue.handle


def field(shape, dtype, seed=3, sigma=3.0):
    return inputs.to_storage(inputs.gaussian_pulse_3d(*shape, sigma) + 0.05 * inputs.random_field_3d(seed, *shape),
                             dtype)


def upload(u, pitch, plane, torch):
    """(nz, ny, nx) storage array -> flat device buffer with the given row and plane strides."""
    nz, ny, nx = u.shape
    tdt = torch.float32 if u.dtype == np.float32 else torch.int16
    host = torch.from_numpy(u if u.dtype == np.float32 else u.view(np.int16))
    buf = torch.zeros(nz * plane, dtype=tdt)
    view = buf.as_strided((nz, ny, nx), (plane, pitch, 1))
    view.copy_(host)
    return buf.cuda()


def download(buf, shape, pitch, plane, storage):
    nz, ny, nx = shape
    a = buf.cpu().as_strided((nz, ny, nx), (plane, pitch, 1)).contiguous().numpy()
    return a.view(np.uint16) if storage != np.float32 else a


def run3d(q, u0, steps, r, dtype, chunks, variant=0, pitch=None, plane=None, halo=None, offset=0):
    torch = torch_cuda()
    nz, ny, nx = u0.shape
    pitch = pitch or nx
    plane = plane or ny * pitch
    cur = upload(u0, pitch, plane, torch)
    if offset:  # shift the field by `offset` elements inside a larger buffer (unaligned layouts)
        big = torch.zeros(cur.numel() + offset, dtype=cur.dtype, device="cuda")
        big[offset:] = cur
        cur = big[offset:]
    prev = torch.zeros_like(cur)
    p = sy.stencil3d_params(nz, ny, nx, r, C2, dtype, pitch=pitch, plane=plane, variant=variant)
    halo = r if halo is None else halo
    sy.sy_stencil3d_start(q, p, cur, prev, chunks, halo)
    for _ in range(steps):
        sy.sy_stencil3d_step(q, p, prev, cur, prev, chunks, halo)
        prev, cur = cur, prev
    torch.cuda.synchronize()
    st = np.float32 if dtype == "f32" else np.uint16
    return download(prev, u0.shape, pitch, plane, st), download(cur, u0.shape, pitch, plane, st)


def bits(a):
    return a.view(np.uint32) if a.dtype == np.float32 else a


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_3d_bit_exact_vs_oracle(q, dtype, r):
    shape = (13, 37, 300)  # ragged in y (tile rows) and x (warp spans of 128 / 256 columns)
    u0 = field(shape, dtype)
    chunks = [(0, 2), (2, 3), (3, 10), (10, 13)]  # includes chunks thinner than the radius
    p, c = run3d(q, u0, 5, r, dtype, chunks)
    op, oc = oracle.wave3d_run_mirror(DT[dtype], u0, 5, r, C2)
    assert np.array_equal(bits(c), bits(oc)) and np.array_equal(bits(p), bits(op))


@pytest.mark.parametrize("r", [1, 2, 3, 4])
@pytest.mark.parametrize("variant", range(0, 11))
def test_3d_every_variant(q, r, variant):
    shape = (20, 45, 260)
    u0 = field(shape, "f32", seed=4)
    p, c = run3d(q, u0, 3, r, "f32", sy.sy_split_rows(20, 3), variant=variant)
    op, oc = oracle.wave3d_run_mirror(oracle.F32, u0, 3, r, C2)
    assert np.array_equal(bits(c), bits(oc)) and np.array_equal(bits(p), bits(op))


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_3d_padded_strides(q, dtype):
    shape = (9, 21, 70)
    u0 = field(shape, dtype, seed=5)
    v = 4 if dtype == "f32" else 8
    pitch = (70 + v - 1) // v * v + v  # padded rows
    plane = 21 * pitch + 3 * v         # padded planes
    p, c = run3d(q, u0, 4, 2, dtype, [(0, 4), (4, 9)], pitch=pitch, plane=plane)
    op, oc = oracle.wave3d_run_mirror(DT[dtype], u0, 4, 2, C2)
    assert np.array_equal(bits(c), bits(oc)) and np.array_equal(bits(p), bits(op))


def test_3d_unaligned_layout_takes_the_scalar_path(q):
    shape = (6, 11, 19)
    u0 = field(shape, "f32", seed=6)
    p, c = run3d(q, u0, 3, 1, "f32", [(0, 3), (3, 6)], offset=1)  # rows not 16-byte aligned
    op, oc = oracle.wave3d_run_mirror(oracle.F32, u0, 3, 1, C2)
    assert np.array_equal(bits(c), bits(oc)) and np.array_equal(bits(p), bits(op))


@pytest.mark.parametrize("variant", [7, 8, 9, 10])
@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_3d_slab_variants_16bit_ragged(q, variant, dtype):
    # strips of 8 / 16 rows over a grid whose rows are not a multiple of either, 16-bit storage
    shape = (9, 53, 300)
    u0 = field(shape, dtype, seed=12)
    p, c = run3d(q, u0, 4, 2, dtype, [(0, 4), (4, 9)], variant=variant)
    op, oc = oracle.wave3d_run_mirror(DT[dtype], u0, 4, 2, C2)
    assert np.array_equal(bits(c), bits(oc)) and np.array_equal(bits(p), bits(op))


@pytest.mark.parametrize("c2", [0.0, 0.07, 0.33])
@pytest.mark.parametrize("dtype,r", [("f32", 1), ("bf16", 2)])
def test_3d_any_c2_bit_exact(q, c2, dtype, r):
    shape = (11, 23, 150)
    u0 = field(shape, dtype, seed=14)
    nz = shape[0]
    p = sy.stencil3d_params(*shape, r, c2, dtype)
    torch = torch_cuda()
    d0 = torch.from_numpy(u0 if dtype == "f32" else u0.view(np.int16)).cuda().reshape(-1)
    a, b = torch.empty_like(d0), torch.empty_like(d0)
    pv, cv, _ = sy.sy_wave3d_run(q, p, d0, a, b, 4, sy.sy_split_rows(nz, 3), r)
    torch.cuda.synchronize()
    byptr = {d0.data_ptr(): d0, a.data_ptr(): a, b.data_ptr(): b}
    st = np.float32 if dtype == "f32" else np.uint16
    op, oc = oracle.wave3d_run_mirror(DT[dtype], u0, 4, r, c2)
    assert np.array_equal(bits(byptr[cv].cpu().numpy().view(st).reshape(shape)), bits(oc))
    assert np.array_equal(bits(byptr[pv].cpu().numpy().view(st).reshape(shape)), bits(op))


def test_3d_degenerate_shapes(q):
    for shape, chunks in [((1, 1, 1), [(0, 1)]), ((1, 8, 8), [(0, 1)]), ((7, 1, 5), [(0, 7)]),
                          ((5, 6, 1), [(0, 2), (2, 5)])]:
        u0 = field(shape, "f32", seed=8, sigma=1.5)
        p, c = run3d(q, u0, 3, 1, "f32", chunks)
        _, oc = oracle.wave3d_run_mirror(oracle.F32, u0, 3, 1, C2)
        assert np.array_equal(bits(c), bits(oc)), shape


def test_3d_run_graph_equals_steps(q):
    torch = torch_cuda()
    shape = (24, 33, 140)
    u0 = field(shape, "f32", seed=9)
    chunks = sy.sy_split_rows(24, 4)
    d0 = torch.from_numpy(u0).cuda().reshape(-1)
    a, b = torch.empty_like(d0), torch.empty_like(d0)
    p = sy.stencil3d_params(*shape, 2, C2, "f32")
    for steps in (0, 1, 2, 7):
        pv, cv, ev = sy.sy_wave3d_run(q, p, d0, a, b, steps, chunks, 2, want_events=True)
        torch.cuda.synchronize()
        byptr = {d0.data_ptr(): d0, a.data_ptr(): a, b.data_ptr(): b}
        op, oc = oracle.wave3d_run_mirror(oracle.F32, u0, steps, 2, C2)
        assert np.array_equal(byptr[cv].cpu().numpy().view(np.uint32), oc.reshape(-1).view(np.uint32))
        assert np.array_equal(byptr[pv].cpu().numpy().view(np.uint32), op.reshape(-1).view(np.uint32))
        assert len(ev) == (steps + 1) * 4
        times = sy.sy_events_elapsed(q, ev)
        assert all(t > 0 for t in times)
    assert np.array_equal(d0.cpu().numpy(), u0.reshape(-1))  # u0 is never written


def test_3d_errors(q):
    torch = torch_cuda()
    a, b, c = (torch.zeros(8 * 8 * 8, device="cuda") for _ in range(3))
    p = sy.stencil3d_params(8, 8, 8, 2, C2, "f32")
    cases = [((p, a, b, c, [(0, 8)], 1), "SY_ERR_HALO_TOO_SMALL"),
             ((p, a, b, c, [(0, 4), (5, 8)], 2), "SY_ERR_BAD_CHUNKS"),
             ((p, a, b, b, [(0, 8)], 2), "SY_ERR_ALIAS"),
             ((sy.stencil3d_params(8, 8, 8, 5, C2, "f32"), a, b, c, [(0, 8)], 5), "SY_ERR_INVALID_ARGUMENT"),
             ((sy.stencil3d_params(8, 8, 8, 1, C2, "f32", plane=63), a, b, c, [(0, 8)], 1),
              "SY_ERR_INVALID_ARGUMENT"),
             ((sy.stencil3d_params(8, 8, 8, 1, C2, "f32", variant=11), a, b, c, [(0, 8)], 1),
              "SY_ERR_INVALID_ARGUMENT")]
    for args, name in cases:
        with pytest.raises(sy.SyError) as e:
            sy.sy_stencil3d_step(q, *args)
        assert e.value.name == name


def test_3d_full_size_sampled_light_cone(q):
    """512^3 FP32, radius 1, 100 steps, 4 chunks of planes, through sy_wave3d_run (the benchmark's
    configuration): sampled points equal the oracle run on the sub-box of their light cone."""
    torch = torch_cuda()
    n, steps, r = 512, 100, 1
    u0 = inputs.to_storage(inputs.gaussian_pulse_3d(n, n, n, 16.0), "f32")
    d0 = torch.from_numpy(u0).cuda().reshape(-1)
    a, b = torch.empty_like(d0), torch.empty_like(d0)
    p = sy.stencil3d_params(n, n, n, r, C2, "f32")
    _, cv, _ = sy.sy_wave3d_run(q, p, d0, a, b, steps, sy.sy_split_rows(n, 4), r)
    torch.cuda.synchronize()
    cur = {d0.data_ptr(): d0, a.data_ptr(): a, b.data_ptr(): b}[cv].reshape(n, n, n)
    h = (steps + 1) * r + 1
    for pt in [(256, 256, 256), (0, 0, 0), (511, 200, 5), (128, 383, 511), (300, 256, 160)]:
        lo = [max(0, pt[d] - h) for d in range(3)]
        hi = [min(n, pt[d] + h + 1) for d in range(3)]
        sub0 = np.ascontiguousarray(u0[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]])
        _, sub = oracle.wave3d_run_mirror(oracle.F32, sub0, steps, r, C2)
        got = cur[pt].item()
        want = sub[pt[0] - lo[0], pt[1] - lo[1], pt[2] - lo[2]]
        assert np.float32(got).view(np.uint32) == want.view(np.uint32), pt


@pytest.mark.parametrize("dtype,r,steps", [("bf16", 1, 100), ("f32", 2, 30), ("f32", 4, 12), ("bf16", 4, 12)])
def test_3d_full_size_other_forms_sampled(q, dtype, r, steps):
    """512^3 in 4 chunks of planes through sy_wave3d_run with the default variant -- the
    benchmark's BF16 radius-1, FP32 radius-2 and FP32 / BF16 radius-4 forms (radius 2 over 30
    and radius 4 over 12 of their 100 steps, so that the light cones stay small; the launches
    are the same): sampled points equal the oracle's precision mirror on the box of their
    light cone, bit for bit."""
    torch = torch_cuda()
    n = 512
    u0 = inputs.to_storage(inputs.gaussian_pulse_3d(n, n, n, 16.0), dtype)
    d0 = torch.from_numpy(u0 if dtype == "f32" else u0.view(np.int16)).cuda().reshape(-1)
    a, b = torch.empty_like(d0), torch.empty_like(d0)
    p = sy.stencil3d_params(n, n, n, r, C2, dtype)
    _, cv, _ = sy.sy_wave3d_run(q, p, d0, a, b, steps, sy.sy_split_rows(n, 4), r)
    torch.cuda.synchronize()
    cur = {d0.data_ptr(): d0, a.data_ptr(): a, b.data_ptr(): b}[cv].reshape(n, n, n).cpu().numpy()
    if dtype != "f32":
        cur = cur.view(np.uint16)
    h = (steps + 1) * r + 1
    for pt in [(256, 256, 256), (0, 0, 0), (511, 200, 5), (128, 383, 511), (300, 256, 160)]:
        lo = [max(0, pt[d] - h) for d in range(3)]
        hi = [min(n, pt[d] + h + 1) for d in range(3)]
        sub0 = np.ascontiguousarray(u0[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]])
        _, sub = oracle.wave3d_run_mirror(DT[dtype], sub0, steps, r, C2)
        assert bits(cur)[pt] == bits(sub)[pt[0] - lo[0], pt[1] - lo[1], pt[2] - lo[2]], pt


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_3d_256_sampled_light_cone(q, dtype):
    """256^3 (fields larger than L2), radius 1, 20 steps, 4 chunks of planes through sy_wave3d_run;
    sampled points against the oracle on their light cones."""
    torch = torch_cuda()
    n, steps, r = 256, 20, 1
    u0 = inputs.to_storage(inputs.gaussian_pulse_3d(n, n, n, 8.0) + 0.01 * inputs.random_field_3d(2, n, n, n), dtype)
    d0 = torch.from_numpy(u0 if dtype == "f32" else u0.view(np.int16)).cuda().reshape(-1)
    a, b = torch.empty_like(d0), torch.empty_like(d0)
    p = sy.stencil3d_params(n, n, n, r, C2, dtype)
    _, cv, _ = sy.sy_wave3d_run(q, p, d0, a, b, steps, sy.sy_split_rows(n, 4), r)
    torch.cuda.synchronize()
    cur = {d0.data_ptr(): d0, a.data_ptr(): a, b.data_ptr(): b}[cv].reshape(n, n, n).cpu().numpy()
    if dtype != "f32":
        cur = cur.view(np.uint16)
    h = (steps + 1) * r + 1
    for pt in [(128, 128, 128), (0, 0, 0), (255, 255, 255), (64, 191, 3), (200, 0, 130), (127, 128, 255)]:
        lo = [max(0, pt[d] - h) for d in range(3)]
        hi = [min(n, pt[d] + h + 1) for d in range(3)]
        sub0 = np.ascontiguousarray(u0[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]])
        _, sub = oracle.wave3d_run_mirror(DT[dtype], sub0, steps, r, C2)
        assert bits(np.asarray(cur[pt]).reshape(1))[0] == bits(sub[pt[0] - lo[0], pt[1] - lo[1], pt[2] - lo[2]]
                                                               .reshape(1))[0], pt


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("r", [1, 2, 4])
def test_3d_energy_matches_oracle(q, dtype, r):
    torch = torch_cuda()
    shape = (11, 23, 140)
    u_new, u_old = field(shape, dtype, seed=21), field(shape, dtype, seed=22)
    up = lambda u: torch.from_numpy(u if dtype == "f32" else u.view(np.int16)).cuda().reshape(-1)
    p = sy.stencil3d_params(*shape, r, C2, dtype)
    E, kin, pot = sy.sy_wave3d_energy(q, p, up(u_new), up(u_old))
    code = DT[dtype]
    un, uo = oracle.storage_to_f64(u_new, code), oracle.storage_to_f64(u_old, code)
    want = oracle.wave3d_energy_f64(un, uo, r, C2)
    lap = oracle.wave3d_step_f64(2 * uo, uo, r, 1.0)  # (2u - 2u) + L u = L u exactly
    abs_sum = ((un - uo) ** 2).sum() + C2 * np.abs(un * lap).sum()
    # same FP64 terms summed in another order: |difference| <= 2 N eps sum|terms|
    tol = 2 * np.prod(shape) * 2.0 ** -53 * abs_sum
    assert abs(E - want["E"]) <= tol and abs(kin - want["kin"]) <= tol and abs(pot - want["pot"]) <= tol / C2
    assert sy.sy_wave3d_energy(q, p, up(u_new), up(u_old)) == (E, kin, pot)  # fixed reduction shape


def test_3d_energy_conserved_full_size(q):
    """512^3 FP32 r = 1, 100 steps through the graph: the FP64 discrete energy of the FP32 fields
    drifts only by rounding."""
    torch = torch_cuda()
    n, steps = 512, 100
    u0 = torch.from_numpy(inputs.to_storage(inputs.gaussian_pulse_3d(n, n, n, 16.0), "f32")).cuda().reshape(-1)
    a, b = torch.empty_like(u0), torch.empty_like(u0)
    p = sy.stencil3d_params(n, n, n, 1, C2, "f32")
    chunks = sy.sy_split_rows(n, 4)
    pv, cv, _ = sy.sy_wave3d_run(q, p, u0, a, b, 0, chunks, 1)  # start only: prev = u^{-1}, cur = u^0
    E0 = sy.sy_wave3d_energy(q, p, cv, pv)[0]
    pv, cv, _ = sy.sy_wave3d_run(q, p, u0, a, b, steps, chunks, 1)
    E1 = sy.sy_wave3d_energy(q, p, cv, pv)[0]
    assert E0 > 0 and abs(E1 - E0) / E0 < 1e-3


def test_3d_tma_unaligned_layout_falls_back(q):
    shape = (6, 11, 19)
    u0 = field(shape, "f32", seed=6)
    p, c = run3d(q, u0, 3, 1, "f32", [(0, 3), (3, 6)], variant=9, offset=1)
    op, oc = oracle.wave3d_run_mirror(oracle.F32, u0, 3, 1, C2)
    assert np.array_equal(bits(c), bits(oc)) and np.array_equal(bits(p), bits(op))


def test_3d_tma_bounded_wait_times_out_and_context_survives(q):
    """Host-injected fault: each block announces its first plane copy but never issues it; every
    wait is bounded, so the blocks give up, the flag comes back as SY_ERR_TIMEOUT and the context
    keeps working."""
    import os

    torch = torch_cuda()
    shape = (12, 20, 140)
    u0 = field(shape, "f32", seed=13)
    d0 = torch.from_numpy(u0).cuda().reshape(-1)
    prev = torch.empty_like(d0)
    p = sy.stencil3d_params(*shape, 1, C2, "f32", variant=9)
    old = os.environ.get("SY_FAULT")
    os.environ["SY_FAULT"] = "w3_timeout"
    try:
        sy.sy_stencil3d_start(q, p, d0, prev, [(0, 12)], 1)
        with pytest.raises(sy.SyError) as e:
            sy.sy_queue_sync(q)
        assert e.value.name == "SY_ERR_TIMEOUT"
    finally:
        if old is None:
            del os.environ["SY_FAULT"]
        else:
            os.environ["SY_FAULT"] = old
    sy.sy_queue_sync(q)  # reported once and cleared
    pv, cv = run3d(q, u0, 3, 1, "f32", [(0, 6), (6, 12)], variant=9)
    op, oc = oracle.wave3d_run_mirror(oracle.F32, u0, 3, 1, C2)
    assert np.array_equal(bits(cv), bits(oc)) and np.array_equal(bits(pv), bits(op))
