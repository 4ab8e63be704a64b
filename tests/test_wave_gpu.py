"""Leapfrog wave stencil on the GPU (row chunks with neighbourhood range mappers,
paper §3) against the oracle.

Bar: bit-exact against the precision mirror (same FP32 operation order, same
storage rounding) for every radius, storage type, chunking, tile variant and
layout; and, for FP32 at the 8192 x 8192 / 200-step workload, max|u - u64| /
max|u64| <= 1e-5 against the FP64 oracle on light-cone samples."""
import math

import numpy as np
import pytest

import oracle
import paper_2505_06022_gb300 as sy
from paper_2505_06022_gb300 import inputs

from gpu_helpers import bits, to_device, to_host, torch_cuda, wave_run

pytestmark = pytest.mark.gpu

DT = {"f32": oracle.F32, "bf16": oracle.BF16, "f16": oracle.F16}


@pytest.fixture(scope="module")
def q():
    torch_cuda()
    with sy.Queue(0) as queue:
        yield queue.handle


def field(ny, nx, dtype, seed=1, smooth=True):
    if smooth:
        a = inputs.gaussian_pulse(ny, nx, max(2.0, min(ny, nx) / 6.0)) + 0.05 * inputs.random_field(seed, ny, nx)
    else:
        a = inputs.random_field(seed, ny, nx).astype(np.float64)
    return inputs.to_storage(a, dtype)


SHAPES = [(8, 8), (1, 1), (1, 200), (300, 1), (33, 131), (64, 128), (17, 257), (70, 1030), (129, 64)]


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("r", [1, 2, 3, 4])
@pytest.mark.parametrize("shape", SHAPES)
def test_bit_exact_vs_mirror(q, dtype, r, shape):
    ny, nx = shape
    u0 = field(ny, nx, dtype, seed=r)
    steps = 7
    chunks = sy.sy_split_rows(ny, min(3, ny))
    gp, gc = wave_run(q, u0, steps, r, 0.25, dtype, chunks)
    op, oc = oracle.wave_run_mirror(DT[dtype], u0, steps, r, 0.25)
    assert np.array_equal(bits(gc), bits(oc)) and np.array_equal(bits(gp), bits(op))


def fornberg_weights() -> dict:
    """(w_0, ..., w_r) per radius from the cited fixture tests/golden/fornberg_d2_weights.txt."""
    from fractions import Fraction
    import os

    out = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "fornberg_d2_weights.txt")):
        if line.strip() and not line.startswith("#"):
            r, *w = line.split()
            out[int(r)] = tuple(float(Fraction(x)) for x in w)
    return out


FORNBERG = fornberg_weights()


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_8x8_two_chunks_vs_dense_operator(q, r):
    """8 x 8 grid stepped in the chunks [0, 3) and [3, 8) (a chunk thinner than 2r, and halos
    reaching across several rows of the other chunk): bit-exact against the oracle's mirror, and
    within FP32 rounding of an FP64 iteration with the dense 64 x 64 operator built here point by
    point from the weights."""
    n, steps, c2 = 8, 7, 0.25
    w = FORNBERG[r]
    L = np.zeros((n * n, n * n))
    for i in range(n):
        for j in range(n):
            row = i * n + j
            L[row, row] += 2 * w[0]
            for k in range(1, r + 1):
                for ii, jj in ((i - k, j), (i + k, j), (i, j - k), (i, j + k)):
                    if 0 <= ii < n and 0 <= jj < n:
                        L[row, ii * n + jj] += w[k]
    u0 = field(n, n, "f32", seed=40 + r)
    gp, gc = wave_run(q, u0, steps, r, c2, "f32", [(0, 3), (3, 8)])
    _, oc = oracle.wave_run_mirror(oracle.F32, u0, steps, r, c2)
    assert np.array_equal(bits(gc), bits(oc))
    x0 = u0.astype(np.float64).reshape(-1)
    prev, cur = x0 + 0.5 * c2 * (L @ x0), x0
    for _ in range(steps):
        prev, cur = cur, 2 * cur - prev + c2 * (L @ cur)
    tol = (1e-5 if r == 1 else 1e-4) * np.max(np.abs(cur))
    assert np.max(np.abs(gc.reshape(-1).astype(np.float64) - cur)) <= tol


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("r", [1, 2, 4])
def test_start_bit_exact(q, dtype, r):
    torch = torch_cuda()
    ny, nx = 45, 300
    u0 = field(ny, nx, dtype, smooth=False)
    d0 = to_device(u0)
    dm1 = torch.empty_like(d0)
    p = sy.stencil_params(ny, nx, r, 0.25, dtype)
    sy.sy_stencil_start(q, p, d0, dm1, [(0, ny)], r)
    torch.cuda.synchronize()
    want = oracle.wave_start_mirror(DT[dtype], u0, r, 0.25)
    st = np.float32 if dtype == "f32" else np.uint16
    assert np.array_equal(bits(to_host(dm1, None, st)), bits(want))


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("r", [1, 4])
def test_chunk_invariance(q, dtype, r):
    # The paper's split across devices must not change results: any chunking, same bits.
    ny, nx = 97, 520
    u0 = field(ny, nx, dtype)
    ref = None
    for chunks in [[(0, ny)], sy.sy_split_rows(ny, 2), sy.sy_split_rows(ny, 4), sy.sy_split_rows(ny, 7),
                   [(0, 1), (1, 2), (2, 50), (50, 96), (96, 97)], [(i, i + 1) for i in range(ny)]]:
        _, c = wave_run(q, u0, 9, r, 0.25, dtype, chunks)
        if ref is None:
            ref = c
        assert np.array_equal(bits(c), bits(ref))
    _, oc = oracle.wave_run_mirror(DT[dtype], u0, 9, r, 0.25)
    assert np.array_equal(bits(ref), bits(oc))


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_every_variant_identical(q, dtype, r):
    """Every variant on a ragged width (700 columns) in rows padded to a 16-byte pitch, so
    that each runs its vector (or TMA) form, and on unpadded rows (the scalar fallback
    where a row is not 16-byte aligned)."""
    ny, nx = 75, 700
    u0 = field(ny, nx, dtype)
    _, oc = oracle.wave_run_mirror(DT[dtype], u0, 5, r, 0.25)
    for v in range(0, sy.sy_stencil_variant_count(r, DT[dtype]) + 1):
        for pitch in (704, None):
            _, c = wave_run(q, u0, 5, r, 0.25, dtype, sy.sy_split_rows(ny, 4), variant=v, pitch=pitch)
            assert np.array_equal(bits(c), bits(oc)), f"variant {v} pitch {pitch}"


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("r", [1, 2, 3, 4])
@pytest.mark.parametrize("shape", [(1, 1), (3, 241), (17, 257), (70, 1030), (129, 64), (40, 480), (9, 2000)])
def test_halo_lane_and_narrow_forms_bit_exact(q, dtype, r, shape):
    """The halo-lane tiles (variants 9-12: 30 of 32 lanes store) and, for 16-bit storage,
    the narrow halo-lane tiles (variants 13-14: 8-byte vectors): tiles narrower than the
    grid, wider than it, ragged at nx, grids shorter than a tile or than the radius, and
    chunks of one row."""
    ny, nx = shape
    u0 = field(ny, nx, dtype, seed=r + 7)
    steps = 6
    _, oc = oracle.wave_run_mirror(DT[dtype], u0, steps, r, 0.25)
    chunkings = [sy.sy_split_rows(ny, min(3, ny))]
    if ny >= 5:
        chunkings.append([(0, 1), (1, 2), (2, ny)])
    for v in ((9, 10, 11, 12, 13, 14) if dtype != "f32" else (9, 10, 11, 12)):
        for chunks in chunkings:
            _, c = wave_run(q, u0, steps, r, 0.25, dtype, chunks, variant=v)
            assert np.array_equal(bits(c), bits(oc)), f"variant {v} chunks {chunks}"


MARCH_SHAPES = [(1, 1), (2, 8), (3, 241), (17, 257), (70, 1030), (129, 64), (40, 480), (9, 2000), (300, 300),
                (600, 1000)]


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
@pytest.mark.parametrize("r", [1, 2, 3, 4])
@pytest.mark.parametrize("shape", MARCH_SHAPES)
def test_march_form_bit_exact(q, dtype, r, shape):
    """Variant 15, the march form (rows streamed into shared memory by TMA, a rolling
    window of 2r+1 rows a lane): rows padded to a 16-byte pitch so that the form runs;
    grids narrower than a strip and wider, ragged at nx, shorter than the radius, chunks of
    one row, and segments shorter than the 2r warm-up rows.  The Taylor start and every
    step are bit-identical to the precision mirror."""
    ny, nx = shape
    pitch = (nx + 7) // 8 * 8
    u0 = field(ny, nx, dtype, seed=r + 3)
    steps = 5
    _, oc = oracle.wave_run_mirror(DT[dtype], u0, steps, r, 0.25)
    chunkings = [[(0, ny)], sy.sy_split_rows(ny, min(4, ny))]
    if ny >= 5:
        chunkings.append([(0, 1), (1, 2), (2, ny - 1), (ny - 1, ny)])
    for chunks in chunkings:
        _, c = wave_run(q, u0, steps, r, 0.25, dtype, chunks, variant=15, pitch=pitch)
        assert np.array_equal(bits(c), bits(oc)), f"chunks {chunks}"
    # an unaligned pitch takes the tile launcher's scalar kernel, with the same results
    if nx % 8:
        _, c = wave_run(q, u0, steps, r, 0.25, dtype, chunkings[-1], variant=15)
        assert np.array_equal(bits(c), bits(oc))


def test_march_bounded_wait_times_out_and_context_survives(q):
    """A host-injected fault (SY_FAULT=march_timeout: each warp's first row copy is never
    issued) makes the march kernel's waits run out: the queue reports SY_ERR_TIMEOUT once,
    and the context then runs the same step correctly."""
    import os

    torch = torch_cuda()
    ny, nx, r = 64, 512, 2
    u0 = field(ny, nx, "bf16", seed=2)
    p = sy.stencil_params(ny, nx, r, 0.25, "bf16", variant=15)
    old = os.environ.get("SY_FAULT")
    os.environ["SY_FAULT"] = "march_timeout"
    try:
        cur = to_device(u0)
        prev = torch.empty_like(cur)
        sy.sy_stencil_start(q, p, cur, prev, [(0, ny)], r)
        with pytest.raises(sy.SyError) as e:
            sy.sy_queue_sync(q)
        assert e.value.name == "SY_ERR_TIMEOUT"
    finally:
        if old is None:
            del os.environ["SY_FAULT"]
        else:
            os.environ["SY_FAULT"] = old
    sy.sy_queue_sync(q)  # reported once and cleared
    _, c = wave_run(q, u0, 3, r, 0.25, "bf16", [(0, ny)], variant=15)
    _, oc = oracle.wave_run_mirror(oracle.BF16, u0, 3, r, 0.25)
    assert np.array_equal(bits(c), bits(oc))


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("pitch_extra", [4, 8, 3, 1])
def test_padded_and_unaligned_pitch(q, dtype, pitch_extra):
    # pitch_extra 4/8 keeps rows 16-byte aligned (vector kernel); 1/3 forces the scalar kernel.
    # Padding holds NaN: it must be neither read as data nor written.
    torch = torch_cuda()
    ny, nx, r = 40, 250, 2
    pitch = nx + pitch_extra
    u0 = field(ny, nx, dtype)
    st = np.float32 if dtype == "f32" else np.uint16
    fill = float("nan") if dtype == "f32" else -1
    cur = to_device(u0, pitch, fill=fill)
    prev = torch.empty_like(cur)
    prev.copy_(cur)
    p = sy.stencil_params(ny, nx, r, 0.25, dtype, pitch=pitch)
    sy.sy_stencil_start(q, p, cur, prev, [(0, 13), (13, ny)], r)
    for _ in range(6):
        sy.sy_stencil_step(q, p, prev, cur, prev, [(0, 13), (13, ny)], r)
        prev, cur = cur, prev
    torch.cuda.synchronize()
    full = to_host(cur, None, st)
    _, oc = oracle.wave_run_mirror(DT[dtype], u0, 6, r, 0.25)
    assert np.array_equal(bits(np.ascontiguousarray(full[:, :nx])), bits(oc))
    pad = full[:, nx:]
    assert (np.isnan(pad).all() if dtype == "f32" else (pad.view(np.int16) == -1).all())


def test_unaligned_base_pointer_uses_scalar_path(q):
    torch = torch_cuda()
    ny, nx, r = 21, 64, 1
    u0 = field(ny, nx, "f32")
    big = torch.zeros(3 * (ny * nx + 4), device="cuda")
    a = big[1: 1 + ny * nx]
    b = big[ny * nx + 6: 2 * ny * nx + 6]
    a.copy_(torch.from_numpy(u0.reshape(-1)))
    p = sy.stencil_params(ny, nx, r, 0.25, "f32")
    sy.sy_stencil_start(q, p, a, b, [(0, ny)], r)
    sy.sy_stencil_step(q, p, b, a, b, [(0, ny)], r)
    torch.cuda.synchronize()
    op, oc = oracle.wave_run_mirror(oracle.F32, u0, 1, r, 0.25)
    assert np.array_equal(b.cpu().numpy().reshape(ny, nx).view(np.uint32), oc.view(np.uint32))


def test_out_of_place_equals_in_place(q):
    torch = torch_cuda()
    ny, nx, r = 50, 333, 3
    u0 = field(ny, nx, "f32")
    cur = to_device(u0)
    prev = torch.empty_like(cur)
    p = sy.stencil_params(ny, nx, r, 0.25, "f32")
    sy.sy_stencil_start(q, p, cur, prev, [(0, ny)], r)
    nxt = torch.empty_like(cur)
    sy.sy_stencil_step(q, p, prev, cur, nxt, [(0, ny)], r)
    sy.sy_stencil_step(q, p, prev, cur, prev, [(0, ny)], r)
    torch.cuda.synchronize()
    assert torch.equal(nxt.view(torch.int32), prev.view(torch.int32))


def test_f32_close_to_f64_small(q):
    ny, nx = 256, 256
    u64 = inputs.gaussian_pulse(ny, nx, 16.0)
    u0 = inputs.to_storage(u64, "f32")
    _, gc = wave_run(q, u0, 200, 1, 0.25, "f32", sy.sy_split_rows(ny, 4))
    _, c64 = oracle.wave_run_f64(u0.astype(np.float64), 200, 1, 0.25)
    assert np.max(np.abs(gc - c64)) / np.max(np.abs(c64)) <= 1e-5


def test_standing_mode_closed_form_small(q):
    ny, nx, mx, my, steps = 120, 200, 16, 32, 200
    u0 = inputs.to_storage(inputs.sine_mode(ny, nx, mx, my), "f32")
    _, gc = wave_run(q, u0, steps, 1, 0.25, "f32", sy.sy_split_rows(ny, 4))
    ty, tx = math.pi * my / (ny + 1), math.pi * mx / (nx + 1)
    om = math.acos(1 - 2 * 0.25 * (math.sin(tx / 2) ** 2 + math.sin(ty / 2) ** 2))
    want = math.cos(steps * om) * inputs.sine_mode(ny, nx, mx, my)
    assert np.max(np.abs(gc - want)) <= 1e-5


def test_errors(q):
    torch = torch_cuda()
    ny, nx = 16, 64
    a = torch.zeros(ny, nx, device="cuda")
    b = torch.zeros(ny, nx, device="cuda")
    c = torch.zeros(ny, nx, device="cuda")
    p = sy.stencil_params(ny, nx, 2, 0.25, "f32")
    cases = [
        (dict(chunks=[(0, 8), (9, 16)], halo=2), "SY_ERR_BAD_CHUNKS"),
        (dict(chunks=[(0, 16)], halo=1), "SY_ERR_HALO_TOO_SMALL"),
        (dict(chunks=[(0, 16)], halo=2, nxt=b), "SY_ERR_ALIAS"),
        (dict(chunks=[(0, 16)], halo=2, nxt=a.view(-1)[1:]), "SY_ERR_ALIAS"),
    ]
    before = sy.sy_queue_launch_count(q)
    for kw, name in cases:
        with pytest.raises(sy.SyError) as e:
            sy.sy_stencil_step(q, p, a, b, kw.get("nxt", c), kw["chunks"], kw["halo"])
        assert e.value.name == name
    for bad in [sy.stencil_params(ny, nx, 5, 0.25, "f32"), sy.stencil_params(ny, nx, 1, 0.25, 9),
                sy.stencil_params(ny, nx, 1, 0.25, "f32", pitch=nx - 1),
                sy.stencil_params(ny, nx, 1, 0.25, "f32", variant=99)]:
        with pytest.raises(sy.SyError) as e:
            sy.sy_stencil_step(q, bad, a, b, c, [(0, ny)], 4)
        assert e.value.name == "SY_ERR_INVALID_ARGUMENT"
    assert sy.sy_queue_launch_count(q) == before
    # an empty grid is a no-op with an empty chunk list
    sy.sy_stencil_step(q, sy.stencil_params(0, 0, 1, 0.25, "f32"), a, b, c, [], 1)


# ---- discrete energy (FP64 reduction on the GPU) --------------------------------

@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_energy_matches_oracle(q, dtype, r):
    ny, nx = 77, 301
    u_new = field(ny, nx, dtype, seed=3, smooth=False)
    u_old = field(ny, nx, dtype, seed=4, smooth=False)
    p = sy.stencil_params(ny, nx, r, 0.25, dtype)
    E, kin, pot = sy.sy_wave_energy(q, p, to_device(u_new), to_device(u_old))
    code = DT[dtype]
    want = oracle.wave_energy_f64(oracle.storage_to_f64(u_new, code), oracle.storage_to_f64(u_old, code), r, 0.25)
    # Same FP64 terms, different summation order: |difference| <= 2 * N * eps * sum|terms|
    # (standard bound for two orders of a sum of N terms); in practice ~1e-15.
    tol = 2 * ny * nx * 2.0 ** -53 * want["abs_sum"]
    assert abs(E - want["E"]) <= tol and abs(kin - want["kin"]) <= tol and abs(pot - want["pot"]) <= 8 * tol
    # fixed reduction shape: identical bits on a repeat call
    assert sy.sy_wave_energy(q, p, to_device(u_new), to_device(u_old)) == (E, kin, pot)


def test_energy_conserved_by_gpu_steps(q):
    torch = torch_cuda()
    # r = 1: the FP32 weights are exact, so only rounding of the field can drift E.
    ny, nx, r = 256, 384, 1
    u0 = inputs.to_storage(inputs.gaussian_pulse(ny, nx, 12.0), "f32")
    cur = to_device(u0)
    prev = torch.empty_like(cur)
    p = sy.stencil_params(ny, nx, r, 0.25, "f32")
    chunks = sy.sy_split_rows(ny, 4)
    sy.sy_stencil_start(q, p, cur, prev, chunks, r)
    E0 = sy.sy_wave_energy(q, p, cur, prev)[0]
    for _ in range(200):
        sy.sy_stencil_step(q, p, prev, cur, prev, chunks, r)
        prev, cur = cur, prev
    E1 = sy.sy_wave_energy(q, p, cur, prev)[0]
    assert E0 > 0 and abs(E1 - E0) / E0 < 1e-3  # FP32 storage: drift from rounding only


# ---- the 8192 x 8192, 200-step, 4-chunk FP32 workload at full size ------------------

def light_cone_box(p, shape, steps, r):
    """Clipped box around p holding every point u^steps(p) depends on (start step included)."""
    h = (steps + 1) * r + 1
    (pi, pj), (ny, nx) = p, shape
    return max(0, pi - h), min(ny, pi + h + 1), max(0, pj - h), min(nx, pj + h + 1)


FULL_SAMPLES = [(0, 0), (0, 8191), (8191, 0), (8191, 8191), (0, 4096), (4096, 0), (8191, 4096), (4096, 8191),
                (2047, 4096), (2048, 4096), (6143, 4100), (6144, 4100), (4095, 4096), (4096, 4096),
                (4096, 4196), (4026, 4166), (4096, 3995), (4200, 4001), (4096, 127), (4096, 128),
                (1000, 7000), (7777, 1234)]


def test_config1_full_size_sampled(q):
    ny = nx = 8192
    steps, r = 200, 1
    u0 = inputs.to_storage(inputs.gaussian_pulse(ny, nx, 64.0), "f32")
    gp, gc = wave_run(q, u0, steps, r, 0.25, "f32", sy.sy_split_rows(ny, 4))
    scale = float(np.max(np.abs(gc)))
    assert scale > 0.05
    worst = 0.0
    for pt in FULL_SAMPLES:
        y0, y1, x0, x1 = light_cone_box(pt, (ny, nx), steps, r)
        sub = np.ascontiguousarray(u0[y0:y1, x0:x1])
        _, m32 = oracle.wave_run_mirror(oracle.F32, sub, steps, r, 0.25)
        _, m64 = oracle.wave_run_f64(sub.astype(np.float64), steps, r, 0.25)
        i, j = pt[0] - y0, pt[1] - x0
        assert gc[pt].view(np.uint32) == m32[i, j].view(np.uint32), pt
        worst = max(worst, abs(float(gc[pt]) - m64[i, j]) / scale)
    assert worst <= 1e-5


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
def test_full_size_sampled_through_wave_run(q, dtype):
    """8192^2, radius 1, 200 steps in 4 chunks with FP32, BF16 or FP16 storage, through
    sy_wave_run -- the CUDA graph of chained, overlapped chunk launches the benchmark times:
    sampled points equal the oracle's precision mirror on the box of their light cone, bit
    for bit."""
    torch = torch_cuda()
    ny = nx = 8192
    steps, r = 200, 1
    u0 = inputs.to_storage(inputs.gaussian_pulse(ny, nx, 64.0), dtype)
    d0 = to_device(u0)
    ua, ub = torch.empty_like(d0), torch.empty_like(d0)
    p = sy.stencil_params(ny, nx, r, 0.25, dtype)
    _, cv, _ = sy.sy_wave_run(q, p, d0, ua, ub, steps, sy.sy_split_rows(ny, 4), r)
    torch.cuda.synchronize()
    st = np.float32 if dtype == "f32" else np.uint16
    gc = to_host({d0.data_ptr(): d0, ua.data_ptr(): ua, ub.data_ptr(): ub}[cv], None, st)
    assert np.any(bits(gc) != 0)
    for pt in FULL_SAMPLES:
        y0, y1, x0, x1 = light_cone_box(pt, (ny, nx), steps, r)
        _, m = oracle.wave_run_mirror(DT[dtype], np.ascontiguousarray(u0[y0:y1, x0:x1]), steps, r, 0.25)
        assert bits(gc)[pt] == bits(m)[pt[0] - y0, pt[1] - x0], pt


@pytest.mark.parametrize("dtype,variant", [("bf16", 0), ("bf16", 10), ("f16", 14), ("f32", 9), ("bf16", 15),
                                           ("f16", 15)])
def test_full_size_radius4_forms_sampled(q, dtype, variant):
    """8192^2, radius 4, 40 steps in 4 chunks through sy_wave_run, with the 16-bit default,
    a halo-lane tile, a narrow tile, the FP32 halo-lane tile and the 16-bit march form
    (segment boundaries every few dozen rows): sampled points (corners, chunk and tile boundaries, the centre) equal the
    precision mirror on the box of their light cone, bit for bit."""
    torch = torch_cuda()
    ny = nx = 8192
    steps, r = 40, 4
    u0 = inputs.to_storage(inputs.gaussian_pulse(ny, nx, 64.0) + 0.01 * inputs.random_field(9, ny, nx), dtype)
    d0 = to_device(u0)
    ua, ub = torch.empty_like(d0), torch.empty_like(d0)
    p = sy.stencil_params(ny, nx, r, 0.25, dtype, variant=variant)
    _, cv, _ = sy.sy_wave_run(q, p, d0, ua, ub, steps, sy.sy_split_rows(ny, 4), r)
    torch.cuda.synchronize()
    st = np.float32 if dtype == "f32" else np.uint16
    gc = to_host({d0.data_ptr(): d0, ua.data_ptr(): ua, ub.data_ptr(): ub}[cv], None, st)
    for pt in FULL_SAMPLES[:12] + [(4096, 239), (4096, 240), (4096, 119), (4096, 120), (2043, 4000)]:
        y0, y1, x0, x1 = light_cone_box(pt, (ny, nx), steps, r)
        _, m = oracle.wave_run_mirror(DT[dtype], np.ascontiguousarray(u0[y0:y1, x0:x1]), steps, r, 0.25)
        assert bits(gc)[pt] == bits(m)[pt[0] - y0, pt[1] - x0], pt


@pytest.mark.parametrize("mx,my", [(1, 1), (16, 32), (1000, 3000)])
def test_config1_mode_closed_form_full_size(q, mx, my):
    # single sin(kx x) sin(ky y) mode on the full grid: u^n = cos(n Omega) u^0 everywhere; the
    # bar (1e-5 of the amplitude) applies to the largest pointwise error and to the L2-relative one
    ny = nx = 8192
    steps = 200
    mode = inputs.sine_mode(ny, nx, mx, my)
    u0 = inputs.to_storage(mode, "f32")
    _, gc = wave_run(q, u0, steps, 1, 0.25, "f32", sy.sy_split_rows(ny, 4))
    ty, tx = math.pi * my / (ny + 1), math.pi * mx / (nx + 1)
    om = math.acos(1 - 2 * 0.25 * (math.sin(tx / 2) ** 2 + math.sin(ty / 2) ** 2))
    want = math.cos(steps * om) * mode
    diff = gc - want
    err = np.max(np.abs(diff))
    l2 = math.sqrt(float(np.sum(diff * diff)) / float(np.sum(mode * mode)))
    assert err <= 1e-5 and l2 <= 1e-5, (err, l2)


def test_config1_energy_drift_full_size(q):
    torch = torch_cuda()
    ny = nx = 8192
    u0 = inputs.to_storage(inputs.gaussian_pulse(ny, nx, 64.0), "f32")
    cur = to_device(u0)
    prev = torch.empty_like(cur)
    p = sy.stencil_params(ny, nx, 1, 0.25, "f32")
    chunks = sy.sy_split_rows(ny, 4)
    sy.sy_stencil_start(q, p, cur, prev, chunks, 1)
    E0 = sy.sy_wave_energy(q, p, cur, prev)[0]
    for _ in range(200):
        sy.sy_stencil_step(q, p, prev, cur, prev, chunks, 1)
        prev, cur = cur, prev
    E1 = sy.sy_wave_energy(q, p, cur, prev)[0]
    assert E0 > 0 and abs(E1 - E0) / E0 < 1e-3


@pytest.mark.parametrize("c2", [0.0, 0.1, 0.3, 0.49, 1.7])
@pytest.mark.parametrize("dtype,r", [("f32", 1), ("f32", 3), ("bf16", 2), ("f16", 1)])
def test_any_c2_bit_exact(q, c2, dtype, r):
    # c2 not a power of two (its FP32 rounding, and c2/2 for the start, enter every update),
    # c2 = 0 (pure inertia) and an unstable c2 = 1.7 (growing values) all stay bit-exact
    ny, nx = 41, 300
    u0 = field(ny, nx, dtype, seed=11)
    gp, gc = wave_run(q, u0, 5, r, c2, dtype, sy.sy_split_rows(ny, 3))
    op, oc = oracle.wave_run_mirror(DT[dtype], u0, 5, r, c2)
    assert np.array_equal(bits(gc), bits(oc)) and np.array_equal(bits(gp), bits(op))


# ---- whole-run entry (CUDA graph) and per-chunk timestamps ---------------------------

@pytest.mark.parametrize("steps", [0, 1, 2, 3, 10])
@pytest.mark.parametrize("dtype,r,nch", [("f32", 1, 4), ("f16", 3, 1), ("bf16", 2, 3)])
def test_wave_run_matches_oracle(q, steps, dtype, r, nch):
    torch = torch_cuda()
    ny, nx = 66, 530
    u0 = field(ny, nx, dtype)
    d0 = to_device(u0)
    ua, ub = torch.empty_like(d0), torch.empty_like(d0)
    p = sy.stencil_params(ny, nx, r, 0.25, dtype)
    chunks = sy.sy_split_rows(ny, nch)
    for _ in range(2):  # the second call replays the cached graph
        pv, cv, evs = sy.sy_wave_run(q, p, d0, ua, ub, steps, chunks, r, want_events=True)
        torch.cuda.synchronize()
        byptr = {d0.data_ptr(): d0, ua.data_ptr(): ua, ub.data_ptr(): ub}
        st = np.float32 if dtype == "f32" else np.uint16
        op, oc = oracle.wave_run_mirror(DT[dtype], u0, steps, r, 0.25)
        assert np.array_equal(bits(to_host(byptr[cv], None, st)), bits(oc))
        assert np.array_equal(bits(to_host(byptr[pv], None, st)), bits(op))
        assert np.array_equal(bits(to_host(d0, None, st)), bits(u0))  # u0 never written
        assert len(evs) == (steps + 1) * nch
        ms = sy.sy_events_elapsed(q, evs)
        assert all(m > 0 for m in ms) and ms[0] == sy.sy_event_elapsed(q, evs[0])


def test_wave_run_events_in_chunk_order(q):
    """The run launches alternate steps' chunks in reverse order; the ids it returns stay in chunk
    order: with a thin and a thick chunk, every step's first id times the thin one."""
    torch = torch_cuda()
    ny, nx, steps = 4096, 4096, 5
    d0 = to_device(inputs.to_storage(inputs.gaussian_pulse(ny, nx, 50.0), "f32"))
    ua, ub = torch.empty_like(d0), torch.empty_like(d0)
    p = sy.stencil_params(ny, nx, 1, 0.25, "f32")
    chunks = [(0, 8), (8, ny)]
    for _ in range(2):
        _, _, evs = sy.sy_wave_run(q, p, d0, ua, ub, steps, chunks, 1, want_events=True)
        torch.cuda.synchronize()
        ms = sy.sy_events_elapsed(q, evs)
        assert len(ms) == 2 * (steps + 1)
        for s in range(steps + 1):
            assert ms[2 * s + 1] > 2 * ms[2 * s], (s, ms)  # about 2-3 us against 20 us


def test_wave_run_graph_cache_follows_every_argument(q):
    """One cached graph per queue: any change of grid parameters, c2, step count, chunks, halo,
    variant or buffers must re-capture; returning to earlier arguments must not replay a stale graph."""
    torch = torch_cuda()
    ny, nx = 40, 264
    u0 = field(ny, nx, "f32", seed=21)
    u1 = field(ny, nx, "f32", seed=22)
    d0, d1 = to_device(u0), to_device(u1)
    ua, ub, uc = (torch.empty_like(d0) for _ in range(3))
    base = dict(r=1, c2=0.25, steps=4, chunks=[(0, 20), (20, 40)], halo=1, variant=0, src=(d0, u0), bufs=(ua, ub))
    cases = [base, dict(base, c2=0.3), dict(base, steps=5), dict(base, chunks=[(0, 7), (7, 40)]), dict(base, halo=2),
             dict(base, variant=3), dict(base, r=2, halo=2), dict(base, src=(d1, u1)), dict(base, bufs=(ub, uc)), base]
    for c in cases:
        dsrc, hsrc = c["src"]
        p = sy.stencil_params(ny, nx, c["r"], c["c2"], "f32", variant=c["variant"])
        pv, cv, _ = sy.sy_wave_run(q, p, dsrc, c["bufs"][0], c["bufs"][1], c["steps"], c["chunks"], c["halo"])
        torch.cuda.synchronize()
        byptr = {t.data_ptr(): t for t in (d0, d1, ua, ub, uc)}
        op, oc = oracle.wave_run_mirror(oracle.F32, hsrc, c["steps"], c["r"], c["c2"])
        assert np.array_equal(bits(to_host(byptr[cv], None, np.float32)), bits(oc)), c
        assert np.array_equal(bits(to_host(byptr[pv], None, np.float32)), bits(op)), c


def test_wave_run_errors(q):
    torch = torch_cuda()
    a = torch.zeros(8, 64, device="cuda")
    b = torch.zeros(8, 64, device="cuda")
    p = sy.stencil_params(8, 64, 1, 0.25, "f32")
    with pytest.raises(sy.SyError) as e:
        sy.sy_wave_run(q, p, a, a, b, 3, [(0, 8)], 1)
    assert e.value.name == "SY_ERR_ALIAS"
    with pytest.raises(sy.SyError) as e:
        sy.sy_wave_run(q, p, a, b, torch.zeros(8, 64, device="cuda"), 3, [(0, 4)], 1)
    assert e.value.name == "SY_ERR_BAD_CHUNKS"
    big = sy.stencil_params(8, 64, 1, 0.25, "f32")
    with pytest.raises(sy.SyError) as e:
        sy.sy_wave_run(q, big, a, b, torch.zeros(8, 64, device="cuda"), 20000, [(0, 8)], 1, want_events=True)
    assert e.value.name == "SY_ERR_INVALID_ARGUMENT"


def test_stream_events_and_energy_window(q):
    import time

    torch = torch_cuda()
    ny, nx = 2048, 4096
    u0 = to_device(inputs.to_storage(inputs.gaussian_pulse(ny, nx, 50.0), "f32"))
    prev, cur = torch.empty_like(u0), u0.clone()
    p = sy.stencil_params(ny, nx, 1, 0.25, "f32")
    chunks = sy.sy_split_rows(ny, 4)
    try:
        sy.sy_meter_begin(q)
        metered = True
    except sy.SyError as e:
        assert e.name == "SY_ERR_NVML_UNAVAILABLE"
        metered = False
    evs = []
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < 0.6:  # the energy counter ticks coarsely: meter >= 0.5 s
        for _ in range(100):
            e = sy.sy_stencil_step(q, p, prev, cur, prev, chunks, 1, want_events=len(evs) < 4000)
            evs += e
            prev, cur = cur, prev
        torch.cuda.synchronize()
    ms = sy.sy_events_elapsed(q, evs)
    assert all(0 < m < 50 for m in ms)
    if metered:
        joules, seconds = sy.sy_meter_end(q)
        assert joules > 0 and seconds >= 0.6
        watts = joules / seconds
        assert 20 < watts < 2000
        kj = [sy.sy_kernel_energy(q, e) for e in evs[:8]]
        assert all(j > 0 for j in kj)
        assert sum(sy.sy_kernel_energy(q, e) for e in evs) <= joules * 1.01
    # per-chunk statistics of the first stepped chunk list: time, bytes, updates (and energy)
    stats = sy.sy_chunk_stats_read(q, p, chunks, evs[:4])
    assert [st["updates"] for st in stats] == [(b - a) * nx for a, b in chunks]
    assert all(st["bytes"] == 12 * st["updates"] and st["ms"] == m for st, m in zip(stats, ms[:4]))
    assert all((st["joules"] > 0) if metered else (st["joules"] == -1.0) for st in stats)


def test_chunk_energy_replay_measures_one_chunk(q):
    """sy_chunk_energy_replay: one chunk's launch replayed alone in a metering window.  Its output
    rows equal a normal step's, its device time per launch is that chunk's, and the power it
    implies is a physical one (NVML energy is not an oracle quantity: parity unpinned)."""
    torch = torch_cuda()
    ny, nx = 2048, 8192
    u0 = to_device(inputs.to_storage(inputs.gaussian_pulse(ny, nx, 50.0), "f32"))
    prev, nxt, ref = u0.clone(), torch.zeros_like(u0), torch.zeros_like(u0)
    p = sy.stencil_params(ny, nx, 1, 0.25, "f32")
    chunks = sy.sy_split_rows(ny, 4)
    a, b = chunks[1]
    ev = sy.sy_stencil_step(q, p, prev, u0, ref, chunks, 1, want_events=True)
    torch.cuda.synchronize()
    chunk_ms = sy.sy_events_elapsed(q, ev)[1]
    cur_before = u0.clone()
    try:
        r = sy.sy_chunk_energy_replay(q, p, prev, u0, nxt, chunks, 1, 1, min_seconds=0.6, min_reps=50)
        metered = True
    except sy.SyError as e:
        assert e.name == "SY_ERR_NVML_UNAVAILABLE"
        metered = False
    torch.cuda.synchronize()
    assert torch.equal(u0, cur_before)  # inputs untouched
    assert torch.equal(nxt[a:b].view(torch.int32), ref[a:b].view(torch.int32))
    assert not nxt[:a].any() and not nxt[b:].any()  # only the chunk's rows are written
    if metered:
        assert r["reps"] >= 50 and r["joules"] > 0
        assert 0.2 * chunk_ms < r["ms"] < 5 * chunk_ms
        watts = r["joules"] / (r["ms"] * 1e-3)
        assert 20 < watts < 2000, watts
    bad = sy.stencil_params(ny, nx, 1, 0.25, "f32")
    with pytest.raises(sy.SyError) as e:
        sy.sy_chunk_energy_replay(q, bad, prev, u0, nxt, chunks, 4, 1)
    assert e.value.name == "SY_ERR_INVALID_ARGUMENT"


def test_energy_counter_ticks(q):
    """The device energy counter is monotone and advances while the GPU works."""
    import time

    try:
        first = sy.sy_energy_read(q)
    except sy.SyError as e:
        assert e.name == "SY_ERR_NVML_UNAVAILABLE"
        return
    vals, t0 = [first], time.perf_counter()
    while time.perf_counter() - t0 < 1.0:
        vals.append(sy.sy_energy_read(q))
        time.sleep(0.002)
    assert all(b >= a for a, b in zip(vals, vals[1:]))
    assert vals[-1] > vals[0]
    assert sy.sy_device_energy(q) >= 0
