"""Pins of the oracle's second workload (the leapfrog step on a 3D grid) and of its
box range mappers, against facts other than the oracle itself: the exact discrete
solution of a separable standing wave, a dense operator assembled from Kronecker
products of 1D matrices, exactness on polynomials, conservation of the discrete
energy, exact FP32 arithmetic on dyadic integers, the light cone, and brute-force
enumeration of cells for the range mappers and the transfers they imply."""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2505_06022_gb300 import inputs

C2 = 0.125  # (c dt/dx)^2 of the 3D workload: stable for r <= 4 (c2 * max |lambda| <= 2.5 < 4)

FORNBERG = {1: [-2.0, 1.0], 2: [-5 / 2, 4 / 3, -1 / 12], 3: [-49 / 18, 3 / 2, -3 / 20, 1 / 90],
            4: [-205 / 72, 8 / 5, -1 / 5, 8 / 315, -1 / 560]}


def mode3_closed_form(shape, modes, c2, n):
    (nz, ny, nx), (mz, my, mx) = shape, modes
    s2 = sum(math.sin(math.pi * m / (k + 1) / 2) ** 2 for k, m in zip(shape, modes))
    cos_om = 1.0 - 2.0 * c2 * s2
    return math.cos(n * math.acos(cos_om)) * inputs.sine_mode_3d(nz, ny, nx, mz, my, mx)


@pytest.mark.parametrize("shape,modes,steps", [((12, 14, 16), (1, 1, 1), 80), ((12, 14, 16), (5, 7, 9), 80),
                                               ((9, 11, 13), (8, 10, 12), 40), ((1, 10, 12), (1, 3, 4), 30),
                                               ((7, 1, 9), (2, 1, 5), 0), ((7, 5, 9), (2, 1, 5), 1)])
def test_3d_standing_wave_closed_form(shape, modes, steps):
    # the product of three sine modes is an eigenvector of the zero-ghost 7-point operator with
    # eigenvalue -4 sum sin^2(theta_d/2); with the Taylor start u^n = cos(n Omega) u^0 exactly
    u0 = inputs.sine_mode_3d(*shape, *modes)
    prev, cur = oracle.wave3d_run_f64(u0, steps, 1, C2)
    assert np.max(np.abs(cur - mode3_closed_form(shape, modes, C2, steps))) <= 1e-12
    assert np.max(np.abs(prev - mode3_closed_form(shape, modes, C2, steps - 1))) <= 1e-12


def d1(n, r):
    w = FORNBERG[r]
    D = np.zeros((n, n))
    for i in range(n):
        D[i, i] = w[0]
        for k in range(1, r + 1):
            for j in (i - k, i + k):
                if 0 <= j < n:
                    D[i, j] = w[k]
    return D


def kron3(nz, ny, nx, r):
    Iz, Iy, Ix = np.eye(nz), np.eye(ny), np.eye(nx)
    return (np.kron(np.kron(d1(nz, r), Iy), Ix) + np.kron(np.kron(Iz, d1(ny, r)), Ix) +
            np.kron(np.kron(Iz, Iy), d1(nx, r)))


@pytest.mark.parametrize("r", [1, 2, 3, 4])
@pytest.mark.parametrize("shape", [(4, 5, 6), (3, 3, 7), (1, 4, 5), (6, 1, 1), (5, 6, 2)])
def test_3d_stencil_matches_dense_kronecker_operator(r, shape):
    L = kron3(*shape, r)
    u0 = inputs.random_field_3d(31 + r, *shape).astype(np.float64)
    a = u0.reshape(-1) + 0.5 * C2 * (L @ u0.reshape(-1))
    b = u0.reshape(-1).copy()
    for _ in range(20):
        a, b = b, 2 * b - a + C2 * (L @ b)
    prev, cur = oracle.wave3d_run_f64(u0, 20, r, C2)
    scale = max(1.0, np.max(np.abs(b)))
    assert np.max(np.abs(cur.reshape(-1) - b)) <= 1e-12 * scale
    assert np.max(np.abs(prev.reshape(-1) - a)) <= 1e-12 * scale


@pytest.mark.parametrize("dt", [oracle.F32, oracle.BF16, oracle.F16])
@pytest.mark.parametrize("r", [1, 3])
def test_3d_start_mirror_is_the_rounded_taylor_start(dt, r):
    # u^{-1} = u^0 + (c2/2) L u^0 with the dense Kronecker operator in FP64: the mirror's start agrees
    # within one rounding of the storage type (relative to the field's size), equals the run's
    # u^{-1} bit for bit, and with c2 = 0 returns u^0 unchanged
    shape = (4, 5, 7)
    name = {oracle.F32: "f32", oracle.BF16: "bf16", oracle.F16: "f16"}[dt]
    u0 = inputs.to_storage(inputs.random_field_3d(61 + r, *shape).astype(np.float64), name)
    x0 = (oracle.storage_to_f64(u0, dt) if dt != oracle.F32 else u0.astype(np.float64)).reshape(-1)
    want = x0 + 0.5 * C2 * (kron3(*shape, r) @ x0)
    um1 = oracle.wave3d_start_mirror(dt, u0, r, C2)
    got = (oracle.storage_to_f64(um1, dt) if dt != oracle.F32 else um1.astype(np.float64)).reshape(-1)
    ulp = {oracle.F32: 2.0 ** -23, oracle.BF16: 2.0 ** -7, oracle.F16: 2.0 ** -10}[dt]
    assert np.max(np.abs(got - want)) <= 4 * ulp * max(1.0, np.max(np.abs(want)))
    prev0, cur0 = oracle.wave3d_run_mirror(dt, u0, 0, r, C2)
    assert np.array_equal(um1.view(np.uint8), prev0.view(np.uint8))
    assert np.array_equal(cur0.view(np.uint8), u0.view(np.uint8))
    assert np.array_equal(oracle.wave3d_start_mirror(dt, u0, r, 0.0).view(np.uint8), u0.view(np.uint8))


@pytest.mark.parametrize("r", [1, 2])
def test_3d_stencil_exact_on_polynomials(r):
    # L applied to z^a y^b x^c (a+b+c <= 2r+1) is the exact Laplacian at points r away from the
    # boundary; c2 L u is read off one step with u_prev = 2u and c2 = 1.
    shape = (12, 13, 14)
    z, y, x = np.meshgrid(*[np.arange(n, dtype=np.float64) - n // 2 for n in shape], indexing="ij")
    inner = tuple(slice(r, n - r) for n in shape)

    def dd(v, p):  # second derivative of v^p
        return p * (p - 1) * v ** (p - 2) if p >= 2 else 0 * v

    for a, b, c in itertools.product(range(2 * r + 2), repeat=3):
        if a + b + c > 2 * r + 1:
            continue
        u = z ** a * y ** b * x ** c
        exact = dd(z, a) * y ** b * x ** c + z ** a * dd(y, b) * x ** c + z ** a * y ** b * dd(x, c)
        got = oracle.wave3d_step_f64(2 * u, u, r, 1.0)
        assert np.max(np.abs(got[inner] - exact[inner])) <= 1e-9 * max(1.0, np.max(np.abs(u))), (a, b, c)


@pytest.mark.parametrize("r", [1, 2, 4])
def test_3d_discrete_energy_conserved(r):
    shape = (14, 16, 18)
    u0 = inputs.gaussian_pulse_3d(*shape, 2.5) + 0.05 * inputs.random_field_3d(9, *shape)
    um1 = oracle.wave3d_start_f64(u0, r, C2)
    E0 = oracle.wave3d_energy_f64(u0, um1, r, C2)
    assert E0["E"] > 0
    prev, cur = um1, u0
    for _ in range(60):
        prev, cur = cur, oracle.wave3d_step_f64(prev, cur, r, C2)
    E1 = oracle.wave3d_energy_f64(cur, prev, r, C2)
    assert abs(E1["E"] - E0["E"]) <= 1e-11 * (E0["kin"] + C2 * abs(E0["pot"]))
    L = kron3(*shape, r)
    d = (cur - prev).reshape(-1)
    E_dense = d @ d - C2 * cur.reshape(-1) @ (L @ prev.reshape(-1))
    assert abs(E1["E"] - E_dense) <= 1e-11 * (E1["kin"] + C2 * abs(E1["pot"]))


def test_3d_mirror_exact_on_dyadic_integers():
    # integers with c2 = 1/8 and r = 1: every intermediate is a short dyadic rational, so FP32
    # arithmetic is exact and the mirror equals FP64 bit for bit
    shape = (9, 11, 13)
    z = inputs.splitmix64(91, int(np.prod(shape)))
    u0 = ((z % np.uint64(129)).astype(np.int64) - 64).astype(np.float64).reshape(shape)
    p64, c64 = oracle.wave3d_run_f64(u0, 3, 1, C2)
    p32, c32 = oracle.wave3d_run_mirror(oracle.F32, u0.astype(np.float32), 3, 1, C2)
    assert np.array_equal(c32.astype(np.float64), c64) and np.array_equal(p32.astype(np.float64), p64)


@pytest.mark.parametrize("r", [1, 2, 4])
def test_3d_mirror_close_to_f64(r):
    shape = (20, 24, 28)
    u0 = inputs.gaussian_pulse_3d(*shape, 3.0).astype(np.float32)
    _, c64 = oracle.wave3d_run_f64(u0.astype(np.float64), 40, r, C2)
    _, c32 = oracle.wave3d_run_mirror(oracle.F32, u0, 40, r, C2)
    assert np.max(np.abs(c32 - c64)) / np.max(np.abs(c64)) < (1e-5 if r == 1 else 1e-4)


def test_3d_mirror_closed_form_mode():
    shape, modes, steps = (16, 20, 24), (3, 5, 7), 60
    u0 = inputs.sine_mode_3d(*shape, *modes)
    _, c32 = oracle.wave3d_run_mirror(oracle.F32, u0.astype(np.float32), steps, 1, C2)
    assert np.max(np.abs(c32 - mode3_closed_form(shape, modes, C2, steps))) < 1e-5


@pytest.mark.parametrize("dt", ["bf16", "f16"])
def test_3d_mirror_16bit_step_is_rounded_f32_step(dt):
    # a 16-bit step widens, runs the FP32 step and rounds once to storage
    shape = (6, 7, 9)
    code = oracle.DTYPES[dt]
    a = inputs.to_storage(inputs.random_field_3d(12, *shape).astype(np.float64), dt)
    b = inputs.to_storage(inputs.random_field_3d(13, *shape).astype(np.float64), dt)
    got = oracle.wave3d_step_mirror(code, a, b, 2, C2)
    widen = oracle.bf16_to_f32 if dt == "bf16" else oracle.f16_to_f32
    f32 = oracle.wave3d_step_mirror(oracle.F32, widen(a), widen(b), 2, C2)
    assert np.array_equal(got, inputs.to_storage(f32.astype(np.float64), dt))


def test_3d_light_cone_subbox_is_exact():
    shape, r, steps = (30, 32, 34), 1, 8
    u0 = inputs.to_storage(inputs.gaussian_pulse_3d(*shape, 3.0) + 0.01 * inputs.random_field_3d(4, *shape), "f32")
    _, full = oracle.wave3d_run_mirror(oracle.F32, u0, steps, r, C2)
    h = (steps + 1) * r + 1
    for p in [(0, 0, 0), (15, 16, 17), (29, 31, 33), (2, 30, 5)]:
        lo = [max(0, p[d] - h) for d in range(3)]
        hi = [min(shape[d], p[d] + h + 1) for d in range(3)]
        sub0 = np.ascontiguousarray(u0[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]])
        _, sub = oracle.wave3d_run_mirror(oracle.F32, sub0, steps, r, C2)
        assert sub[p[0] - lo[0], p[1] - lo[1], p[2] - lo[2]].view(np.uint32) == full[p].view(np.uint32)


def test_3d_energy_detects_wrong_sign():
    shape = (10, 10, 10)
    u0 = inputs.gaussian_pulse_3d(*shape, 2.0)
    um1 = oracle.wave3d_start_f64(u0, 1, C2)
    E0 = oracle.wave3d_energy_f64(u0, um1, 1, C2)["E"]
    prev, cur = um1, u0
    for _ in range(10):
        prev, cur = cur, oracle.wave3d_step_f64(prev, cur, 1, -C2)
    assert abs(oracle.wave3d_energy_f64(cur, prev, 1, C2)["E"] - E0) > 1e-6 * abs(E0)


# --- 9. box range mappers, by enumerating cells ----------------------------------------

def cells(box):
    (l0, l1, l2), (h0, h1, h2) = box
    return {(a, b, c) for a in range(l0, h0) for b in range(l1, h1) for c in range(l2, h2)}


def brute_required(kind, chunk, extent, radius, dim, fixed):
    """The cells a kernel over `chunk` may access under each mapper's access pattern."""
    inside = lambda p: all(0 <= p[d] < extent[d] for d in range(3))
    out = set()
    if kind == oracle.RM_ALL:
        return cells(((0, 0, 0), tuple(extent)))
    if kind == oracle.RM_FIXED:
        return {p for p in cells(fixed) if inside(p)}
    for q in cells(chunk):
        if kind == oracle.RM_ONE_TO_ONE:
            out.add(q)
        elif kind == oracle.RM_NEIGHBOURHOOD:
            for off in itertools.product(*[range(-radius[d], radius[d] + 1) for d in range(3)]):
                p = tuple(q[d] + off[d] for d in range(3))
                if inside(p):
                    out.add(p)
        elif kind == oracle.RM_SLICE:
            for v in range(extent[dim]):
                p = list(q)
                p[dim] = v
                out.add(tuple(p))
    return out


CASES = [(oracle.RM_ONE_TO_ONE, (0, 0, 0), 0, ((0, 0, 0), (0, 0, 0))),
         (oracle.RM_NEIGHBOURHOOD, (1, 0, 2), 0, ((0, 0, 0), (0, 0, 0))),
         (oracle.RM_NEIGHBOURHOOD, (3, 2, 1), 0, ((0, 0, 0), (0, 0, 0))),
         (oracle.RM_SLICE, (0, 0, 0), 0, ((0, 0, 0), (0, 0, 0))),
         (oracle.RM_SLICE, (0, 0, 0), 2, ((0, 0, 0), (0, 0, 0))),
         (oracle.RM_ALL, (0, 0, 0), 0, ((0, 0, 0), (0, 0, 0))),
         (oracle.RM_FIXED, (0, 0, 0), 0, ((1, -2, 3), (4, 3, 9)))]


def chunkings(extent):
    """Chunk lists tiling the extent: along dimension 0, along dimension 1, and a 2 x 2 grid."""
    e0, e1, e2 = extent
    yield [((a, 0, 0), (b, e1, e2)) for a, b in oracle.split_rows(e0, 3)]
    yield [((0, a, 0), (e0, b, e2)) for a, b in [(0, 1), (1, 2), (2, e1)]]
    yield [((a, c, 0), (b, d, e2)) for a, b in oracle.split_rows(e0, 2) for c, d in oracle.split_rows(e1, 2)]


@pytest.mark.parametrize("kind,radius,dim,fixed", CASES)
def test_rm_box_is_the_clipped_access_set(kind, radius, dim, fixed):
    extent = (6, 5, 7)
    for chunk in [((0, 0, 0), (6, 5, 7)), ((2, 1, 3), (4, 3, 5)), ((0, 4, 0), (1, 5, 2)), ((5, 0, 6), (6, 5, 7))]:
        box = oracle.rm_box(kind, chunk, extent, radius, dim, fixed)
        assert cells(box) == brute_required(kind, chunk, extent, radius, dim, fixed), (kind, chunk)


@pytest.mark.parametrize("kind,radius,dim,fixed", CASES)
def test_rm_box_transfers_cover_exactly_the_missing_cells(kind, radius, dim, fixed):
    extent = (6, 5, 7)
    for chunks in chunkings(extent):
        owner = {}
        for c, ch in enumerate(chunks):
            for p in cells(ch):
                owner[p] = c
        assert len(owner) == 6 * 5 * 7  # the chunk list tiles the buffer
        got = oracle.rm_box_transfers(kind, chunks, extent, radius, dim, fixed)
        cover = {}
        for src, dst, box in got:
            assert src != dst and cells(box) <= cells(chunks[src])
            for p in cells(box):
                assert (dst, p) not in cover
                cover[(dst, p)] = src
        want = {}
        for dst, ch in enumerate(chunks):
            for p in brute_required(kind, ch, extent, radius, dim, fixed) - cells(ch):
                want[(dst, p)] = owner[p]
        assert cover == want
