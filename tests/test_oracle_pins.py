"""Pins of the CPU oracle to facts outside itself (CPU only).

Each test ties an oracle routine to something it cannot simply agree with by
construction: a published value (tests/golden), a closed-form solution, an
exact invariant, a special case where the arithmetic is exact, a library
routine the oracle does not use, or brute force on tiny inputs.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2505_06022_gb300 import inputs

GOLDEN = __file__.rsplit("/", 1)[0] + "/golden/"


def golden_weights():
    out = {}
    for line in open(GOLDEN + "fornberg_d2_weights.txt"):
        if line.startswith("#") or not line.strip():
            continue
        parts = line.split()
        out[int(parts[0])] = [Fraction(p) for p in parts[1:]]
    return out


# --- input generator (shared by both sides) ---------------------------------

def test_splitmix64_published_vectors():
    for line in open(GOLDEN + "splitmix64_vectors.txt"):
        if line.startswith("#") or not line.strip():
            continue
        p = line.split()
        if p[0] == "buckets":
            state, n, counts = int(p[1]), int(p[2]), [int(c) for c in p[3:]]
            f = inputs.uniform01_f64(state, n)
            assert np.bincount((f * 5).astype(int), minlength=5).tolist() == counts
        else:
            state, idx, want = int(p[0]), int(p[1]), int(p[2])
            assert int(inputs.splitmix64(state, 1, offset=idx)[0]) == want


def test_uniform_pm1_exact_and_in_range():
    x = inputs.uniform_pm1_f32(0, 1 << 16)
    assert x.dtype == np.float32 and x.min() >= -1.0 and x.max() < 1.0
    m = (inputs.splitmix64(0, 1 << 16) >> np.uint64(40)).astype(np.float64)
    assert np.array_equal(x.astype(np.float64), m / 2 ** 23 - 1.0)


# --- 1. SAXPY (paper §2 Listing 1) --------------------------------------------

def _rn32(v64):
    return np.asarray(v64, np.float64).astype(np.float32)


@pytest.mark.parametrize("n", [0, 1, 7, 1000, 1 << 14])
def test_saxpy_f32_is_two_single_roundings(n):
    # x, y are 24-bit fixed point, so alpha*x and fl(alpha*x)+y are exact in FP64;
    # IEEE single arithmetic is the exact result rounded once.
    x, y = inputs.saxpy_inputs(n, seed=0)
    alpha = 2.5
    z = oracle.saxpy_f32(alpha, x, y)
    t = _rn32(alpha * x.astype(np.float64))
    want = _rn32(t.astype(np.float64) + y.astype(np.float64))
    assert z.dtype == np.float32 and np.array_equal(z.view(np.uint32), want.view(np.uint32))


def test_saxpy_special_cases():
    x, y = inputs.saxpy_inputs(4096, seed=3)
    assert np.array_equal(oracle.saxpy_f32(0.0, x, y), y)
    assert np.array_equal(oracle.saxpy_f32(1.0, x, np.zeros_like(y)), x)
    assert np.array_equal(oracle.saxpy_f32(-1.0, x, x), np.zeros_like(x))
    z64 = oracle.saxpy_f64(2.5, x, y)
    assert np.array_equal(z64, 2.5 * x.astype(np.float64) + y.astype(np.float64))  # exact here
    # FP32 result within one rounding of each operation of the FP64 result
    z32 = oracle.saxpy_f32(2.5, x, y).astype(np.float64)
    assert np.max(np.abs(z32 - z64)) <= 2 * 2.0 ** -24 * 4.0


# --- 2. range mappers (paper §3) ----------------------------------------------

@pytest.mark.parametrize("ny,k", [(8192, 4), (10, 3), (7, 7), (5, 1), (100, 9), (0, 1)])
def test_split_rows_tiles(ny, k):
    ch = oracle.split_rows(ny, k)
    assert len(ch) == k and ch[0][0] == 0 and ch[-1][1] == ny
    for (a, b), (c, d) in zip(ch, ch[1:]):
        assert b == c
    sizes = [b - a for a, b in ch]
    assert max(sizes) - min(sizes) <= 1 and sizes == sorted(sizes, reverse=True)
    if ny >= k:
        assert oracle.chunks_valid(ny, ch)


def test_rm_neighbourhood_brute_force():
    for ny in (1, 5, 17):
        for r in (1, 2, 4):
            for a in range(ny):
                for b in range(a + 1, ny + 1):
                    touched = {i + d for i in range(a, b) for d in range(-r, r + 1) if 0 <= i + d < ny}
                    lo, hi = oracle.rm_neighbourhood(a, b, r, ny)
                    assert set(range(lo, hi)) == touched
                    assert oracle.rm_one_to_one(a, b) == (a, b)


def test_chunks_valid_rejects():
    assert not oracle.chunks_valid(10, [(0, 5), (6, 10)])      # gap
    assert not oracle.chunks_valid(10, [(0, 6), (5, 10)])      # overlap
    assert not oracle.chunks_valid(10, [(0, 5), (5, 9)])       # short
    assert not oracle.chunks_valid(10, [(0, 0), (0, 10)])      # empty chunk
    assert not oracle.chunks_valid(10, [(5, 10), (0, 5)])      # out of order
    assert oracle.chunks_valid(10, [(0, 1), (1, 10)])


# --- 3. weights -----------------------------------------------------------------

@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_weights_match_fornberg_table(r):
    want = [float(f) for f in golden_weights()[r]]
    got = oracle.d2_weights(r)
    np.testing.assert_allclose(got, want, rtol=2e-16, atol=0)


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_weights_moment_conditions(r):
    # sum_k w_k (f(-k) + f(k)) + w_0 f(0) = f''(0) exactly for f = x^m, m <= 2r+1,
    # and fails at m = 2r+2 (accuracy order exactly 2r).
    w = [Fraction(x) for x in golden_weights()[r]]
    got = oracle.d2_weights(r)
    for m in range(0, 2 * r + 3):
        val = (w[0] if m == 0 else 0) + sum(w[k] * ((-k) ** m + k ** m) for k in range(1, r + 1))
        num = got[0] * (1.0 if m == 0 else 0.0) + sum(got[k] * ((-k) ** m + k ** m) for k in range(1, r + 1))
        exact = 2 if m == 2 else 0
        if m <= 2 * r + 1:
            assert val == exact
            assert abs(num - exact) < 1e-9 * max(1, 4 ** m)
        else:
            assert val != exact


# --- 4. FP64 stencil --------------------------------------------------------------

def mode_closed_form(ny, nx, mx, my, c2, n):
    ty, tx = math.pi * my / (ny + 1), math.pi * mx / (nx + 1)
    cos_om = 1.0 - 2.0 * c2 * (math.sin(tx / 2) ** 2 + math.sin(ty / 2) ** 2)
    return math.cos(n * math.acos(cos_om)) * inputs.sine_mode(ny, nx, mx, my)


@pytest.mark.parametrize("ny,nx,mx,my,steps", [(48, 64, 1, 1, 200), (48, 64, 16, 32, 200), (37, 53, 50, 30, 60),
                                               (64, 48, 3, 5, 0), (64, 48, 3, 5, 1), (1, 9, 4, 1, 40)])
def test_standing_wave_closed_form(ny, nx, mx, my, steps):
    # u^n = cos(n Omega) u^0 with cos(Omega) = 1 - 2 c2 (sin^2(tx/2) + sin^2(ty/2)): the exact
    # discrete solution of the zero-ghost 5-point leapfrog with the Taylor start.
    c2 = 0.25
    u0 = inputs.sine_mode(ny, nx, mx, my)
    prev, cur = oracle.wave_run_f64(u0, steps, 1, c2)
    want_cur = mode_closed_form(ny, nx, mx, my, c2, steps)
    want_prev = mode_closed_form(ny, nx, mx, my, c2, steps - 1)
    assert np.max(np.abs(cur - want_cur)) <= 1e-12 * max(1.0, np.max(np.abs(u0)))
    assert np.max(np.abs(prev - want_prev)) <= 1e-12


def kron_operator(ny, nx, r):
    """Dense L = I (x) D_nx + D_ny (x) I from textbook weights; truncation = zero ghosts."""
    w = [float(f) for f in golden_weights()[r]]

    def d1(n):
        D = np.zeros((n, n))
        for i in range(n):
            D[i, i] = w[0]
            for k in range(1, r + 1):
                for j in (i - k, i + k):
                    if 0 <= j < n:
                        D[i, j] = w[k]
        return D

    return np.kron(np.eye(ny), d1(nx)) + np.kron(d1(ny), np.eye(nx))


@pytest.mark.parametrize("r", [1, 2, 3, 4])
@pytest.mark.parametrize("ny,nx", [(8, 8), (7, 9), (3, 5), (1, 6)])
def test_stencil_matches_dense_kronecker_operator(r, ny, nx):
    c2 = 0.25
    L = kron_operator(ny, nx, r)
    u0 = inputs.random_field(11 + r, ny, nx).astype(np.float64)
    um1 = u0.reshape(-1) + 0.5 * c2 * (L @ u0.reshape(-1))
    a, b = um1, u0.reshape(-1).copy()
    for _ in range(25):
        a, b = b, 2 * b - a + c2 * (L @ b)
    prev, cur = oracle.wave_run_f64(u0, 25, r, c2)
    scale = max(1.0, np.max(np.abs(b)))
    assert np.max(np.abs(cur.reshape(-1) - b)) <= 1e-12 * scale
    assert np.max(np.abs(prev.reshape(-1) - a)) <= 1e-12 * scale


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_stencil_exact_on_polynomials(r):
    # Interior points far from the boundary: L applied to x^a y^b (a+b <= 2r+1) gives the
    # exact Laplacian.  Extract c2*L u from one step with u_prev = 2u.
    ny, nx = 24, 26
    i = np.arange(ny, dtype=np.float64)[:, None] - 11.0
    j = np.arange(nx, dtype=np.float64)[None, :] - 13.0
    inner = (slice(r, ny - r), slice(r, nx - r))
    for a in range(0, 2 * r + 2):
        for b in range(0, 2 * r + 2 - a):
            u = (j ** a) * (i ** b) * np.ones((ny, nx))
            lap_exact = (a * (a - 1) * j ** max(a - 2, 0) * i ** b if a >= 2 else 0 * u) + \
                        (b * (b - 1) * i ** max(b - 2, 0) * j ** a if b >= 2 else 0 * u)
            got = oracle.wave_step_f64(2 * u, u, r, 1.0)
            err = np.max(np.abs(got[inner] - np.broadcast_to(lap_exact, u.shape)[inner]))
            assert err <= 1e-9 * max(1.0, np.max(np.abs(u))), (a, b, err)


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_discrete_energy_conserved(r):
    c2 = 0.25
    ny, nx = 40, 56
    u0 = inputs.gaussian_pulse(ny, nx, 4.0) + 0.1 * inputs.random_field(5, ny, nx)
    um1 = oracle.wave_start_f64(u0, r, c2)
    E0 = oracle.wave_energy_f64(u0, um1, r, c2)
    assert E0["E"] > 0
    prev, cur = um1, u0
    for _ in range(200):
        prev, cur = cur, oracle.wave_step_f64(prev, cur, r, c2)
    E1 = oracle.wave_energy_f64(cur, prev, r, c2)
    assert abs(E1["E"] - E0["E"]) <= 1e-12 * E0["abs_sum"]
    # the energy formula itself on the dense operator
    L = kron_operator(ny, nx, r)
    d = (cur - prev).reshape(-1)
    E_dense = d @ d - c2 * cur.reshape(-1) @ (L @ prev.reshape(-1))
    assert abs(E1["E"] - E_dense) <= 1e-12 * E1["abs_sum"]


def test_energy_detects_wrong_sign():
    # A flipped force sign breaks conservation: guards the invariant test's power.
    c2 = 0.25
    u0 = inputs.gaussian_pulse(30, 30, 3.0)
    um1 = oracle.wave_start_f64(u0, 1, c2)
    E0 = oracle.wave_energy_f64(u0, um1, 1, c2)["E"]
    prev, cur = um1, u0
    for _ in range(20):
        prev, cur = cur, oracle.wave_step_f64(prev, cur, 1, -c2)
    assert abs(oracle.wave_energy_f64(cur, prev, 1, c2)["E"] - E0) > 1e-6 * abs(E0)


def test_light_cone_subbox_is_exact():
    # The value at p after s steps depends only on points within (s+1)*r (start step
    # included); the oracle on a clipped sub-box reproduces it bit for bit.  Full-size
    # GPU parity tests rely on this.
    ny, nx, r, steps = 96, 80, 2, 12
    u0 = inputs.to_storage(inputs.gaussian_pulse(ny, nx, 9.0) + 0.01 * inputs.random_field(3, ny, nx), "f32")
    _, full = oracle.wave_run_mirror(oracle.F32, u0, steps, r, 0.25)
    h = (steps + 1) * r + 1
    for (pi, pj) in [(0, 0), (50, 40), (95, 79), (3, 77), (60, 1)]:
        y0, y1 = max(0, pi - h), min(ny, pi + h + 1)
        x0, x1 = max(0, pj - h), min(nx, pj + h + 1)
        _, sub = oracle.wave_run_mirror(oracle.F32, np.ascontiguousarray(u0[y0:y1, x0:x1]), steps, r, 0.25)
        assert sub[pi - y0, pj - x0].view(np.uint32) == full[pi, pj].view(np.uint32)


# --- 5. precision mirror -----------------------------------------------------------

def test_mirror_f32_exact_on_dyadic_integers():
    # Integer fields with c2 = 1/4 and r = 1: every intermediate is a short dyadic
    # rational, so FP32 arithmetic is exact and the mirror equals FP64 bit for bit.
    rng = inputs.splitmix64(77, 33 * 29)
    u0 = ((rng % np.uint64(129)).astype(np.int64) - 64).astype(np.float64).reshape(33, 29)
    p64, c64 = oracle.wave_run_f64(u0, 3, 1, 0.25)
    p32, c32 = oracle.wave_run_mirror(oracle.F32, u0.astype(np.float32), 3, 1, 0.25)
    assert np.array_equal(c32.astype(np.float64), c64) and np.array_equal(p32.astype(np.float64), p64)


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_mirror_f32_close_to_f64(r):
    ny, nx, steps = 64, 72, 100
    u0 = inputs.gaussian_pulse(ny, nx, 6.0)
    _, c64 = oracle.wave_run_f64(u0.astype(np.float32).astype(np.float64), steps, r, 0.25)
    _, c32 = oracle.wave_run_mirror(oracle.F32, u0.astype(np.float32), steps, r, 0.25)
    # r = 1: weights 1, -4 and c2 = 1/4 are exact in FP32, only the adds round.
    # r >= 2: the FP32-rounded weights (up to 2^-24 relative each) no longer sum to
    # zero, which perturbs the operator itself; over 100 steps that gives ~3e-5.
    bar = 2e-5 if r == 1 else 1e-4
    assert np.max(np.abs(c32 - c64)) / np.max(np.abs(c64)) < bar


def test_mirror_f32_closed_form_mode():
    ny, nx, steps = 48, 64, 200
    u0 = inputs.sine_mode(ny, nx, 16, 32)
    _, c32 = oracle.wave_run_mirror(oracle.F32, u0.astype(np.float32), steps, 1, 0.25)
    want = mode_closed_form(ny, nx, 16, 32, 0.25, steps)
    assert np.max(np.abs(c32 - want)) / np.max(np.abs(u0)) < 1e-5


def _interesting_floats():
    rng = inputs.splitmix64(2024, 200000)
    bits = (rng >> np.uint64(32)).astype(np.uint32)
    vals = bits.view(np.float32)
    vals = vals[np.isfinite(vals)]
    extra = np.array([0.0, -0.0, 1.0, -1.0, 65504.0, 65519.996, 65520.0, 65536.0, 1e-8, 5.96e-8, 2.98e-8,
                      2.9802322e-08, 6.1035156e-05, 6.0975552e-05, 3.0e38, 1e-40, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8,
                      1.0 + 2 ** -11, 1.0 + 3 * 2 ** -11, np.inf, -np.inf], np.float32)
    small = (inputs.uniform_pm1_f32(9, 50000) * np.float32(1e-4)).astype(np.float32)
    return np.concatenate([vals[:60000], extra, small])


def test_f16_rounding_matches_ieee_conversion():
    v = _interesting_floats()
    got = oracle.f32_to_f16(v)
    want = v.astype(np.float16).view(np.uint16)
    assert np.array_equal(got, want)
    back = oracle.f16_to_f32(want)
    assert np.array_equal(back.view(np.uint32), want.view(np.float16).astype(np.float32).view(np.uint32))
    assert oracle.f32_to_f16(np.array([np.nan], np.float32))[0] & 0x7C00 == 0x7C00


def test_bf16_rounding_matches_torch_conversion():
    torch = pytest.importorskip("torch")
    v = _interesting_floats()
    got = oracle.f32_to_bf16(v)
    want = torch.from_numpy(v).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(got, want)
    back = oracle.bf16_to_f32(want)
    assert np.array_equal(back.view(np.uint32), want.astype(np.uint32) << 16)


@pytest.mark.parametrize("dt", ["bf16", "f16"])
@pytest.mark.parametrize("r", [1, 2, 4])
def test_mirror_16bit_step_is_rounded_f32_step(dt, r):
    # One 16-bit-storage step = RN16(FP32 mirror step on the widened inputs).
    code = oracle.DTYPES[dt]
    ny, nx = 21, 34
    up = inputs.to_storage(inputs.random_field(1, ny, nx).astype(np.float64), dt)
    uc = inputs.to_storage(inputs.random_field(2, ny, nx).astype(np.float64), dt)
    wide = lambda a: oracle.storage_to_f64(a, code).astype(np.float32)
    got = oracle.wave_step_mirror(code, up, uc, r, 0.25)
    f32 = oracle.wave_step_mirror(oracle.F32, wide(up), wide(uc), r, 0.25)
    want = inputs.to_storage(f32.astype(np.float64), dt)
    assert np.array_equal(got, want)
    got_s = oracle.wave_start_mirror(code, uc, r, 0.25)
    want_s = inputs.to_storage(oracle.wave_start_mirror(oracle.F32, wide(uc), r, 0.25).astype(np.float64), dt)
    assert np.array_equal(got_s, want_s)


def test_f16_widening_exact():
    allbits = np.arange(65536, dtype=np.uint32).astype(np.uint16)
    finite = (allbits & 0x7C00) != 0x7C00
    want = allbits.view(np.float16).astype(np.float64)
    got = oracle.f16_bits_to_f64_fast(allbits)
    assert np.array_equal(got[finite], want[finite])


# --- 7. MLP ------------------------------------------------------------------------

def _mlp_case(B=7, F=5, H=6, O=2, seed=3):
    P = oracle.mlp_param_count(F, H, O)
    p = inputs.uniform_pm1_f32(seed, P).astype(np.float64) * 0.7
    X = inputs.uniform_pm1_f32(seed + 1, B * F).astype(np.float64).reshape(B, F)
    T = inputs.uniform_pm1_f32(seed + 2, B * O).astype(np.float64).reshape(B, O)
    return p, X, T, (F, H, O)


def test_mlp_param_count():
    assert oracle.mlp_param_count(10, 64, 2) == 10 * 64 + 64 + 64 * 64 + 64 + 2 * 64 + 2


def test_mlp_gradient_central_differences():
    p, X, T, (F, H, O) = _mlp_case()
    loss, g = oracle.mlp_loss_grad(X, T, p, F, H, O)
    fd = np.empty_like(p)
    h = 1e-6
    for i in range(p.size):
        e = np.zeros_like(p)
        e[i] = h
        lp, _ = oracle.mlp_loss_grad(X, T, p + e, F, H, O)
        lm, _ = oracle.mlp_loss_grad(X, T, p - e, F, H, O)
        fd[i] = (lp - lm) / (2 * h)
    assert np.max(np.abs(g - fd)) <= 1e-7 * max(1.0, np.max(np.abs(g)))
    # loss is the mean squared error of the forward outputs
    Y = oracle.mlp_forward(X, p, F, H, O)
    assert abs(loss - np.mean((Y - T) ** 2)) <= 1e-15 * max(1.0, loss)


def test_mlp_forward_special_cases():
    F, H, O = 1, 1, 1
    # W1 = 1, b1 = 0, W2 = 1, b2 = 0, W3 = 1, b3 = 0  ->  y = silu(silu(x))
    p = np.array([1.0, 0.0, 1.0, 0.0, 1.0, 0.0])
    xs = np.array([[-3.0], [-0.5], [0.0], [0.7], [4.0]])
    silu = lambda z: z / (1.0 + math.exp(-z))
    Y = oracle.mlp_forward(xs, p, F, H, O)
    for x, y in zip(xs[:, 0], Y[:, 0]):
        assert abs(y - silu(silu(x))) <= 1e-15
    # all weights zero -> output is b3
    F, H, O = 4, 8, 2
    P = oracle.mlp_param_count(F, H, O)
    p = np.zeros(P)
    p[-2:] = [0.25, -3.0]
    Y = oracle.mlp_forward(np.ones((3, F)), p, F, H, O)
    assert np.array_equal(Y, np.tile([0.25, -3.0], (3, 1)))


def test_adam_constant_gradient_closed_form():
    # With a constant gradient g the bias-corrected moments are exactly g and g^2, so
    # every step moves each parameter by -lr * g / (|g| + eps).
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    p = np.zeros(4)
    m, v = np.zeros(4), np.zeros(4)
    lr, eps = 1e-2, 1e-8
    for t in range(1, 6):
        oracle.adam_step(p, g, m, v, t, lr, 0.9, 0.999, eps)
        np.testing.assert_allclose(p, -t * lr * g / (np.abs(g) + eps), rtol=1e-12, atol=1e-18)


def test_oracle_results_do_not_depend_on_the_thread_count():
    # every output point is computed independently, so 1 thread and all threads give the same bits
    u0 = inputs.to_storage(inputs.gaussian_pulse(96, 130, 9.0) + 0.05 * inputs.random_field(71, 96, 130), "f32")
    u3 = inputs.to_storage(inputs.random_field_3d(72, 9, 20, 33).astype(np.float64), "bf16")
    x, y = inputs.saxpy_inputs(10007, seed=73)
    n0 = oracle.threads()
    try:
        runs = []
        for n in (1, max(2, n0)):
            oracle.set_threads(n)
            runs.append((oracle.wave_run_mirror(oracle.F32, u0, 9, 2, 0.25), oracle.wave_run_f64(u0.astype(np.float64), 9, 2, 0.25),
                         oracle.wave3d_run_mirror(oracle.BF16, u3, 4, 1, 0.125), oracle.saxpy_f32(2.5, x, y)))
    finally:
        oracle.set_threads(n0)
    (m1, f1, t1, s1), (m2, f2, t2, s2) = runs
    for a, b in [(m1[0], m2[0]), (m1[1], m2[1]), (f1[1], f2[1]), (t1[1], t2[1]), (s1, s2)]:
        assert np.array_equal(np.asarray(a).view(np.uint8), np.asarray(b).view(np.uint8))
