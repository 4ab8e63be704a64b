"""The oracle's pins are strong enough to catch plausible mistakes.

Each case plants one mistake (a dropped term, a wrong sign, a shifted index, a
transposed operand, a wrong weight, a wrong rounding) into a copy of oracle.c,
compiles it on the CPU into a temporary library, and runs the relevant pin
checks against it: at least one must fail.  The real oracle is untouched."""
import ctypes as C
import math
import os
import subprocess

import numpy as np
import pytest

from paper_2505_06022_gb300 import inputs

ORACLE_C = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "oracle.c")

MUTATIONS = {
    "saxpy_add_to_sub": ("z[i] = ax + y[i];", "z[i] = ax - y[i];"),
    "stencil_drop_horizontal": ("acc = acc + w[k] * (vert + horz);", "acc = acc + w[k] * vert;"),
    "stencil_shift_index": ("ghost64(u, ny, nx, i + k, j)", "ghost64(u, ny, nx, i + k - 1 + 1 * (k > 1), j)"),
    "stencil_transpose": ("ghost64(u, ny, nx, i, j - k) + ghost64(u, ny, nx, i, j + k)",
                          "ghost64(u, ny, nx, j - k, i) + ghost64(u, ny, nx, j + k, i)"),
    "stencil_wrong_sign": ("(2.0 * u - u_prev[i * nx + j]) + c2 * lap64", "(2.0 * u - u_prev[i * nx + j]) - c2 * lap64"),
    "start_full_c2": ("(0.5 * c2) * lap64(u0", "c2 * lap64(u0"),
    "ghost_not_zero": ("return 0.0; /* Dirichlet-zero ghost */", "return u[((i + ny) % ny) * nx + ((j + nx) % nx)];"),
    "weight_formula": ("w[0] = -2.0 * sum;", "w[0] = -2.0 * sum + 1e-3;"),
    "mirror_fma_order": ("float inertia = two_u - up;", "float inertia = two_u - up + 0.0f * lap;\n            inertia = inertia + 1e-7f * up;"),
    "bf16_truncate": ("b += 0x7fffu + keep_lsb;", "b += 0;"),
    "f16_ties_away": ("double n = nearbyint(a / quantum);", "double n = floor(a / quantum + 0.5);"),
    "energy_sign": ("return kin - c2 * pot;", "return kin + c2 * pot;"),
    "mlp_grad_drop_silu": ("dz1[i] = s * silu_grad(z1[i]);", "dz1[i] = s;"),
    "wave3d_drop_depth": ("acc = acc + w[m] * ((vert + horz) + depth);", "acc = acc + w[m] * (vert + horz);"),
    "wave3d_centre_2w0": ("double acc = (3.0 * w[0]) * u[(k * ny + i) * nx + j];",
                          "double acc = (2.0 * w[0]) * u[(k * ny + i) * nx + j];"),
    "wave3d_depth_shift": ("ghost3(u, nz, ny, nx, k + m, i, j);", "ghost3(u, nz, ny, nx, k + m, i + 1, j);"),
    "mirror3d_drop_depth": ("float pair = plane + depth;", "float pair = plane;"),
    "rm_box_one_sided": ("                hi += radius[d];", "                hi += 0 * radius[d];"),
    "rm_transfers_no_clip": ("box[d] = need[d] > own[d] ? need[d] : own[d];", "box[d] = need[d];"),
}


def build_mutant(tmp_path, name):
    src = open(ORACLE_C).read()
    old, new = MUTATIONS[name]
    assert src.count(old) >= 1, f"mutation anchor for {name} not found"
    mutated = src.replace(old, new)
    path = tmp_path / f"{name}.c"
    path.write_text(mutated)
    lib = tmp_path / f"lib{name}.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", str(path),
                    "-o", str(lib), "-lm"], check=True, capture_output=True)
    L = C.CDLL(str(lib))
    return L


def _p(a):
    return a.ctypes.data


def pins_hold(L):
    """A compact re-run of the oracle pins against library L; False as soon as one fails."""
    i64, dbl, flt, vp = C.c_int64, C.c_double, C.c_float, C.c_void_p
    L.oracle_saxpy_f32.argtypes = [i64, flt, vp, vp, vp]
    L.oracle_wave_run_f64.argtypes = [i64, i64, C.c_int, dbl, i64, vp, vp, vp]
    L.oracle_wave_run_mirror.argtypes = [C.c_int, i64, i64, C.c_int, flt, i64, vp, vp, vp]
    L.oracle_wave_energy_f64.argtypes = [i64, i64, C.c_int, dbl, vp, vp, vp, vp, vp]
    L.oracle_wave_energy_f64.restype = dbl
    L.oracle_wave_step_f64.argtypes = [i64, i64, C.c_int, dbl, vp, vp, vp]
    L.oracle_d2_weights.argtypes = [C.c_int, vp]
    L.oracle_f32_to_bf16.argtypes = [flt]
    L.oracle_f32_to_bf16.restype = C.c_uint16
    L.oracle_f32_to_f16.argtypes = [flt]
    L.oracle_f32_to_f16.restype = C.c_uint16
    L.oracle_mlp_loss_grad.argtypes = [i64, C.c_int, C.c_int, C.c_int, vp, vp, vp, vp]
    L.oracle_mlp_loss_grad.restype = dbl
    L.oracle_wave3d_run_f64.argtypes = [i64, i64, i64, C.c_int, dbl, i64, vp, vp, vp]
    L.oracle_wave3d_run_mirror.argtypes = [C.c_int, i64, i64, i64, C.c_int, flt, i64, vp, vp, vp]
    L.oracle_rm_box.argtypes = [C.c_int, vp, C.c_int, vp, vp, vp, vp]
    L.oracle_rm_box_transfers.argtypes = [C.c_int, vp, C.c_int, vp, vp, C.c_int, vp, vp, C.c_int]

    # SAXPY: two single roundings
    x, y = inputs.saxpy_inputs(257, seed=0)
    z = np.empty_like(x)
    L.oracle_saxpy_f32(x.size, 2.5, _p(x), _p(y), _p(z))
    want = (np.float32(2.5) * x.astype(np.float64)).astype(np.float32).astype(np.float64) + y.astype(np.float64)
    if not np.array_equal(z, want.astype(np.float32)):
        return False
    # weights: Fornberg r = 2
    w = np.zeros(5)
    L.oracle_d2_weights(2, _p(w))
    if not np.allclose(w[:3], [-2.5, 4 / 3, -1 / 12], rtol=1e-15, atol=0):
        return False
    # closed-form standing wave, non-square grid
    ny, nx, mx, my, steps = 24, 37, 5, 3, 30
    u0 = inputs.sine_mode(ny, nx, mx, my)
    prev, cur = np.empty_like(u0), np.empty_like(u0)
    L.oracle_wave_run_f64(ny, nx, 1, 0.25, steps, _p(u0), _p(prev), _p(cur))
    ty, tx = math.pi * my / (ny + 1), math.pi * mx / (nx + 1)
    om = math.acos(1 - 2 * 0.25 * (math.sin(tx / 2) ** 2 + math.sin(ty / 2) ** 2))
    if np.max(np.abs(cur - math.cos(steps * om) * u0)) > 1e-12:
        return False
    # energy conservation for r = 3 (and the energy's own sign through E > 0)
    g = inputs.gaussian_pulse(20, 22, 2.5)
    um1, g_copy = np.empty_like(g), np.empty_like(g)  # keep both alive across the call
    L.oracle_wave_run_f64(20, 22, 3, 0.25, 0, _p(g), _p(um1), _p(g_copy))
    e = lambda a, b: L.oracle_wave_energy_f64(20, 22, 3, 0.25, _p(a), _p(b), None, None, None)
    E0 = e(g, um1)
    pv, cv = np.empty_like(g), np.empty_like(g)
    L.oracle_wave_run_f64(20, 22, 3, 0.25, 40, _p(g), _p(pv), _p(cv))
    E1 = e(cv, pv)
    if not (E0 > 0 and abs(E1 - E0) <= 1e-10 * abs(E0)):
        return False
    # FP32 mirror equals FP64 on an exact dyadic integer case
    iu = ((inputs.splitmix64(77, 15 * 13) % np.uint64(129)).astype(np.int64) - 64).astype(np.float64).reshape(15, 13)
    p64, c64 = np.empty_like(iu), np.empty_like(iu)
    L.oracle_wave_run_f64(15, 13, 1, 0.25, 3, _p(iu), _p(p64), _p(c64))
    i32 = iu.astype(np.float32)
    p32, c32 = np.empty_like(i32), np.empty_like(i32)
    L.oracle_wave_run_mirror(0, 15, 13, 1, 0.25, 3, _p(i32), _p(p32), _p(c32))
    if not np.array_equal(c32.astype(np.float64), c64):
        return False
    # 16-bit rounding against library conversions
    vals = np.array([1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -11, 1.0 + 3 * 2 ** -11, 3.0e-6, 65519.0, -2.5e-5],
                    np.float32)
    for v in vals:
        if L.oracle_f32_to_f16(float(v)) != int(np.float16(v).view(np.uint16)):
            return False
    import torch

    for v in vals:
        want_b = int(torch.tensor([float(v)], dtype=torch.float32).to(torch.bfloat16).view(torch.int16).item()) & 0xFFFF
        if L.oracle_f32_to_bf16(float(v)) != want_b:
            return False
    # 3D: closed-form separable mode (r = 1) and the dense Kronecker operator (r = 2)
    shape = (7, 8, 9)
    u3 = inputs.sine_mode_3d(*shape, 2, 3, 4)
    p3, c3 = np.empty_like(u3), np.empty_like(u3)
    L.oracle_wave3d_run_f64(*shape, 1, 0.125, 12, _p(u3), _p(p3), _p(c3))
    s2 = sum(math.sin(math.pi * m / (n + 1) / 2) ** 2 for n, m in zip(shape, (2, 3, 4)))
    if np.max(np.abs(c3 - math.cos(12 * math.acos(1 - 0.25 * s2)) * u3)) > 1e-12:
        return False
    from test_oracle_pins_3d import kron3

    shape = (4, 5, 3)
    r3 = inputs.random_field_3d(5, *shape).astype(np.float64)
    K = kron3(*shape, 2)
    a, b = r3.reshape(-1) + 0.0625 * (K @ r3.reshape(-1)), r3.reshape(-1).copy()
    for _ in range(6):
        a, b = b, 2 * b - a + 0.125 * (K @ b)
    p3, c3 = np.empty_like(r3), np.empty_like(r3)
    L.oracle_wave3d_run_f64(*shape, 2, 0.125, 6, _p(r3), _p(p3), _p(c3))
    if np.max(np.abs(c3.reshape(-1) - b)) > 1e-12 * max(1.0, np.max(np.abs(b))):
        return False
    # 3D mirror: exact on dyadic integers
    iz = ((inputs.splitmix64(91, 5 * 6 * 7) % np.uint64(129)).astype(np.int64) - 64).astype(np.float64)
    iz = iz.reshape(5, 6, 7)
    p64, c64 = np.empty_like(iz), np.empty_like(iz)
    L.oracle_wave3d_run_f64(5, 6, 7, 1, 0.125, 3, _p(iz), _p(p64), _p(c64))
    i32 = iz.astype(np.float32)
    p32, c32 = np.empty_like(i32), np.empty_like(i32)
    L.oracle_wave3d_run_mirror(0, 5, 6, 7, 1, 0.125, 3, _p(i32), _p(p32), _p(c32))
    if not np.array_equal(c32.astype(np.float64), c64):
        return False
    # box range mappers and transfers against enumerated cells
    from test_oracle_pins_3d import brute_required, cells

    ext = np.array([6, 5, 7], np.int64)
    rad = np.array([1, 2, 1], np.int64)
    fx = np.zeros(6, np.int64)
    chunk = np.array([2, 1, 3, 4, 3, 5], np.int64)
    out = np.zeros(6, np.int64)
    L.oracle_rm_box(1, _p(rad), 0, _p(fx), _p(chunk), _p(ext), _p(out))
    box = ((int(out[0]), int(out[1]), int(out[2])), (int(out[3]), int(out[4]), int(out[5])))
    if cells(box) != brute_required(1, ((2, 1, 3), (4, 3, 5)), (6, 5, 7), (1, 2, 1), 0, None):
        return False
    chunks = [((0, 0, 0), (3, 5, 7)), ((3, 0, 0), (6, 5, 7))]
    flat = np.array([v for c in chunks for part in c for v in part], np.int64)
    recs = np.zeros(8 * 4, np.int64)
    n = L.oracle_rm_box_transfers(1, _p(rad), 0, _p(fx), _p(flat), 2, _p(ext), _p(recs), 4)
    got = set()
    for t in range(max(n, 0)):
        src, dst, b6 = int(recs[8 * t]), int(recs[8 * t + 1]), recs[8 * t + 2: 8 * t + 8]
        bx = ((int(b6[0]), int(b6[1]), int(b6[2])), (int(b6[3]), int(b6[4]), int(b6[5])))
        if not cells(bx) <= cells(chunks[src]):
            return False
        got |= {(dst, p) for p in cells(bx)}
    want = {(d, p) for d, ch in enumerate(chunks)
            for p in brute_required(1, ch, (6, 5, 7), (1, 2, 1), 0, None) - cells(ch)}
    if got != want:
        return False
    # MLP gradient against central differences (first-layer weights, where the mutation bites)
    F, H, O, B = 3, 4, 2, 5
    P = H * F + H + H * H + H + O * H + O
    prm = inputs.uniform_pm1_f32(3, P).astype(np.float64) * 0.7
    X = inputs.uniform_pm1_f32(4, B * F).astype(np.float64).reshape(B, F)
    T = inputs.uniform_pm1_f32(5, B * O).astype(np.float64).reshape(B, O)
    grad = np.empty(P)
    L.oracle_mlp_loss_grad(B, F, H, O, _p(X), _p(T), _p(prm), _p(grad))
    h = 1e-6
    for i in range(H * F):
        e_ = np.zeros(P)
        e_[i] = h
        gp, gm = np.empty(P), np.empty(P)
        pp, pm = prm + e_, prm - e_  # named: the C call needs them alive
        lp = L.oracle_mlp_loss_grad(B, F, H, O, _p(X), _p(T), _p(pp), _p(gp))
        lm = L.oracle_mlp_loss_grad(B, F, H, O, _p(X), _p(T), _p(pm), _p(gm))
        if abs((lp - lm) / (2 * h) - grad[i]) > 1e-7 * max(1.0, np.max(np.abs(grad))):
            return False
    return True


def test_unmutated_copy_passes_the_pins(tmp_path):
    src = open(ORACLE_C).read()
    path = tmp_path / "same.c"
    path.write_text(src)
    lib = tmp_path / "libsame.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", str(path),
                    "-o", str(lib), "-lm"], check=True, capture_output=True)
    assert pins_hold(C.CDLL(str(lib)))


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(tmp_path, name):
    assert not pins_hold(build_mutant(tmp_path, name)), f"planted mistake {name} passed every pin"
