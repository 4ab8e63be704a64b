"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds the random-number generator and the initial fields only; it
contains none of the method's arithmetic (no SAXPY, no stencil, no energy).  Both
sides of every parity test receive the arrays made here, generated once on the
host and uploaded, so their inputs are bit-identical.

Generator: splitmix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014).  It is counter-based: the k-th output (k = 0, 1, ...)
of the stream with state s is mix(s + (k+1) * 0x9E3779B97F4A7C15) with the
published mixing function, so any element can be produced independently.
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(state: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs offset .. offset+n-1 of the splitmix64 stream with the given state."""
    k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(state & 0xFFFFFFFFFFFFFFFF) + k * GOLDEN_GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_pm1_f32(state: int, n: int) -> np.ndarray:
    """n values in [-1, 1): u = (z >> 40) * 2^-24 in [0, 1), value = 2u - 1.

    Each value is m / 2^23 - 1 for a 24-bit integer m, so it is exact in FP32."""
    m = (splitmix64(state, n) >> np.uint64(40)).astype(np.int64)
    return ((m - (1 << 23)).astype(np.float64) / float(1 << 23)).astype(np.float32)


def uniform01_f64(state: int, n: int, offset: int = 0) -> np.ndarray:
    """n values in [0, 1) with 53 random bits: (z >> 11) * 2^-53."""
    return (splitmix64(state, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def saxpy_inputs(n: int, seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """x from the stream with state 2*seed, y from state 2*seed+1 (element k = k-th output)."""
    return uniform_pm1_f32(2 * seed, n), uniform_pm1_f32(2 * seed + 1, n)


def gaussian_pulse(ny: int, nx: int, sigma: float, amplitude: float = 1.0) -> np.ndarray:
    """u0[i, j] = A * g(i - ny//2) * g(j - nx//2), g(d) = exp(-d^2 / (2 sigma^2)), in FP64.

    The pulse is centred on the integer index (ny//2, nx//2); the product of two
    1D Gaussians equals the 2D Gaussian exp(-r^2/(2 sigma^2)) up to FP64 rounding."""
    gy = np.exp(-((np.arange(ny, dtype=np.float64) - ny // 2) ** 2) / (2.0 * sigma * sigma))
    gx = np.exp(-((np.arange(nx, dtype=np.float64) - nx // 2) ** 2) / (2.0 * sigma * sigma))
    return amplitude * np.outer(gy, gx)


def sine_mode(ny: int, nx: int, mx: int, my: int) -> np.ndarray:
    """u0[i, j] = sin(pi*my*(i+1)/(ny+1)) * sin(pi*mx*(j+1)/(nx+1)), in FP64."""
    sy = np.sin(math.pi * my * np.arange(1, ny + 1, dtype=np.float64) / (ny + 1))
    sx = np.sin(math.pi * mx * np.arange(1, nx + 1, dtype=np.float64) / (nx + 1))
    return np.outer(sy, sx)


def random_field(state: int, ny: int, nx: int) -> np.ndarray:
    """Uniform [-1, 1) FP32 field (exact values), for operator-level tests."""
    return uniform_pm1_f32(state, ny * nx).reshape(ny, nx)


def gaussian_pulse_3d(nz: int, ny: int, nx: int, sigma: float, amplitude: float = 1.0) -> np.ndarray:
    """u0[k, i, j] = A * g(k - nz//2) * g(i - ny//2) * g(j - nx//2), g as in gaussian_pulse, FP64."""
    g = [np.exp(-((np.arange(n, dtype=np.float64) - n // 2) ** 2) / (2.0 * sigma * sigma)) for n in (nz, ny, nx)]
    return amplitude * g[0][:, None, None] * g[1][None, :, None] * g[2][None, None, :]


def sine_mode_3d(nz: int, ny: int, nx: int, mz: int, my: int, mx: int) -> np.ndarray:
    """u0[k, i, j] = sin(pi*mz*(k+1)/(nz+1)) sin(pi*my*(i+1)/(ny+1)) sin(pi*mx*(j+1)/(nx+1)), FP64."""
    s = [np.sin(math.pi * m * np.arange(1, n + 1, dtype=np.float64) / (n + 1)) for n, m in ((nz, mz), (ny, my),
                                                                                           (nx, mx))]
    return s[0][:, None, None] * s[1][None, :, None] * s[2][None, None, :]


def random_field_3d(state: int, nz: int, ny: int, nx: int) -> np.ndarray:
    """Uniform [-1, 1) FP32 field (exact values) of shape (nz, ny, nx)."""
    return uniform_pm1_f32(state, nz * ny * nx).reshape(nz, ny, nx)


def to_storage(a64: np.ndarray, dtype: str) -> np.ndarray:
    """Round an FP64 field to its storage format: FP32 (float32 array), or BF16 /
    FP16 bit patterns (uint16 array).  16-bit values are rounded from the FP32
    value with round-to-nearest-even (torch / numpy conversions)."""
    f32 = np.ascontiguousarray(a64, dtype=np.float32)
    if dtype == "f32":
        return f32
    if dtype == "f16":
        return f32.astype(np.float16).view(np.uint16)
    if dtype == "bf16":
        import torch

        return torch.from_numpy(f32).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16).copy()
    raise ValueError(f"unknown storage dtype {dtype!r}")


def batch_grids(count: int = 64, seed: int = 1, side_lo: int = 256, side_hi: int = 4096,
                radii: tuple[int, ...] = (1, 2, 4)) -> list[tuple[int, int, int]]:
    """(H, W, r) for `count` independent grids.

    Per grid three consecutive outputs of the stream with state `seed`: H and W are
    round(exp(U(ln lo, ln hi))) (log-uniform), r = radii[z mod len(radii)]."""
    z = splitmix64(seed, 3 * count)
    out = []
    lo, hi = math.log(side_lo), math.log(side_hi)
    for g in range(count):
        uh = float(z[3 * g] >> np.uint64(11)) * 2.0 ** -53
        uw = float(z[3 * g + 1] >> np.uint64(11)) * 2.0 ** -53
        H = int(round(math.exp(lo + (hi - lo) * uh)))
        W = int(round(math.exp(lo + (hi - lo) * uw)))
        r = radii[int(z[3 * g + 2] % np.uint64(len(radii)))]
        out.append((H, W, r))
    return out


def batch_initial(H: int, W: int, dtype: str = "f32") -> np.ndarray:
    """Initial field of one batched grid: centred Gaussian with sigma = min(H, W) / 16."""
    return to_storage(gaussian_pulse(H, W, min(H, W) / 16.0), dtype)


def cost_corpus_shapes(seed: int = 4, n_stencil: int = 560, n_saxpy: int = 40, side_lo: int = 512,
                       side_hi: int = 16384, n_lo: int = 1 << 16, n_hi: int = 1 << 28) -> list[dict]:
    """Synthetic kernel corpus for the cost model.

    Stencils: sides ny, nx log-uniform in [side_lo, side_hi] (independent), radius
    uniform in 1..4, storage FP32 or BF16 with equal odds.  SAXPY: n log-uniform in
    [n_lo, n_hi].  Five consecutive outputs of the stream with state `seed` per shape."""
    z = splitmix64(seed, 5 * (n_stencil + n_saxpy))
    u = (z >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    out = []
    lo, hi = math.log(side_lo), math.log(side_hi)
    for s in range(n_stencil):
        uy, ux, ur, ud = u[5 * s], u[5 * s + 1], u[5 * s + 2], u[5 * s + 3]
        out.append({"kind": 1, "ny": int(round(math.exp(lo + (hi - lo) * uy))),
                    "nx": int(round(math.exp(lo + (hi - lo) * ux))), "radius": 1 + int(ur * 4),
                    "dtype": "f32" if ud < 0.5 else "bf16"})
    nlo, nhi = math.log(n_lo), math.log(n_hi)
    for s in range(n_stencil, n_stencil + n_saxpy):
        out.append({"kind": 0, "n": int(round(math.exp(nlo + (nhi - nlo) * u[5 * s]))), "dtype": "f32"})
    return out
