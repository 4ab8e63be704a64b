"""Writes precision_error_8192.txt: the error of each storage type's precision
mirror against the FP64 oracle on the 2D wave workload, computed by the oracle
alone (no GPU, nothing of the product's arithmetic).

Workload: 8192 x 8192 grid, Gaussian pulse (sigma = 64 cells, amplitude 1) at the
centre, c2 = (c dt/dx)^2 = 0.25, radius 1, Taylor start and 200 leapfrog steps,
Dirichlet-zero ghosts.  The value of a point after n steps depends only on the
initial values within (n + 1) r cells of it (the light cone), so both oracles run
on the central (2H + 1)^2 box grown by that cone, and their values on the central
box equal those of the whole grid.  Error measures on the central box (H = 500):
max |u - u64|, that over max |u64|, and the L2-relative error; plus the relative
drift of the discrete energy E^{n+1/2} = sum (u^{n+1} - u^n)^2 - c2 sum u^{n+1} L u^n
from (u^0, u^{-1}) to (u^200, u^199), over the whole grown box (the points outside
it hold the pulse's tail below 1e-25, which does not show in E).

Run from the repository root:  python tests/golden/make_precision_error.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2505_06022_gb300 import inputs  # noqa: E402  (seeded inputs only)

N, STEPS, R, C2, SIGMA, H = 8192, 200, 1, 0.25, 64.0, 500
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "precision_error_8192.txt")


def measure() -> dict:
    cone = (STEPS + 1) * R + 1
    c = N // 2
    lo, hi = c - H - cone, c + H + cone + 1
    u64 = inputs.gaussian_pulse(N, N, SIGMA)[lo:hi, lo:hi].copy()
    _, ref_full = oracle.wave_run_f64(u64, STEPS, R, C2)
    ref = ref_full[cone:cone + 2 * H + 1, cone:cone + 2 * H + 1]
    out = {}
    for name, code in oracle.DTYPES.items():
        u0 = inputs.to_storage(inputs.gaussian_pulse(N, N, SIGMA), name)[lo:hi, lo:hi].copy()
        um1 = oracle.wave_start_mirror(code, u0, R, C2)
        prev, cur = oracle.wave_run_mirror(code, u0, STEPS, R, C2)
        w = lambda a: oracle.storage_to_f64(a, code)  # noqa: E731
        d = w(cur)[cone:cone + 2 * H + 1, cone:cone + 2 * H + 1] - ref
        e0 = oracle.wave_energy_f64(w(u0), w(um1), R, C2)["E"]
        e1 = oracle.wave_energy_f64(w(cur), w(prev), R, C2)["E"]
        out[name] = {"max_abs": float(np.max(np.abs(d))),
                     "max_rel": float(np.max(np.abs(d)) / np.max(np.abs(ref))),
                     "l2_rel": float(np.sqrt(np.sum(d * d) / np.sum(ref * ref))),
                     "energy_drift": float((e1 - e0) / e0)}
    return out


def write(values: dict, path: str = OUT) -> None:
    with open(path, "w") as f:
        f.write("# Error of the precision mirror against the FP64 oracle, 2D wave, 8192^2, sigma 64,\n"
                "# c2 0.25, radius 1, 200 steps; central 1001^2 box; energy drift over the run.\n"
                "# Written by tests/golden/make_precision_error.py (the oracle only).\n"
                "# format: storage max_abs max_rel l2_rel energy_drift\n")
        for name in ("f32", "bf16", "f16"):
            v = values[name]
            f.write(f"{name} {v['max_abs']!r} {v['max_rel']!r} {v['l2_rel']!r} {v['energy_drift']!r}\n")


def read(path: str = OUT) -> dict:
    out = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        name, *vals = line.split()
        out[name] = dict(zip(("max_abs", "max_rel", "l2_rel", "energy_drift"), map(float, vals)))
    return out


if __name__ == "__main__":
    write(measure())
    print(open(OUT).read())
