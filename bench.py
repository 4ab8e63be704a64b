#!/usr/bin/env python3
"""Benchmark of the hot path: the 2D leapfrog wave stencil, FP32, 8192 x 8192,
200 steps, split into 4 row chunks with a radius-1 neighbourhood halo, every
chunk launch timed by device-side timestamps and energy-attributed (NVML).

One bench "step" = one whole simulation: the Taylor start plus 200 leapfrog
steps over the 4 chunks (804 kernel launches, one sy_wave_run call replaying its
CUDA graph), from the initial field already resident in HBM.  Units: grid-point updates (200 * 8192^2 per step).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl sy|reference]

Prints ONE JSON line (rank 0).  With N > 1 (torchrun), every rank runs an
independent replica on its own GPU (the single-GPU chunk split keeps the
paper's semantics; the cross-GPU halo exchange is not exercised here), and
`value` is the updates of all ranks / the slowest rank's time ("weak" scaling).

`--impl reference` times the CPU oracle (the FP32 precision mirror, the same
arithmetic as the GPU path) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NY = NX = 8192
STEPS = 200
CHUNKS = 4
RADIUS = 1
HALO = 1
C2 = 0.25
SIGMA = 64.0
BYTES_PER_UPDATE = 12  # read u^n and u^{n-1}, write u^{n+1} (FP32; 6 for 16-bit storage)
METRIC = "stencil GB/s & updates/s (fraction of HBM peak), J/update; learned/batched vs plain"
WORKLOAD = ("wave2d leapfrog 5-point FP32, 8192x8192, c*dt/dx=0.5, 200 steps, Dirichlet-zero, "
            "Gaussian sigma=64 at centre, 4 row chunks, halo radius 1")


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "source": "fallback"}


def device_info(index: int) -> dict:
    """GPU name, driver version and the host's core count, for the record."""
    import torch

    info = {"name": torch.cuda.get_device_name(index), "host_cores": os.cpu_count()}
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(index), "--query-gpu=driver_version,memory.total",
                              "--format=csv,noheader"], capture_output=True, text=True, timeout=20).stdout.strip()
        driver, mem = [v.strip() for v in out.split(",")[:2]]
        info.update({"driver": driver, "memory_total": mem})
    except Exception:
        pass
    return info


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class ClockSampler:
    """nvidia-smi samples of SM clock, power and throttle reasons; stop(window) keeps the
    samples taken inside the timed region (host wall-clock window), where there are any."""

    # power.draw.instant: the instantaneous reading (power.draw averages over about a second,
    # longer than the benchmark's timed region)
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw.instant,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "50", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    @staticmethod
    def parse(lines, window=None) -> dict:
        """Summary of nvidia-smi CSV lines (FIELDS order); with window = (t0, t1) in host
        epoch seconds, only the samples inside it count, unless none falls inside."""
        import datetime

        rows = []
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                t = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                t = None
            try:
                rows.append((t, float(parts[2]), float(parts[3]), float(parts[4]), parts[6:10]))
            except ValueError:
                continue
        inside = [r for r in rows if window and r[0] is not None and window[0] <= r[0] <= window[1]]
        used = inside or rows
        if not used:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in used for n, v in zip(names, r[4]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[1] for r in used), "sm_max_mhz": max(r[2] for r in used),
                "reasons": reasons, "samples": len(used), "samples_in_timed_region": len(inside),
                "power_w_median": statistics.median(r[3] for r in used)}

    def stop(self, window=None) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self._t.join(timeout=2)
        return self.parse(self.lines, window)


def kernel_source_sha() -> str:
    h = hashlib.sha256()
    for name in ("wave_kernel.cuh", "wave.cu", "wave_f32.cu", "stamp.cuh"):
        with open(os.path.join(ROOT, "paper_2505_06022_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def kernel_label(dtype: str, variant: int = 0) -> str:
    """The dominant kernel of the timed step: the 2D step's variant for this storage type
    (the default unless one is asked for; 16-bit radius-1 4-row tiles run the 96-register form,
    16-bit radius 3-4 8-row tiles of 128 threads the 168-register form)."""
    import paper_2505_06022_gb300 as sy

    code = sy.DTYPE_CODES[dtype]
    v = variant or sy.sy_stencil_default_variant(RADIUS, code)
    rows, _, threads = sy.sy_stencil_variant_info(RADIUS, code, v)
    if dtype != "f32" and v == 15:
        return f"wave_march_kernel<{dtype},{RADIUS}> x {threads} threads, one 2048x8192 chunk per launch"
    if v >= 13:
        name = "wave_hln_kernel"
    elif v >= 9:
        name = "wave_hl_kernel_b3" if dtype != "f32" and RADIUS >= 3 and rows == 8 and threads == 128 \
            else "wave_hl_kernel"
    elif dtype != "f32" and RADIUS == 1 and rows == 4:
        name = "wave_vec_kernel_r96"
    elif dtype != "f32" and RADIUS >= 3 and rows == 8 and threads == 128:
        name = "wave_vec_kernel_b3"
    else:
        name = "wave_vec_kernel"
    return f"{name}<{dtype},{RADIUS},{rows},false> x {threads} threads, one 2048x8192 chunk per launch"


def ncu_traffic() -> float | None:
    """Per-launch DRAM bytes of the wave kernel from the committed ncu summary, if
    it was captured from the current kernel source."""
    path = os.path.join(ROOT, "profiles", "wave_f32_8192_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        if d.get("source_sha") == kernel_source_sha():
            return float(d["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


# ---------------------------------------------------------------------------
# CPU oracle leg (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------

def oracle_sample(seconds: float = 10.0) -> dict:
    """FP32 mirror of the oracle on full-width row bands of the same field, steps
    repeated until about `seconds` of CPU work; returns updates/s."""
    import numpy as np

    import oracle
    from paper_2505_06022_gb300 import inputs

    rows = 512
    u = inputs.to_storage(inputs.gaussian_pulse(NY, NX, SIGMA)[NY // 2 - rows // 2: NY // 2 + rows // 2], "f32")
    prev = oracle.wave_start_mirror(oracle.F32, u, RADIUS, C2)
    cur = u
    steps, t0 = 0, time.perf_counter()
    while True:
        nxt = oracle.wave_step_mirror(oracle.F32, prev, cur, RADIUS, C2)
        prev, cur = cur, nxt
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    upd = steps * rows * NX
    return {"value": upd / el, "unit": "updates/s", "cores": oracle.threads(), "kind": "oracle",
            "sample": f"FP32 mirror oracle, {rows}x{NX} rows of the 8192^2 Gaussian field, {steps} steps "
                      f"({upd:.3g} updates, {el:.1f} s)", "seconds": el, "updates": upd}


def run_reference(args) -> None:
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle

    per = max(2.0, min(20.0, 60.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_sample(per / 4)
    vals = [oracle_sample(per) for _ in range(args.steps)]
    tot_upd = sum(v["updates"] for v in vals)
    tot_s = sum(v["seconds"] for v in vals)
    value = tot_upd / tot_s
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": vals[0]["sample"]},
        "cpu_baseline": {"value": value, "unit": "updates/s", "cores": oracle.threads(), "kind": "oracle",
                         "sample": f"each step: {vals[0]['sample']}"},
        "e2e": {"value": value, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# The other forms of the path, each against the plain form on the same GPU
# ---------------------------------------------------------------------------

def _metered(q, stream, fn, min_seconds: float = 1.0, min_reps: int = 3):
    """Run fn() repeatedly for >= min_seconds inside one NVML metering window;
    returns (reps, device ms per rep, joules or None)."""
    import torch

    import paper_2505_06022_gb300 as sy

    torch.cuda.synchronize()
    try:
        sy.sy_meter_begin(q.handle)
        metered = True
    except sy.SyError:
        metered = False
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps, t0 = 0, time.perf_counter()
    e0.record(stream)
    while reps < min_reps or time.perf_counter() - t0 < min_seconds:
        fn()
        reps += 1
        if reps % 4 == 0:
            torch.cuda.synchronize()
    e1.record(stream)
    torch.cuda.synchronize()
    joules = None
    if metered:
        try:
            joules, _ = sy.sy_meter_end(q.handle)
        except sy.SyError:
            joules = None
    return reps, e0.elapsed_time(e1) / reps, joules


_F64_CORE = None


def f64_core() -> tuple:
    """The FP64 oracle's u^200 on the central (2H+1)^2 points of the 8192^2 Gaussian workload,
    H = 500: run on the box grown by the light cone ((STEPS + 1) * RADIUS + 1 cells), which
    makes the inner values exact.  Outside that region the field is the Gaussian's tail and the
    dispersive fringe of the pulse, ~1e-9 (reported as max_abs_u_outside, a bound on the error
    there together with the oracle's equally small values).  Returns (values, (y0, x0))."""
    global _F64_CORE
    if _F64_CORE is None:
        import oracle
        from paper_2505_06022_gb300 import inputs

        H, cone = 500, (STEPS + 1) * RADIUS + 1
        c = NY // 2
        lo, hi = c - H - cone, c + H + cone + 1
        u64 = inputs.gaussian_pulse(NY, NX, SIGMA)[lo:hi, lo:hi].copy()
        _, cur = oracle.wave_run_f64(u64, STEPS, RADIUS, C2)
        _F64_CORE = (cur[cone: cone + 2 * H + 1, cone: cone + 2 * H + 1].copy(), (c - H, c - H))
    return _F64_CORE


def error_vs_f64(got64) -> dict:
    """Max-abs, max-relative (to max |u_64|) and L2-relative error of a final 8192^2 field
    against the FP64 oracle on the central region; plus the largest |u| outside it."""
    import numpy as np

    ref, (y0, x0) = f64_core()
    n = ref.shape[0]
    d = got64[y0: y0 + n, x0: x0 + n] - ref
    outside = np.abs(got64.copy())
    outside[y0: y0 + n, x0: x0 + n] = 0.0
    return {"region": f"central {n}x{n} points (the FP64 oracle on the light-cone-grown box)",
            "max_abs": float(np.max(np.abs(d))), "max_rel": float(np.max(np.abs(d)) / np.max(np.abs(ref))),
            "l2_rel": float(np.sqrt(np.sum(d * d) / np.sum(ref * ref))),
            "max_abs_u_outside": float(np.max(outside))}


def measure_precision_form(q, stream, dtype: str) -> dict:
    """8192^2 Gaussian, 200 steps, 4 chunks, with `dtype` storage: throughput, J/update,
    max-abs / max-relative / L2 error against the FP64 oracle, discrete-energy drift."""
    import numpy as np
    import torch

    import oracle
    import paper_2505_06022_gb300 as sy
    from paper_2505_06022_gb300 import inputs

    p = sy.stencil_params(NY, NX, RADIUS, C2, dtype)
    chunks = sy.sy_split_rows(NY, CHUNKS)
    u64 = inputs.gaussian_pulse(NY, NX, SIGMA)
    host = inputs.to_storage(u64, dtype)
    u0 = torch.from_numpy(host if dtype == "f32" else host.view(np.int16)).cuda()
    A, B = torch.empty_like(u0), torch.empty_like(u0)
    byptr = {u0.data_ptr(): u0, A.data_ptr(): A, B.data_ptr(): B}
    # energy at the start: E(u^0, u^{-1})
    pv, cv, _ = sy.sy_wave_run(q.handle, p, u0, A, B, 0, chunks, HALO)
    E0 = sy.sy_wave_energy(q.handle, p, byptr[cv], byptr[pv])[0]
    run = lambda: sy.sy_wave_run(q.handle, p, u0, A, B, STEPS, chunks, HALO)
    run()
    reps, ms, joules = _metered(q, stream, run)
    pv, cv, _ = run()
    torch.cuda.synchronize()
    E1 = sy.sy_wave_energy(q.handle, p, byptr[cv], byptr[pv])[0]
    got = byptr[cv].cpu().numpy()
    got = got.astype(np.float64) if dtype == "f32" else oracle.storage_to_f64(got.view(np.uint16), oracle.DTYPES[dtype])
    err = error_vs_f64(got)
    esize = 4 if dtype == "f32" else 2
    upd = STEPS * NY * NX
    drift = (E1 - E0) / E0
    return {"dtype": dtype, "updates_per_s": upd / (ms * 1e-3), "gb_per_s": 3 * esize * upd / (ms * 1e-3) / 1e9,
            "ms_per_sim": ms, "j_per_update": None if not joules else joules / (reps * upd),
            "error_vs_f64": err, "energy_drift_rel": drift, **stated_accuracy(dtype, dict(err, energy_drift=drift))}


def stated_accuracy(dtype: str, errors: dict) -> dict:
    """tolerance_<measure> keys (the stored bounds of the accuracy module), whether every
    measured error is within them, and whether the storage type is usable on this workload."""
    from paper_2505_06022_gb300 import accuracy

    res = accuracy.check(dtype, errors)
    out = {f"tolerance_{k}": bound for k, (_, bound, _) in res.items()}
    out["within_tolerance"] = all(ok for (_, _, ok) in res.values())
    out["usable"] = accuracy.USABLE[dtype]
    return out


def measure_batched(q, stream) -> dict:
    """64 uneven grids (sides log-uniform in [256, 4096], seed 1, radius in {1, 2, 4}), 100 steps:
    one persistent launch per step in a CUDA graph (tile height tuned over {2, 4, 8}) against
    one launch per grid per step (in a CUDA graph, and from the host stream)."""
    import numpy as np
    import torch

    import paper_2505_06022_gb300 as sy
    from paper_2505_06022_gb300 import inputs

    shapes = inputs.batch_grids()
    steps = 100
    fields = []
    for ny, nx, r in shapes:
        pitch = (nx + 3) // 4 * 4
        ub = torch.zeros((ny, pitch), dtype=torch.float32, device="cuda")
        ub[:, :nx] = torch.from_numpy(inputs.batch_initial(ny, nx, "f32")).cuda()
        fields.append((ny, nx, pitch, r, torch.empty_like(ub), ub))
    points = sum(ny * nx for ny, nx, *_ in fields)
    upd = steps * points
    best = None
    modes_ms = {}
    for tile_rows in (0, 2, 4, 8):
        plan = sy.sy_stencil_batch_plan(q.handle, [(ny, nx, pitch, r, C2, ua, ub) for ny, nx, pitch, r, ua, ub
                                                   in fields], "f32", tile_rows)
        sy.sy_stencil_batch_start(plan)
        sy.sy_stencil_batch_capture(plan, steps)
        sy.sy_stencil_batch_run(plan)
        reps, ms, joules = _metered(q, stream, lambda: sy.sy_stencil_batch_run(plan), min_seconds=0.2)
        modes_ms[tile_rows] = ms
        if best is None or ms < best[1]:
            best = (tile_rows, ms, joules, reps)
        sy.sy_stencil_batch_destroy(plan)
    tile_rows, _, _, _ = best
    plan = sy.sy_stencil_batch_plan(q.handle, [(ny, nx, pitch, r, C2, ua, ub) for ny, nx, pitch, r, ua, ub
                                               in fields], "f32", tile_rows)
    sy.sy_stencil_batch_capture(plan, steps)
    sy.sy_stencil_batch_run(plan)
    l0 = q.launches
    sy.sy_stencil_batch_run(plan)
    batched_launches = q.launches - l0
    reps, ms, joules = _metered(q, stream, lambda: sy.sy_stencil_batch_run(plan))
    sy.sy_stencil_batch_destroy(plan)

    # the cross-step form: the whole run as one cooperative launch, a grid barrier per step
    plan = sy.sy_stencil_batch_plan(q.handle, [(ny, nx, pitch, r, C2, ua, ub) for ny, nx, pitch, r, ua, ub
                                               in fields], "f32", 0)
    sy.sy_stencil_batch_capture_persistent(plan, steps)
    sy.sy_stencil_batch_run(plan)
    reps_p, ms_p, joules_p = _metered(q, stream, lambda: sy.sy_stencil_batch_run(plan))
    sy.sy_queue_sync(q.handle)  # a barrier that gave up would show here
    sy.sy_stencil_batch_destroy(plan)

    # baseline: one launch per grid per step
    params = [(sy.stencil_params(ny, nx, r, C2, "f32", pitch=pitch), ua, ub, [(0, ny)], r)
              for ny, nx, pitch, r, ua, ub in fields]

    def per_grid_steps():
        for s in range(steps):
            for p, ua, ub, ch, r in params:
                prev, cur = (ua, ub) if s % 2 == 0 else (ub, ua)
                sy.sy_stencil_step(qg.handle, p, prev, cur, prev, ch, r)

    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        qg = sy.Queue(q.device, side)
        per_grid_steps()  # warm-up (and occupancy lookups) outside the capture
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=side):
        per_grid_steps()
    g.replay()
    reps_g, ms_g, joules_g = _metered(q, stream, g.replay)
    qs = sy.Queue(q.device, stream)
    qg_saved = qg
    qg = qs
    reps_s, ms_s, _ = _metered(q, stream, per_grid_steps, min_seconds=0.3, min_reps=2)
    qg = qg_saved
    qs.close()
    del g

    # Energy per update by radius class: each class's grids alone in a plan of their own
    # (>= 1 s metering window each), and the plain 8192^2 single field at the same radius
    # (4 chunks, 20 steps): the batch's J/update is the classes' update-weighted mix.
    per_class = {}
    for r in sorted({f[3] for f in fields}):
        sub = [f for f in fields if f[3] == r]
        cplan = sy.sy_stencil_batch_plan(q.handle, [(ny, nx, pitch, rr, C2, ua, ub)
                                                    for ny, nx, pitch, rr, ua, ub in sub], "f32", 0)
        sy.sy_stencil_batch_capture(cplan, steps)
        sy.sy_stencil_batch_run(cplan)
        reps_c, ms_c, j_c = _metered(q, stream, lambda: sy.sy_stencil_batch_run(cplan))
        sy.sy_stencil_batch_destroy(cplan)
        pts = sum(ny * nx for ny, nx, *_ in sub)
        per_class[f"r{r}"] = {"grids": len(sub), "points": pts, "updates_per_s": steps * pts / (ms_c * 1e-3),
                              "ms_per_run": ms_c,
                              "j_per_update": None if not j_c else j_c / (reps_c * steps * pts),
                              "avg_power_w": None if not j_c else j_c / (reps_c * ms_c * 1e-3),
                              "zero_fraction_u0": float(np.mean([float((inputs.batch_initial(ny, nx, "f32") == 0)
                                                                        .mean()) for ny, nx, *_ in sub])),
                              "plain_8192": plain_radius_energy(q, stream, r),
                              "plain_8192_dense": plain_radius_energy(q, stream, r, sigma=NX / 16)}
    return {"grids": len(fields), "points": points, "steps": steps, "tile_rows": tile_rows,
            "per_class": per_class,
            "modes_ms_per_run": {str(k): v for k, v in modes_ms.items()},
            "cross_step_updates_per_s": upd / (ms_p * 1e-3), "cross_step_ms_per_run": ms_p,
            "cross_step_j_per_update": None if not joules_p else joules_p / (reps_p * upd),
            "batched_updates_per_s": upd / (ms * 1e-3), "batched_gb_per_s": 12 * upd / (ms * 1e-3) / 1e9,
            "batched_ms_per_run": ms, "batched_j_per_update": None if not joules else joules / (reps * upd),
            "per_grid_graph_updates_per_s": upd / (ms_g * 1e-3), "per_grid_graph_ms_per_run": ms_g,
            "per_grid_graph_j_per_update": None if not joules_g else joules_g / (reps_g * upd),
            "per_grid_stream_updates_per_s": upd / (ms_s * 1e-3), "per_grid_stream_ms_per_run": ms_s,
            "launches_per_run": {"batched": batched_launches, "per_grid": steps * len(fields)},
            "mode": "one launch per radius class per step" if tile_rows == 0 else "one launch per step"}


def plain_radius_energy(q, stream, r: int, steps: int = 20, sigma: float = SIGMA) -> dict:
    """The 8192^2 FP32 single field at radius r (4 chunks, halo r, `steps` steps, whole runs
    graph-replayed) from a Gaussian of width `sigma`: updates/s, J/update and average power
    over a >= 1 s window.  With the headline's sigma = 64 most of the field is exactly zero;
    sigma = 512 (the batched grids' recipe, side / 16) leaves almost no point zero."""
    import torch

    import paper_2505_06022_gb300 as sy
    from paper_2505_06022_gb300 import inputs

    host = inputs.to_storage(inputs.gaussian_pulse(NY, NX, sigma), "f32")
    u0 = torch.from_numpy(host).cuda()
    A, B = torch.empty_like(u0), torch.empty_like(u0)
    p = sy.stencil_params(NY, NX, r, C2, "f32")
    chunks = sy.sy_split_rows(NY, CHUNKS)
    run = lambda: sy.sy_wave_run(q.handle, p, u0, A, B, steps, chunks, r)  # noqa: E731
    run()
    reps, ms, joules = _metered(q, stream, run)
    upd = steps * NY * NX
    return {"steps": steps, "sigma": sigma, "zero_fraction_u0": float((host == 0).mean()),
            "updates_per_s": upd / (ms * 1e-3),
            "j_per_update": None if not joules else joules / (reps * upd),
            "avg_power_w": None if not joules else joules / (reps * ms * 1e-3)}


def measure_saxpy(q, stream) -> dict:
    """SAXPY (the paper's Listing 1): N = 2^20, alpha = 2.5, seed 0 (the configured case,
    latency-bound: 12.6 MB per call), and N = 2^24, 2^26, 2^28 (up to 3.2 GB per call, HBM-bound); elements/s
    and GB/s (12 B per element) over back-to-back calls, and the result checked bit for bit
    against fl(fl(alpha x) + y) computed on the host in FP64 (exact for these inputs)."""
    import numpy as np
    import torch

    import paper_2505_06022_gb300 as sy
    from paper_2505_06022_gb300 import inputs

    out = {}
    for log2n in (20, 24, 26, 28):
        n = 1 << log2n
        x, y = inputs.saxpy_inputs(n, seed=0)
        xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
        zd = torch.empty_like(xd)
        calls = {20: 2000, 24: 400, 26: 100, 28: 40}[log2n]
        run = lambda: [sy.sy_saxpy(q.handle, n, 2.5, xd, yd, zd) for _ in range(calls)]
        run()
        reps, ms, joules = _metered(q, stream, run, min_seconds=0.5)
        per = ms / calls
        z = zd.cpu().numpy()
        want = ((np.float32(2.5) * x.astype(np.float64)).astype(np.float32).astype(np.float64)
                + y.astype(np.float64)).astype(np.float32)
        out[f"n_2^{log2n}"] = {"elements_per_s": n / (per * 1e-3), "gb_per_s": 12 * n / (per * 1e-3) / 1e9,
                               "us_per_call": per * 1e3, "bit_exact": bool(np.array_equal(z.view(np.uint32),
                                                                                         want.view(np.uint32))),
                               "j_per_element": None if not joules else joules / (reps * calls * n)}
        if log2n == 20:
            # the same calls captured into one CUDA graph (100 per replay): the device-side rate,
            # without the Python-to-C call in front of every launch
            side = torch.cuda.Stream()
            side.wait_stream(stream)
            with torch.cuda.stream(side):
                qs = sy.Queue(q.device, side)
                sy.sy_saxpy(qs.handle, n, 2.5, xd, yd, zd)
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=side):
                for _ in range(100):
                    sy.sy_saxpy(qs.handle, n, 2.5, xd, yd, zd)
            zd.zero_()
            g.replay()
            reps_g, ms_g, _ = _metered(q, stream, g.replay, min_seconds=0.3)
            zg = zd.cpu().numpy()
            out["n_2^20"]["graph"] = {"elements_per_s": n / (ms_g / 100 * 1e-3),
                                      "gb_per_s": 12 * n / (ms_g / 100 * 1e-3) / 1e9,
                                      "us_per_call": ms_g / 100 * 1e3, "calls_per_replay": 100,
                                      "bit_exact": bool(np.array_equal(zg.view(np.uint32), want.view(np.uint32)))}
            del g
            qs.close()
        del xd, yd, zd
    return out


def measure_temporal(q, stream, T: int, dtype: str = "f32", radius: int = 1) -> dict:
    """The headline simulation (8192^2, 200 steps, 4 row chunks) with temporal blocking: the
    Taylor start, then 200/T passes of T steps each (halo T*r), from the resident initial field;
    optionally with another storage type or stencil radius.  Not the headline configuration (its
    halo is 1); reported beside it, with the single-step run of the same storage and radius."""
    import numpy as np
    import torch

    import paper_2505_06022_gb300 as sy
    from paper_2505_06022_gb300 import inputs

    host = inputs.to_storage(inputs.gaussian_pulse(NY, NX, SIGMA), dtype)
    u0 = torch.from_numpy(host if dtype == "f32" else host.view(np.int16)).cuda()
    A, C, D = (torch.empty_like(u0) for _ in range(3))
    Bw = torch.empty_like(u0)
    p = sy.stencil_params(NY, NX, radius, C2, dtype)
    chunks = sy.sy_split_rows(NY, CHUNKS)
    halo = T * radius

    def sim():
        sy.sy_stencil_start(q.handle, p, u0, A, chunks, halo)
        pairs = [(A, u0), (C, D), (A, Bw)]
        cur = pairs[0]
        for k in range(STEPS // T):
            nxt = pairs[1] if k % 2 == 0 else pairs[2]
            sy.sy_stencil_multistep(q.handle, p, T, cur[0], cur[1], nxt[0], nxt[1], chunks, halo)
            cur = nxt
        return cur

    sim()
    reps, ms, joules = _metered(q, stream, sim)
    sy.sy_queue_sync(q.handle)
    esize = 4 if dtype == "f32" else 2
    upd = STEPS * NY * NX
    out = {"T": T, "dtype": dtype, "radius": radius, "halo": halo, "updates_per_s": upd / (ms * 1e-3),
           "ms_per_sim": ms, "hbm_bytes_per_update": 4 * esize / T,
           "j_per_update": None if not joules else joules / (reps * upd),
           "equivalent_single_step_gb_per_s": 3 * esize * upd / (ms * 1e-3) / 1e9}
    if radius != 1 or dtype != "f32":  # the single-step run it replaces (same storage, radius, halo)
        run = lambda: sy.sy_wave_run(q.handle, p, u0, A, C, STEPS, chunks, radius)  # noqa: E731
        run()
        reps1, ms1, j1 = _metered(q, stream, run)
        out["single_step_updates_per_s"] = upd / (ms1 * 1e-3)
        out["single_step_j_per_update"] = None if not j1 else j1 / (reps1 * upd)
    return out


def measure_split(q, stream) -> dict:
    """Split-buffer mode on the headline simulation (8192^2 FP32, 200 steps, 4 chunks, halo 1):
    every chunk in a buffer of its own with its halo rows, the rows the range mappers say each
    chunk needs moved by one halo-exchange kernel before every step (sy_stencil_step_split), the
    whole simulation captured in a CUDA graph; against the shared-buffer run's rate."""
    import numpy as np
    import torch

    import paper_2505_06022_gb300 as sy
    from paper_2505_06022_gb300 import inputs

    chunks = sy.sy_split_rows(NY, CHUNKS)
    u0 = inputs.to_storage(inputs.gaussian_pulse(NY, NX, SIGMA), "f32")
    cur0, prev, cur = [], [], []
    for c, (a, b) in enumerate(chunks):
        lo, _, rows = sy.sy_split_layout(NY, chunks, HALO, c)
        t = torch.zeros(rows, NX, dtype=torch.float32, device="cuda")
        t[lo: lo + (b - a)] = torch.from_numpy(np.ascontiguousarray(u0[a:b])).cuda()
        cur0.append(t)
        cur.append(torch.empty_like(t))
        prev.append(torch.empty_like(t))
    p = sy.stencil_params(NY, NX, RADIUS, C2, "f32")
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    qs = sy.Queue(q.device, side)

    def sim():
        for c in range(CHUNKS):
            cur[c].copy_(cur0[c])
        sy.sy_stencil_start_split(qs.handle, p, cur, prev, chunks, HALO)
        a_, b_ = prev, cur
        for _ in range(STEPS):
            sy.sy_stencil_step_split(qs.handle, p, a_, b_, a_, chunks, HALO)
            a_, b_ = b_, a_

    with torch.cuda.stream(side):
        sim()  # warm-up outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        sim()
    g.replay()
    reps, ms, joules = _metered(q, stream, g.replay)
    torch.cuda.synchronize()
    qs.close()
    upd = STEPS * NY * NX
    n_tr = len(sy.sy_rm_transfers(NY, chunks, HALO))
    return {"chunks": CHUNKS, "halo": HALO, "transfers_per_step": n_tr, "updates_per_s": upd / (ms * 1e-3),
            "ms_per_sim": ms, "j_per_update": None if not joules else joules / (reps * upd),
            "mode": "chunk-local buffers, one halo-exchange kernel before each step, launches overlapped, CUDA graph"}


def measure_wave3d(q, stream, dtype: str = "f32", radius: int = 1) -> dict:
    """Second workload: the leapfrog step on a 512^3 grid (c2 = 1/8, Gaussian sigma = 16 at the
    centre), 100 steps in 4 chunks of planes with halo r, one sy_wave3d_run replay per
    simulation from the resident initial field; 3 x sizeof(storage) bytes per update."""
    import numpy as np
    import torch

    import paper_2505_06022_gb300 as sy
    from paper_2505_06022_gb300 import inputs

    n, steps = 512, 100
    host = inputs.to_storage(inputs.gaussian_pulse_3d(n, n, n, 16.0), dtype)
    u0 = torch.from_numpy(host if dtype == "f32" else host.view(np.int16)).cuda().reshape(-1)
    a, b = torch.empty_like(u0), torch.empty_like(u0)
    p = sy.stencil3d_params(n, n, n, radius, 0.125, dtype)
    chunks = sy.sy_split_rows(n, 4)
    run = lambda: sy.sy_wave3d_run(q.handle, p, u0, a, b, steps, chunks, radius)
    run()
    l0 = q.launches
    run()
    launches = q.launches - l0
    reps, ms, joules = _metered(q, stream, run)
    esize = 4 if dtype == "f32" else 2
    upd = steps * n ** 3
    gbs = 3 * esize * upd / (ms * 1e-3) / 1e9
    peak = measured_peaks()["hbm_gbs"]
    rows, threads = sy.sy_stencil3d_variant_info(radius, dtype, 0)
    return {"grid": [n, n, n], "dtype": dtype, "radius": radius, "steps": steps, "chunks": 4,
            "tile": {"rows": rows, "threads": threads}, "updates_per_s": upd / (ms * 1e-3), "gb_per_s": gbs,
            "frac_hbm_measured": gbs / peak, "ms_per_sim": ms, "launches_per_sim": launches,
            "j_per_update": None if not joules else joules / (reps * upd)}


def batched_pick(models, modes_ms: dict, steps: int = 100) -> dict:
    """The cost model's choice of the batched plan's tile heights (config 2): per-class heights
    (mode 0: 4 rows for FP32 radius 1/2/4) or one height for every grid (2, 4, 8), by the least
    predicted total time of the 64 grids' steps; with the measured rate of that mode and of the
    default (mode 0), taken from the batched form's timing of every mode."""
    import numpy as np

    import paper_2505_06022_gb300 as sy
    from paper_2505_06022_gb300 import costmodel, inputs

    grids = inputs.batch_grids()
    points = sum(ny * nx for ny, nx, _ in grids)
    pred = {}
    for mode in (0, 2, 4, 8):
        feats = []
        for ny, nx, r in grids:
            rows = mode or (8 if r == 3 else 4)
            feats.append(sy.sy_cost_features(1, sy.SY_F32, r, ny, nx, rows, 128, 128, 1))
        pred[mode] = float(np.sum(np.exp(costmodel.predict(models, np.stack(feats))[:, 0])))
    pick = min(pred, key=pred.get)
    rate = lambda m: steps * points / (modes_ms[m] * 1e-3)  # noqa: E731
    return {"modes": [0, 2, 4, 8], "predicted_total_ms": {str(k): v for k, v in pred.items()},
            "pick_tile_rows": pick, "pick_updates_per_s": rate(pick), "default_tile_rows": 0,
            "default_updates_per_s": rate(0), "best_measured_tile_rows": min(modes_ms, key=modes_ms.get)}


def measure_learned(q, stream, batched_modes_ms: dict | None = None) -> dict:
    """The learned cost model, end to end on this GPU: the library tunes a reduced
    corpus exhaustively (220 shapes), trains its MLP on 80% of the shapes with its own
    kernels, and reports regret on the held-out 20% for the model and for the default
    configuration, and the held-out shapes' total throughput under each; then the model picks
    the tile variant of the headline workload (8192^2 FP32, radius 1, 4 chunks) -- its argmin,
    and the fastest of its top three timed once each on the workload -- and the picks and the
    default are timed as whole simulations."""
    import numpy as np
    import torch

    import paper_2505_06022_gb300 as sy
    from paper_2505_06022_gb300 import costmodel, inputs

    shapes = inputs.cost_corpus_shapes(n_stencil=200, n_saxpy=20, side_hi=8192, n_hi=1 << 26)
    t0 = time.perf_counter()
    corpus = costmodel.measure(q, shapes, reps=3)
    t_measure = time.perf_counter() - t0
    train_ids, test_ids = costmodel.split_shapes(len(shapes))
    t1 = time.perf_counter()
    models = costmodel.train_ensemble(q, corpus, train_ids, n=3, epochs=250)
    t_train = time.perf_counter() - t1
    res = costmodel.evaluate(q, models, shapes, corpus, test_ids)
    single = costmodel.evaluate(q, models[0], shapes, corpus, test_ids)["model"]
    # choice for the headline workload among the tile variants (chunking fixed at 4): the argmin of
    # the ensemble's mean predicted log time
    nv = sy.sy_stencil_variant_count(1, sy.SY_F32)
    infos = [sy.sy_stencil_variant_info(1, sy.SY_F32, v) for v in range(1, nv + 1)]
    feats = np.stack([sy.sy_cost_features(1, sy.SY_F32, 1, NY, NX, r, c, t, CHUNKS) for r, c, t in infos])
    pred = costmodel.predict(models, feats)[:, 0]
    pick = 1 + int(np.argmin(pred))
    ranked = [1 + int(i) for i in np.argsort(pred)]
    batched = batched_pick(models, batched_modes_ms) if batched_modes_ms else None
    for m in models:
        sy.sy_mlp_destroy(m)
    u0 = torch.from_numpy(inputs.to_storage(inputs.gaussian_pulse(NY, NX, SIGMA), "f32")).cuda()
    A, B = torch.empty_like(u0), torch.empty_like(u0)
    chunks = sy.sy_split_rows(NY, CHUNKS)
    # the model's ranking, verified: the top three candidates each timed once on the workload itself
    # (three simulations instead of an exhaustive sweep over every variant)
    def one_sim_ms(variant):
        p = sy.stencil_params(NY, NX, 1, C2, "f32", variant=variant)
        sy.sy_wave_run(q.handle, p, u0, A, B, STEPS, chunks, HALO)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sy.sy_wave_run(q.handle, p, u0, A, B, STEPS, chunks, HALO)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    top3 = ranked[:3]
    verified = min(top3, key=one_sim_ms)
    timing = {}
    default_v = sy.sy_stencil_default_variant(1, sy.SY_F32)
    measured = {}
    for name, variant in (("default", default_v), ("learned", pick), ("learned_top3_verified", verified)):
        if variant not in measured:  # a pick that is the default configuration is the same measurement
            p = sy.stencil_params(NY, NX, 1, C2, "f32", variant=variant)
            run = lambda: sy.sy_wave_run(q.handle, p, u0, A, B, STEPS, chunks, HALO)  # noqa: E731
            run()
            reps, ms, joules = _metered(q, stream, run)
            upd = STEPS * NY * NX
            measured[variant] = {"updates_per_s": upd / (ms * 1e-3),
                                 "j_per_update": None if not joules else joules / (reps * upd)}
        timing[name] = dict(measured[variant], variant=variant, same_as_default=variant == default_v)
    timing["learned_top3_verified"]["candidates"] = top3
    rows, cols, thr = infos[pick - 1]
    return {"corpus_rows": int(corpus["X"].shape[0]), "corpus_shapes": len(shapes), "measure_s": t_measure,
            "train_s": t_train, "ensemble": 3, "held_out_shapes": int(test_ids.size), "regret_model": res["model"],
            "regret_single_model": single,
            "regret_default": res["default"], "regret_random_expected": res["random_expected_mean"],
            "held_out_totals": res["held_out_totals"],
            "headline_pick": {"variant": pick, "tile_rows": rows, "threads": thr}, "headline": timing,
            "batched": batched}


# ---------------------------------------------------------------------------
# GPU leg
# ---------------------------------------------------------------------------

def run_gpu(args) -> None:
    import numpy as np
    import torch

    global RADIUS, HALO, BYTES_PER_UPDATE, WORKLOAD
    if args.radius != 1 or args.dtype != "f32" or args.variant:  # a non-headline variant of the workload
        RADIUS = HALO = args.radius
        BYTES_PER_UPDATE = 3 * (4 if args.dtype == "f32" else 2)
        WORKLOAD = WORKLOAD.replace("5-point FP32", f"radius-{RADIUS} star, {args.dtype.upper()} storage") \
                           .replace("halo radius 1", f"halo radius {RADIUS}")

    import paper_2505_06022_gb300 as sy
    from paper_2505_06022_gb300 import inputs

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    stream = torch.cuda.current_stream()
    q = sy.Queue(local, stream)
    p = sy.stencil_params(NY, NX, RADIUS, C2, args.dtype, variant=args.variant)
    chunks = sy.sy_split_rows(NY, CHUNKS)

    u0_host = inputs.to_storage(inputs.gaussian_pulse(NY, NX, SIGMA), args.dtype)
    u0 = torch.from_numpy(u0_host if args.dtype == "f32" else u0_host.view(np.int16)).cuda()  # resident, never written
    A = torch.empty_like(u0)
    B = torch.empty_like(u0)

    def simulate(u_init, collect: bool):
        """Start + STEPS chunked leapfrog steps from u_init (read only), one graph replay."""
        return sy.sy_wave_run(q.handle, p, u_init, A, B, STEPS, chunks, HALO, want_events=collect)

    for _ in range(args.warmup):
        simulate(u0, True)
    torch.cuda.synchronize()

    # ---- timed region: K whole simulations, device-timed on the launching stream ----
    launches0 = q.launches
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    have_energy = True
    try:
        sy.sy_meter_begin(q.handle)
    except sy.SyError:
        have_energy = False
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    wall0 = time.time()
    t_start.record(stream)
    events = []
    for _ in range(args.steps):
        _, _, events = simulate(u0, True)  # per-chunk ids of the latest run
    t_end.record(stream)
    torch.cuda.synchronize()
    wall1 = time.time()
    joules = seconds = None
    if have_energy:
        try:
            joules, seconds = sy.sy_meter_end(q.handle)
        except sy.SyError:
            have_energy = False
    if dist:
        dist.barrier()
    clk = clocks.stop((wall0, wall1))
    ms_total = t_start.elapsed_time(t_end)
    launches = q.launches - launches0
    if dist:
        t = torch.tensor([ms_total], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = float(t.item())

    updates_per_step = STEPS * NY * NX
    value = world * args.steps * updates_per_step / (ms_total * 1e-3)

    # Roofline of the dominant kernel (the chunked leapfrog step, 800 of the 804
    # launches of a step): algorithmic bytes per launch / average launch duration,
    # both over the CUDA-event-timed region.  The start's 4 launches move 8 B/point.
    bytes_per_sim = (2 * BYTES_PER_UPDATE // 3) * NY * NX + STEPS * BYTES_PER_UPDATE * NY * NX
    launches_per_sim = (STEPS + 1) * CHUNKS
    avg_ms = ms_total / (args.steps * launches_per_sim)
    alg_bytes = bytes_per_sim / launches_per_sim
    achieved = alg_bytes / (avg_ms * 1e-3) / 1e9
    # kernel-only view from the per-chunk device timestamps of the last run
    stamp_ms = sy.sy_events_elapsed(q.handle, events)[CHUNKS:]
    chunk_bytes = BYTES_PER_UPDATE * (NY // CHUNKS) * NX
    peaks = measured_peaks()
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"],
                "traffic": ncu_traffic() if (args.dtype == "f32" and RADIUS == 1) else None,
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if peaks["source"] == "measured"
                else "fallback 6.8 TB/s",
                "kernel": kernel_label(args.dtype, args.variant),
                "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": avg_ms,
                "frac_of_nominal_8000": achieved / 8000.0,
                "stamp_avg_chunk_ms": statistics.mean(stamp_ms),
                "stamp_chunk_gbs": chunk_bytes / (statistics.mean(stamp_ms) * 1e-3) / 1e9}
    energy = None
    if have_energy and joules is not None:
        # J/update over a window of >= 2 s (20 periods of NVML's 100 ms energy counter):
        # the timed region when it is that long, else a dedicated window of whole
        # simulations right after it; idle power from a 2 s window with the GPU idle.
        sims = args.steps
        if seconds < 2.0:
            torch.cuda.synchronize()
            sy.sy_meter_begin(q.handle)
            sims, t0 = 0, time.perf_counter()
            while sims < 3 or time.perf_counter() - t0 < 2.0:
                _, _, events = simulate(u0, True)
                sims += 1
                if sims % 4 == 0:
                    torch.cuda.synchronize()
            torch.cuda.synchronize()
            joules, seconds = sy.sy_meter_end(q.handle)
        torch.cuda.synchronize()
        sy.sy_meter_begin(q.handle)
        time.sleep(2.0)
        idle_j, idle_s = sy.sy_meter_end(q.handle)
        if joules > 0:
            idle_w = idle_j / idle_s
            kern_j = [sy.sy_kernel_energy(q.handle, e) for e in events[CHUNKS:]]
            energy = {"joules": joules, "window_s": seconds, "simulations": sims,
                      "j_per_update": joules / (sims * updates_per_step), "avg_power_w": joules / seconds,
                      "idle_w": idle_w,
                      "j_per_update_above_idle": (joules - idle_w * seconds) / (sims * updates_per_step),
                      "chunk_kernel_j_mean": statistics.mean(kern_j),
                      "chunk_kernel_j_note": "attributed: window power x kernel time (sy_kernel_energy)"}
            # the same chunk kernel measured alone: chunk 1 replayed in its own >= 1 s window
            rep = sy.sy_chunk_energy_replay(q.handle, p, A, u0, B, chunks, 1, HALO, min_seconds=1.0)
            energy["chunk_replay"] = {"chunk": 1, "j_per_launch": rep["joules"], "ms_per_launch": rep["ms"],
                                      "launches": rep["reps"],
                                      "j_per_update": rep["joules"] / ((chunks[1][1] - chunks[1][0]) * NX),
                                      "note": "measured: the chunk's launch replayed alone in one NVML window "
                                              "(sy_chunk_energy_replay)"}

    # ---- e2e: whole simulations from host memory, through sy_wave_run_host ----
    # Every step hands the library the pinned host initial field and receives the final
    # field in pinned host memory; the library makes both copies (one per direction, on
    # its own copy streams, overlapping the neighbouring steps' simulations).  The timed
    # region is host wall-clock from a synchronised start to sy_queue_sync after the last
    # step, so every copy is inside it.  The sequential form (sync after every step, no
    # overlap) is reported beside it.  Each form is timed three times; the median counts.
    e2e = None
    if True:
        h_in = torch.from_numpy(u0_host if args.dtype == "f32" else u0_host.view(np.int16)).pin_memory()
        h_out = [torch.empty_like(h_in).pin_memory() for _ in range(2)]
        k_e2e = max(1, args.steps)  # the same step count as the device-timed region

        def host_steps(k, sync_each):
            for i in range(k):
                sy.sy_wave_run_host(q.handle, p, h_in, h_out[i % 2], STEPS, chunks, HALO)
                if sync_each:
                    sy.sy_queue_sync(q.handle)
            sy.sy_queue_sync(q.handle)

        host_steps(2, False)  # first calls allocate the work sets and capture their graphs
        _, cv_d, _ = simulate(u0, False)
        torch.cuda.synchronize()
        want_out = {A.data_ptr(): A, B.data_ptr(): B, u0.data_ptr(): u0}[cv_d].cpu()
        assert torch.equal(h_out[0], want_out) and torch.equal(h_out[1], want_out), \
            "sy_wave_run_host result differs from the device-buffer run"

        def timed(sync_each):
            out = []
            for _ in range(3):
                torch.cuda.synchronize()
                if dist:
                    dist.barrier()
                t0 = time.perf_counter()
                host_steps(k_e2e, sync_each)
                out.append((time.perf_counter() - t0) * 1e3)
            return statistics.median(out)

        h_out[0].zero_()
        ms_e2e = timed(False)
        ms_seq = timed(True)
        if dist:  # the job takes as long as its slowest replica
            t = torch.tensor([ms_e2e, ms_seq], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms_e2e, ms_seq = float(t[0].item()), float(t[1].item())
        assert torch.equal(h_out[0], want_out), "sy_wave_run_host result changed between calls"
        e2e = {"value": world * k_e2e * updates_per_step / (ms_e2e * 1e-3), "unit": "updates/s",
               "h2d_bytes_per_step": h_in.numel() * h_in.element_size(),
               "d2h_bytes_per_step": h_out[0].numel() * h_out[0].element_size(),
               "ms_per_step": ms_e2e / k_e2e, "steps": k_e2e, "repeats": 3,
               "api": "sy_wave_run_host (C ABI, pinned host buffers in and out)",
               "timing": "host wall clock, synchronised start to sy_queue_sync after the last step",
               "mode": "the library's copies overlap the neighbouring steps' simulations",
               "sequential_value": world * k_e2e * updates_per_step / (ms_seq * 1e-3)}

    # accuracy of the headline's final field against the FP64 oracle (tolerance 1e-5 relative)
    accuracy = None
    if rank == 0 and args.dtype == "f32" and RADIUS == 1 and args.cpu_seconds > 0:
        _, cv_h, _ = simulate(u0, False)
        torch.cuda.synchronize()
        final = {A.data_ptr(): A, B.data_ptr(): B, u0.data_ptr(): u0}[cv_h].cpu().numpy().astype(np.float64)
        err = error_vs_f64(final)
        accuracy = dict(err, **stated_accuracy("f32", err))

    forms = None
    if rank == 0 and world == 1 and args.forms and args.dtype == "f32" and RADIUS == 1:
        # the other forms are single-GPU comparisons; with replicas they would hold every GPU idle
        forms = {"plain_f32": {"updates_per_s": value, "gb_per_s": value * BYTES_PER_UPDATE / 1e9,
                               "j_per_update": None if not energy else energy["j_per_update"]}}
        for dt in ("bf16", "f16"):
            forms[dt] = measure_precision_form(q, stream, dt)
        forms["saxpy"] = measure_saxpy(q, stream)
        forms["wave3d_f32_r1"] = measure_wave3d(q, stream, "f32", 1)
        forms["wave3d_bf16_r1"] = measure_wave3d(q, stream, "bf16", 1)
        forms["wave3d_f32_r2"] = measure_wave3d(q, stream, "f32", 2)
        forms["wave3d_f32_r4"] = measure_wave3d(q, stream, "f32", 4)
        forms["wave3d_bf16_r4"] = measure_wave3d(q, stream, "bf16", 4)
        forms["batched"] = measure_batched(q, stream)
        forms["split_buffers"] = measure_split(q, stream)
        forms["temporal_T2"] = measure_temporal(q, stream, 2)
        forms["temporal_T4"] = measure_temporal(q, stream, 4)
        forms["temporal_T4_bf16"] = measure_temporal(q, stream, 4, "bf16")
        forms["temporal_T2_r4"] = measure_temporal(q, stream, 2, "f32", 4)
        forms["temporal_T4_r4"] = measure_temporal(q, stream, 4, "f32", 4)
        forms["learned"] = measure_learned(q, stream, {int(k): v for k, v in
                                                      forms["batched"]["modes_ms_per_run"].items()})
    if dist:
        dist.barrier()
    if rank == 0:
        cpu = None
        if world == 1 and args.cpu_seconds > 0:
            import oracle

            cpu = oracle_sample(args.cpu_seconds)
            all_cores = oracle.threads()
            oracle.set_threads(1)  # the same sample on one host core, for the per-core rate
            try:
                one = oracle_sample(max(2.0, args.cpu_seconds / 4))
            finally:
                oracle.set_threads(all_cores)
            cpu["single_thread_value"] = one["value"]
        line = {
            "metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
            "config": {"workload": WORKLOAD, "updates_per_step": updates_per_step,
                       "launches_per_step": launches // max(1, args.steps),
                       "l2": ("inputs larger than L2 (three 256 MiB fields, 161 GB of algorithmic traffic per "
                              "simulation), so simulations need no L2 flush between them; inside a simulation "
                              "the sweep direction alternates, so each time step starts on rows the previous "
                              "one left in L2"),
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
            "gb_per_s": value * BYTES_PER_UPDATE / 1e9,
            "frac_hbm_measured": value * BYTES_PER_UPDATE / 1e9 / peaks["hbm_gbs"],
            "roofline": roofline,
            "energy": energy,
            "accuracy": accuracy,
            "e2e": e2e,
            "gpu_launches": launches,
            "forms": forms,
            "clocks": clk,
            "device": device_info(local),
            "cpu_baseline": None if cpu is None else {k: cpu[k] for k in ("value", "unit", "cores", "kind",
                                                                          "sample", "single_thread_value")},
        }
        print(json.dumps(line), flush=True)
    q.close()
    if dist:
        dist.destroy_process_group()


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sy", choices=["sy", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--forms", type=int, default=1,
                    help="also measure the BF16/FP16, batched and learned forms (rank 0, headline workload)")
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16", "f16"],
                    help="field storage of the wave workload (headline: f32)")
    ap.add_argument("--radius", type=int, default=1, choices=[1, 2, 3, 4],
                    help="stencil and halo radius of the wave workload (headline: 1)")
    ap.add_argument("--variant", type=int, default=0,
                    help="2D step variant (0 = the library default; used for profiling captures)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "sy":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
