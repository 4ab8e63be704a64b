"""GB300-native range-mapped data-parallel kernels with energy metering.

The compute path is libsy.so: hand-written sm_103a CUDA behind the C ABI declared
in include/sy.h.  This package is its thin Python binding: every function named
`sy_*` here marshals its arguments (torch tensors -> device pointers, Python
lists -> C arrays) and calls the C entry point of the same name; no step of the
computation runs in Python or PyTorch.  PyTorch provides device memory and
streams only.

The library is loaded on first use, not at import, so `inputs` can be imported
on hosts without a GPU.  If libsy.so is missing or older than its sources it is
built with nvcc; if that is impossible the call raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

__all__ = [
    "SyError", "lib", "lib_path", "Queue", "Chunk", "StencilParams",
    "SY_F32", "SY_BF16", "SY_F16", "DTYPE_CODES",
]

SY_F32, SY_BF16, SY_F16 = 0, 1, 2
SY_STREAM_LEGACY = 0x1  # cudaStreamLegacy
DTYPE_CODES = {"f32": SY_F32, "bf16": SY_BF16, "f16": SY_F16}

STATUS = {
    0: "SY_OK", 1: "SY_ERR_INVALID_ARGUMENT", 2: "SY_ERR_NULL_POINTER", 3: "SY_ERR_ALIAS",
    4: "SY_ERR_BAD_CHUNKS", 5: "SY_ERR_HALO_TOO_SMALL", 6: "SY_ERR_UNSUPPORTED", 7: "SY_ERR_CUDA",
    8: "SY_ERR_NVML_UNAVAILABLE", 9: "SY_ERR_TIMEOUT", 10: "SY_ERR_OUT_OF_MEMORY", 11: "SY_ERR_NOT_READY",
    12: "SY_ERR_IO", 13: "SY_ERR_NVML",
}


class SyError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status
        self.name = STATUS.get(status, str(status))


class Chunk(C.Structure):
    _fields_ = [("begin", C.c_int64), ("end", C.c_int64)]


class BatchGrid(C.Structure):
    _fields_ = [("ny", C.c_int64), ("nx", C.c_int64), ("pitch", C.c_int64), ("radius", C.c_int32),
                ("c2", C.c_float), ("u_a", C.c_void_p), ("u_b", C.c_void_p)]


class TuneRecord(C.Structure):
    _fields_ = [("variant", C.c_int32), ("tile_rows", C.c_int32), ("tile_cols", C.c_int32),
                ("threads", C.c_int32), ("chunks", C.c_int32), ("ms", C.c_double)]


class CostQuery(C.Structure):
    _fields_ = [("kind", C.c_int32), ("dtype", C.c_int32), ("radius", C.c_int32), ("ny", C.c_int64),
                ("nx", C.c_int64), ("tile_rows", C.c_int32), ("tile_cols", C.c_int32), ("threads", C.c_int32),
                ("chunks", C.c_int32)]


SY_COST_FEATURES = 13


class Transfer(C.Structure):
    _fields_ = [("src", C.c_int32), ("dst", C.c_int32), ("row_begin", C.c_int64), ("row_end", C.c_int64)]


class Stencil3dParams(C.Structure):
    _fields_ = [("nz", C.c_int64), ("ny", C.c_int64), ("nx", C.c_int64), ("pitch", C.c_int64), ("plane", C.c_int64),
                ("radius", C.c_int32), ("dtype", C.c_int32), ("c2", C.c_float), ("variant", C.c_int32)]


class Box(C.Structure):
    _fields_ = [("lo", C.c_int64 * 3), ("hi", C.c_int64 * 3)]


class RangeMapper(C.Structure):
    _fields_ = [("kind", C.c_int32), ("dim", C.c_int32), ("radius", C.c_int64 * 3), ("fixed", Box)]


class BoxTransfer(C.Structure):
    _fields_ = [("src", C.c_int32), ("dst", C.c_int32), ("box", Box)]


SY_RM_ONE_TO_ONE, SY_RM_NEIGHBOURHOOD, SY_RM_SLICE, SY_RM_ALL, SY_RM_FIXED = 0, 1, 2, 3, 4


class FreqPoint(C.Structure):
    _fields_ = [("sm_mhz", C.c_uint32), ("seconds", C.c_double), ("joules", C.c_double)]


SY_TARGET_MIN_TIME, SY_TARGET_MIN_ENERGY, SY_TARGET_MIN_EDP, SY_TARGET_MIN_ED2P = 0, 1, 2, 3
MEASURE_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_uint32, C.POINTER(C.c_double), C.POINTER(C.c_double))


class StencilParams(C.Structure):
    _fields_ = [("ny", C.c_int64), ("nx", C.c_int64), ("pitch", C.c_int64), ("radius", C.c_int32),
                ("dtype", C.c_int32), ("c2", C.c_float), ("variant", C.c_int32)]


_p = C.c_void_p
_i64 = C.c_int64
_u64 = C.c_uint64
_st = C.c_int
_lock = threading.Lock()
_lib = None

# name: (argtypes) -- every entry returns sy_status unless listed in _RESTYPE
_SIGS = {
    "sy_status_string": [_st],
    "sy_last_error": [],
    "sy_abi_version": [],
    "sy_queue_create": [C.c_int, _p, _p],
    "sy_queue_destroy": [_p],
    "sy_queue_sync": [_p],
    "sy_queue_stream": [_p, _p],
    "sy_queue_launch_count": [_p, _p],
    "sy_event_elapsed": [_p, _u64, _p],
    "sy_events_elapsed": [_p, _p, C.c_int, _p],
    "sy_energy_read": [_p, _p],
    "sy_device_energy": [_p, _p],
    "sy_meter_begin": [_p],
    "sy_meter_end": [_p, _p, _p],
    "sy_kernel_energy": [_p, _u64, _p],
    "sy_saxpy": [_p, _i64, C.c_float, _p, _p, _p, _p],
    "sy_saxpy_split": [_p, _i64, C.c_float, _p, _p, _p, _p, C.c_int, _p],
    "sy_split_rows": [_i64, C.c_int, _p],
    "sy_rm_one_to_one": [Chunk, _p],
    "sy_rm_neighbourhood": [Chunk, C.c_int, _i64, _p],
    "sy_chunks_validate": [_i64, _p, C.c_int],
    "sy_stencil_step": [_p, _p, _p, _p, _p, _p, C.c_int, C.c_int, _p],
    "sy_stencil_start": [_p, _p, _p, _p, _p, C.c_int, C.c_int, _p],
    "sy_stencil_variant_count": [C.c_int, C.c_int, _p],
    "sy_stencil_variant_info": [C.c_int, C.c_int, C.c_int, _p, _p, _p],
    "sy_wave_energy": [_p, _p, _p, _p, _p, _p, _p],
    "sy_wave_energy_static": [_p, _p, _p, _p, _p],
    "sy_rm_transfers": [_i64, _p, C.c_int, C.c_int, _p, C.c_int, _p],
    "sy_split_layout": [_i64, _p, C.c_int, C.c_int, C.c_int, _p, _p, _p],
    "sy_stencil_step_split": [_p, _p, _p, _p, _p, _p, C.c_int, C.c_int, _p],
    "sy_stencil_start_split": [_p, _p, _p, _p, _p, C.c_int, C.c_int, _p],
    "sy_stencil_step_rows": [_p, _p, _p, _p, _p, _i64, _i64, C.c_int, C.c_int, _p],
    "sy_tune_stencil": [_p, _p, _p, _p, _p, _p, C.c_int, C.c_int, _p, C.c_int, _p],
    "sy_tune_saxpy": [_p, _i64, _p, _p, _p, _p, C.c_int, C.c_int, _p, C.c_int, _p],
    "sy_saxpy_variant_count": [_p],
    "sy_saxpy_variant_info": [C.c_int, _p, _p],
    "sy_saxpy_config": [_p, _i64, C.c_float, _p, _p, _p, C.c_int, _p, C.c_int, _p],
    "sy_cost_features": [_p, _p],
    "sy_mlp_create": [_p, C.c_int, C.c_int, C.c_int, _u64, _p],
    "sy_mlp_destroy": [_p],
    "sy_mlp_param_count": [_p, _p],
    "sy_mlp_get_params": [_p, _p, _i64],
    "sy_mlp_get_grad": [_p, _p, _i64],
    "sy_mlp_set_params": [_p, _p, _i64],
    "sy_mlp_forward": [_p, _p, _i64, _p],
    "sy_mlp_loss_grad": [_p, _p, _p, _i64, _p],
    "sy_mlp_adam_step": [_p, C.c_float, C.c_float, C.c_float, C.c_float],
    "sy_mlp_train": [_p, _p, _p, _i64, C.c_int, C.c_int, C.c_float, _u64, _p],
    "sy_mlp_normalization": [_p, _p, _p, _p, _p],
    "sy_cost_model_predict": [_p, _p, _i64, _p],
    "sy_cost_model_choose": [_p, _p, C.c_int, C.c_int, _p],
    "sy_mlp_save": [_p, C.c_char_p],
    "sy_mlp_load": [_p, C.c_char_p, _p],
    "sy_stencil_batch_plan": [_p, _p, C.c_int, C.c_int, C.c_int, _p],
    "sy_stencil_batch_info": [_p, _p, _p, _p],
    "sy_stencil_batch_start": [_p, C.c_int],
    "sy_stencil_batch_step": [_p, C.c_int, C.c_int],
    "sy_stencil_batch_capture": [_p, _i64],
    "sy_stencil_batch_capture_persistent": [_p, _i64],
    "sy_stencil_batch_run": [_p],
    "sy_stencil_batch_times": [_p, _p, C.c_int],
    "sy_stencil_batch_destroy": [_p],
    "sy_stencil_multistep": [_p, _p, C.c_int, _p, _p, _p, _p, _p, C.c_int, C.c_int, _p],
    "sy_wave_run": [_p, _p, _p, _p, _p, _i64, _p, C.c_int, C.c_int, _p, _p, _p],
    "sy_wave_run_host": [_p, _p, _p, _p, _p, _i64, _p, C.c_int, C.c_int, _p],
    "sy_stencil_default_variant": [C.c_int, C.c_int, _p],
    "sy_chunk_energy_replay": [_p, _p, _p, _p, _p, _p, C.c_int, C.c_int, C.c_int, C.c_double, C.c_int, _p, _p,
                               _p],
    "sy_stencil3d_step": [_p, _p, _p, _p, _p, _p, C.c_int, C.c_int, _p],
    "sy_stencil3d_start": [_p, _p, _p, _p, _p, C.c_int, C.c_int, _p],
    "sy_wave3d_run": [_p, _p, _p, _p, _p, _i64, _p, C.c_int, C.c_int, _p, _p, _p],
    "sy_stencil3d_variant_count": [C.c_int, C.c_int, _p],
    "sy_wave3d_energy": [_p, _p, _p, _p, _p, _p, _p],
    "sy_chunk_stats_read": [_p, _p, _p, _p, C.c_int, _p],
    "sy_checkpoint_save": [_p, C.c_char_p, _p, _p, _p, _i64],
    "sy_checkpoint_load": [_p, C.c_char_p, _p, _p, _p, _p],
    "sy_stencil3d_step_planes": [_p, _p, _p, _p, _p, _i64, _i64, C.c_int, C.c_int, _p],
    "sy_tune_stencil3d": [_p, _p, _p, _p, _p, _p, C.c_int, C.c_int, _p, C.c_int, _p],
    "sy_tune_exhaustive": [_p, C.c_int, _p, _i64, _p, _p, _p, _p, C.c_int, C.c_int, _p, C.c_int, _p, _p],
    "sy_mlp_backward": [_p, _p, _p, _i64, _p],
    "sy_stencil3d_variant_info": [C.c_int, C.c_int, C.c_int, _p, _p],
    "sy_rm_box": [_p, _p, _p, _p],
    "sy_rm_box_transfers": [_p, _p, C.c_int, _p, _p, C.c_int, _p],
    "sy_clock_choose": [C.c_int, _p, C.c_int, _p],
    "sy_clock_nvml_index": [C.c_int, _p],
    "sy_clock_supported": [C.c_uint32, _p, _p, C.c_int, _p],
    "sy_clock_current": [C.c_uint32, _p, _p],
    "sy_clock_lock": [C.c_uint32, C.c_uint32],
    "sy_clock_unlock": [C.c_uint32],
    "sy_clock_sweep": [C.c_uint32, _p, C.c_int, MEASURE_FN, _p, C.c_int, _p, _p],
}
_RESTYPE = {"sy_status_string": C.c_char_p, "sy_last_error": C.c_char_p, "sy_abi_version": C.c_int}


def lib_path() -> str:
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "libsy.so")


def lib() -> C.CDLL:
    """Load libsy.so, building it first if it is missing or stale."""
    global _lib
    with _lock:
        if _lib is None:
            from . import _build

            path = _build.build()
            L = C.CDLL(path)
            for name, args in _SIGS.items():
                fn = getattr(L, name, None)
                if fn is None:
                    continue
                fn.argtypes = args
                fn.restype = _RESTYPE.get(name, _st)
            _lib = L
    return _lib


def _call(name: str, *args) -> None:
    L = lib()
    rc = getattr(L, name)(*args)
    if rc != 0:
        raise SyError(rc, L.sy_last_error().decode(errors="replace"))


def _ptr(t) -> int | None:
    """Device (or host) address of a tensor / integer address / None.  A tensor must be
    contiguous: the library reads its own layout (pitch, plane) from the call's
    parameters, so a strided view would be read as something else."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if hasattr(t, "is_contiguous") and not t.is_contiguous():
        raise ValueError("tensor arguments must be contiguous (pass the pitch / plane of a padded layout instead "
                         "of a strided view)")
    return t.data_ptr()


def _chunks(chunks) -> tuple[C.Array, int]:
    chunks = list(chunks)
    arr = (Chunk * max(1, len(chunks)))(*[Chunk(int(a), int(b)) for a, b in chunks])
    return arr, len(chunks)


# ---------------------------------------------------------------------------
# C entry points, one wrapper per name
# ---------------------------------------------------------------------------

def sy_abi_version() -> int:
    return lib().sy_abi_version()


def sy_status_string(status: int) -> str:
    return lib().sy_status_string(status).decode()


def sy_queue_create(device: int = 0, stream: int | None = None) -> int:
    h = C.c_void_p()
    _call("sy_queue_create", device, stream, C.byref(h))
    return h.value


def sy_queue_destroy(q: int) -> None:
    _call("sy_queue_destroy", q)


def sy_queue_sync(q: int) -> None:
    _call("sy_queue_sync", q)


def sy_queue_stream(q: int) -> int:
    s = C.c_void_p()
    _call("sy_queue_stream", q, C.byref(s))
    return s.value or 0


def sy_queue_launch_count(q: int) -> int:
    n = C.c_uint64()
    _call("sy_queue_launch_count", q, C.byref(n))
    return n.value


def sy_event_elapsed(q: int, ev: int) -> float:
    ms = C.c_double()
    _call("sy_event_elapsed", q, ev, C.byref(ms))
    return ms.value


def sy_events_elapsed(q: int, events) -> list[float]:
    evs = list(events)
    arr = (C.c_uint64 * max(1, len(evs)))(*evs)
    ms = (C.c_double * max(1, len(evs)))()
    _call("sy_events_elapsed", q, arr, len(evs), ms)
    return list(ms[: len(evs)])


def sy_energy_read(q: int) -> int:
    mj = C.c_uint64()
    _call("sy_energy_read", q, C.byref(mj))
    return mj.value


def sy_device_energy(q: int) -> float:
    j = C.c_double()
    _call("sy_device_energy", q, C.byref(j))
    return j.value


def sy_meter_begin(q: int) -> None:
    _call("sy_meter_begin", q)


def sy_meter_end(q: int) -> tuple[float, float]:
    j, s = C.c_double(), C.c_double()
    _call("sy_meter_end", q, C.byref(j), C.byref(s))
    return j.value, s.value


def sy_kernel_energy(q: int, ev: int) -> float:
    j = C.c_double()
    _call("sy_kernel_energy", q, ev, C.byref(j))
    return j.value


def sy_saxpy(q: int, n: int, alpha: float, x, y, z, want_event: bool = False) -> int:
    ev = C.c_uint64()
    _call("sy_saxpy", q, n, alpha, _ptr(x), _ptr(y), _ptr(z), C.byref(ev) if want_event else None)
    return ev.value


def sy_saxpy_split(q: int, n: int, alpha: float, x, y, z, chunks, want_events: bool = False) -> list[int]:
    arr, k = _chunks(chunks)
    evs = (C.c_uint64 * max(1, k))()
    _call("sy_saxpy_split", q, n, alpha, _ptr(x), _ptr(y), _ptr(z), arr, k, evs if want_events else None)
    return list(evs[:k]) if want_events else []


def sy_split_rows(n: int, k: int) -> list[tuple[int, int]]:
    arr = (Chunk * max(1, k))()
    _call("sy_split_rows", n, k, arr)
    return [(arr[i].begin, arr[i].end) for i in range(k)]


def sy_rm_one_to_one(chunk) -> tuple[int, int]:
    out = Chunk()
    _call("sy_rm_one_to_one", Chunk(*chunk), C.byref(out))
    return out.begin, out.end


def sy_rm_neighbourhood(chunk, radius: int, n: int) -> tuple[int, int]:
    out = Chunk()
    _call("sy_rm_neighbourhood", Chunk(*chunk), radius, n, C.byref(out))
    return out.begin, out.end


def sy_chunks_validate(n: int, chunks) -> None:
    arr, k = _chunks(chunks)
    _call("sy_chunks_validate", n, arr, k)


def stencil_params(ny: int, nx: int, radius: int = 1, c2: float = 0.25, dtype: str | int = "f32",
                   pitch: int | None = None, variant: int = 0) -> StencilParams:
    code = DTYPE_CODES[dtype] if isinstance(dtype, str) else int(dtype)
    return StencilParams(ny, nx, nx if pitch is None else pitch, radius, code, c2, variant)


def sy_stencil_step(q: int, p: StencilParams, u_prev, u_cur, u_next, chunks, halo_radius: int,
                    want_events: bool = False) -> list[int]:
    arr, k = _chunks(chunks)
    evs = (C.c_uint64 * max(1, k))()
    _call("sy_stencil_step", q, C.byref(p), _ptr(u_prev), _ptr(u_cur), _ptr(u_next), arr, k, halo_radius,
          evs if want_events else None)
    return list(evs[:k]) if want_events else []


def sy_stencil_start(q: int, p: StencilParams, u0, u_m1, chunks, halo_radius: int,
                     want_events: bool = False) -> list[int]:
    arr, k = _chunks(chunks)
    evs = (C.c_uint64 * max(1, k))()
    _call("sy_stencil_start", q, C.byref(p), _ptr(u0), _ptr(u_m1), arr, k, halo_radius,
          evs if want_events else None)
    return list(evs[:k]) if want_events else []


def sy_wave_energy_static(stream: int | None, p: StencilParams, u_new, u_old, out3) -> None:
    """Allocation-free energy: writes (energy, kinetic, potential) into the
    caller's device buffer out3 (3 float64) on `stream` (None = legacy default)."""
    _call("sy_wave_energy_static", stream or None, C.byref(p), _ptr(u_new), _ptr(u_old), _ptr(out3))


def sy_stencil_batch_plan(q: int, grids, dtype: str | int = "f32", tile_rows: int = 0) -> int:
    """grids: iterable of (ny, nx, pitch, radius, c2, u_a, u_b) with tensors or addresses."""
    code = DTYPE_CODES[dtype] if isinstance(dtype, str) else int(dtype)
    gl = list(grids)
    arr = (BatchGrid * max(1, len(gl)))(*[BatchGrid(ny, nx, pitch, r, c2, _ptr(a), _ptr(b))
                                         for (ny, nx, pitch, r, c2, a, b) in gl])
    h = C.c_void_p()
    _call("sy_stencil_batch_plan", q, arr, len(gl), code, tile_rows, C.byref(h))
    return h.value


def sy_stencil_batch_info(plan: int) -> tuple[int, int, int]:
    t, pts, b = C.c_int64(), C.c_int64(), C.c_int()
    _call("sy_stencil_batch_info", plan, C.byref(t), C.byref(pts), C.byref(b))
    return t.value, pts.value, b.value


def sy_stencil_batch_start(plan: int, timed: bool = False) -> None:
    _call("sy_stencil_batch_start", plan, int(timed))


def sy_stencil_batch_step(plan: int, parity: int, timed: bool = False) -> None:
    _call("sy_stencil_batch_step", plan, parity, int(timed))


def sy_stencil_batch_capture(plan: int, steps: int) -> None:
    _call("sy_stencil_batch_capture", plan, steps)


def sy_stencil_batch_capture_persistent(plan: int, steps: int) -> None:
    _call("sy_stencil_batch_capture_persistent", plan, steps)


def sy_stencil_batch_run(plan: int) -> None:
    _call("sy_stencil_batch_run", plan)


def sy_stencil_batch_times(plan: int, n: int) -> list[float]:
    ms = (C.c_double * max(1, n))()
    _call("sy_stencil_batch_times", plan, ms, n)
    return list(ms[:n])


def sy_stencil_batch_destroy(plan: int) -> None:
    _call("sy_stencil_batch_destroy", plan)


def sy_rm_transfers(ny: int, chunks, halo_radius: int) -> list[tuple[int, int, int, int]]:
    """[(src, dst, row_begin, row_end)] inferred from the neighbourhood range mappers."""
    arr, k = _chunks(chunks)
    n = C.c_int()
    _call("sy_rm_transfers", ny, arr, k, halo_radius, None, 0, C.byref(n))
    out = (Transfer * max(1, n.value))()
    _call("sy_rm_transfers", ny, arr, k, halo_radius, out, n.value, C.byref(n))
    return [(out[i].src, out[i].dst, out[i].row_begin, out[i].row_end) for i in range(n.value)]


def sy_split_layout(ny: int, chunks, halo_radius: int, chunk: int) -> tuple[int, int, int]:
    arr, k = _chunks(chunks)
    lo, hi, rows = C.c_int64(), C.c_int64(), C.c_int64()
    _call("sy_split_layout", ny, arr, k, halo_radius, chunk, C.byref(lo), C.byref(hi), C.byref(rows))
    return lo.value, hi.value, rows.value


def _ptr_list(ts):
    return (C.c_void_p * max(1, len(ts)))(*[_ptr(t) for t in ts])


def sy_stencil_step_split(q: int, p: StencilParams, local_prev, local_cur, local_next, chunks, halo_radius: int,
                          want_events: bool = False) -> list[int]:
    arr, k = _chunks(chunks)
    evs = (C.c_uint64 * max(1, k))()
    _call("sy_stencil_step_split", q, C.byref(p), _ptr_list(local_prev), _ptr_list(local_cur),
          _ptr_list(local_next), arr, k, halo_radius, evs if want_events else None)
    return list(evs[:k]) if want_events else []


def sy_stencil_start_split(q: int, p: StencilParams, local_u0, local_um1, chunks, halo_radius: int) -> None:
    arr, k = _chunks(chunks)
    _call("sy_stencil_start_split", q, C.byref(p), _ptr_list(local_u0), _ptr_list(local_um1), arr, k,
          halo_radius, None)


def sy_stencil_step_rows(q: int, p: StencilParams, u_prev, u_cur, u_next, row_begin: int, row_end: int,
                         halo_radius: int, start: bool = False, want_event: bool = False) -> int:
    ev = C.c_uint64()
    _call("sy_stencil_step_rows", q, C.byref(p), _ptr(u_prev), _ptr(u_cur), _ptr(u_next), row_begin, row_end,
          halo_radius, int(start), C.byref(ev) if want_event else None)
    return ev.value


def _records(arr, n) -> list[dict]:
    return [{"variant": arr[i].variant, "tile_rows": arr[i].tile_rows, "tile_cols": arr[i].tile_cols,
             "threads": arr[i].threads, "chunks": arr[i].chunks, "ms": arr[i].ms} for i in range(n)]


def sy_tune_stencil(q: int, p: StencilParams, u_prev, u_cur, u_next, chunk_counts=(1, 2, 4, 8), reps: int = 3):
    counts = (C.c_int * len(chunk_counts))(*chunk_counts)
    cap = sy_stencil_variant_count(p.radius, p.dtype) * len(chunk_counts)
    out = (TuneRecord * cap)()
    n = C.c_int()
    _call("sy_tune_stencil", q, C.byref(p), _ptr(u_prev), _ptr(u_cur), _ptr(u_next), counts, len(chunk_counts),
          reps, out, cap, C.byref(n))
    return _records(out, n.value)


def sy_tune_saxpy(q: int, n: int, x, y, z, chunk_counts=(1, 2, 4, 8), reps: int = 3):
    counts = (C.c_int * len(chunk_counts))(*chunk_counts)
    cap = sy_saxpy_variant_count() * len(chunk_counts)
    out = (TuneRecord * cap)()
    k = C.c_int()
    _call("sy_tune_saxpy", q, n, _ptr(x), _ptr(y), _ptr(z), counts, len(chunk_counts), reps, out, cap, C.byref(k))
    return _records(out, k.value)


def sy_saxpy_variant_count() -> int:
    n = C.c_int()
    _call("sy_saxpy_variant_count", C.byref(n))
    return n.value


def sy_saxpy_variant_info(variant: int) -> tuple[int, int]:
    t, w = C.c_int(), C.c_int()
    _call("sy_saxpy_variant_info", variant, C.byref(t), C.byref(w))
    return t.value, w.value


def sy_saxpy_config(q: int, n: int, alpha: float, x, y, z, variant: int, chunks, want_events: bool = False):
    arr, k = _chunks(chunks)
    evs = (C.c_uint64 * max(1, k))()
    _call("sy_saxpy_config", q, n, alpha, _ptr(x), _ptr(y), _ptr(z), variant, arr, k, evs if want_events else None)
    return list(evs[:k]) if want_events else []


def sy_cost_features(kind: int, dtype: int, radius: int, ny: int, nx: int, tile_rows: int, tile_cols: int,
                     threads: int, chunks: int):
    import numpy as np

    out = np.empty(SY_COST_FEATURES, np.float32)
    qy = CostQuery(kind, dtype, radius, ny, nx, tile_rows, tile_cols, threads, chunks)
    _call("sy_cost_features", C.byref(qy), out.ctypes.data)
    return out


def _f32(a):
    import numpy as np

    return np.ascontiguousarray(a, dtype=np.float32)


def sy_mlp_create(q: int, in_features: int, hidden: int = 64, out_features: int = 2, seed: int = 0) -> int:
    h = C.c_void_p()
    _call("sy_mlp_create", q, in_features, hidden, out_features, seed, C.byref(h))
    return h.value


def sy_mlp_destroy(m: int) -> None:
    _call("sy_mlp_destroy", m)


def sy_mlp_param_count(m: int) -> int:
    n = C.c_int64()
    _call("sy_mlp_param_count", m, C.byref(n))
    return n.value


def sy_mlp_get_params(m: int):
    import numpy as np

    out = np.empty(sy_mlp_param_count(m), np.float32)
    _call("sy_mlp_get_params", m, out.ctypes.data, out.size)
    return out


def sy_mlp_get_grad(m: int):
    import numpy as np

    out = np.empty(sy_mlp_param_count(m), np.float32)
    _call("sy_mlp_get_grad", m, out.ctypes.data, out.size)
    return out


def sy_mlp_set_params(m: int, params) -> None:
    a = _f32(params)
    _call("sy_mlp_set_params", m, a.ctypes.data, a.size)


def sy_mlp_forward(m: int, d_X, B: int, d_Y) -> None:
    _call("sy_mlp_forward", m, _ptr(d_X), B, _ptr(d_Y))


def sy_mlp_loss_grad(m: int, d_X, d_T, B: int, want_loss: bool = True) -> float | None:
    loss = C.c_float()
    _call("sy_mlp_loss_grad", m, _ptr(d_X), _ptr(d_T), B, C.byref(loss) if want_loss else None)
    return loss.value if want_loss else None


def sy_mlp_adam_step(m: int, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8) -> None:
    _call("sy_mlp_adam_step", m, lr, beta1, beta2, eps)


def sy_mlp_train(m: int, X, T, epochs: int, batch: int, lr: float, seed: int = 0) -> float:
    Xa, Ta = _f32(X), _f32(T)
    loss = C.c_float()
    _call("sy_mlp_train", m, Xa.ctypes.data, Ta.ctypes.data, Xa.shape[0], epochs, batch, lr, seed, C.byref(loss))
    return loss.value


def sy_mlp_normalization(m: int, F: int, O: int):
    import numpy as np

    xm, xs, ym, ys = (np.empty(F, np.float32), np.empty(F, np.float32), np.empty(O, np.float32),
                      np.empty(O, np.float32))
    _call("sy_mlp_normalization", m, xm.ctypes.data, xs.ctypes.data, ym.ctypes.data, ys.ctypes.data)
    return xm, xs, ym, ys


def sy_cost_model_predict(m: int, features, out_features: int = 2):
    import numpy as np

    F = _f32(features)
    pred = np.empty((F.shape[0], out_features), np.float32)
    _call("sy_cost_model_predict", m, F.ctypes.data, F.shape[0], pred.ctypes.data)
    return pred


def sy_cost_model_choose(m: int, features, objective: int = 0) -> int:
    F = _f32(features)
    best = C.c_int()
    _call("sy_cost_model_choose", m, F.ctypes.data, F.shape[0], objective, C.byref(best))
    return best.value


def sy_mlp_save(m: int, path: str) -> None:
    _call("sy_mlp_save", m, path.encode())


def sy_mlp_load(q: int, path: str) -> int:
    h = C.c_void_p()
    _call("sy_mlp_load", q, path.encode(), C.byref(h))
    return h.value


def sy_wave_run(q: int, p: StencilParams, u0, u_a, u_b, steps: int, chunks, halo_radius: int,
                want_events: bool = False):
    """Start + `steps` chunked leapfrog steps (graph-captured, cached).  Returns
    (prev_ptr, cur_ptr, events): the device addresses holding u^{steps-1} and
    u^{steps} (each equal to one of u0, u_a, u_b) and the per-chunk event ids."""
    arr, k = _chunks(chunks)
    n_ev = (steps + 1) * k
    evs = (C.c_uint64 * max(1, n_ev))() if want_events else None
    pv, cv = C.c_void_p(), C.c_void_p()
    _call("sy_wave_run", q, C.byref(p), _ptr(u0), _ptr(u_a), _ptr(u_b), steps, arr, k, halo_radius, evs,
          C.byref(pv), C.byref(cv))
    return pv.value, cv.value, (list(evs[:n_ev]) if want_events else [])


def _host_ptr(a) -> int | None:
    """Host address of a numpy array / CPU tensor / integer address / None (C-contiguous only)."""
    if a is None or isinstance(a, int):
        return a
    if hasattr(a, "ctypes"):  # numpy
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be C-contiguous")
        return a.ctypes.data
    if getattr(a, "is_cuda", False):
        raise ValueError("sy_wave_run_host takes host memory; pass device tensors to sy_wave_run")
    return _ptr(a)


def sy_wave_run_host(q: int, p: StencilParams, host_u0, host_out, steps: int, chunks, halo_radius: int,
                     host_prev_out=None, want_events: bool = False) -> list[int]:
    """sy_wave_run on host memory (numpy arrays or CPU tensors, pinned for overlap): copies
    host_u0 in, runs the start and `steps` chunked steps, copies u^{steps} into host_out (and
    u^{steps-1} into host_prev_out).  Asynchronous: results are valid after sy_queue_sync."""
    arr, k = _chunks(chunks)
    n_ev = (steps + 1) * k
    evs = (C.c_uint64 * max(1, n_ev))() if want_events else None
    _call("sy_wave_run_host", q, C.byref(p), _host_ptr(host_u0), _host_ptr(host_out), _host_ptr(host_prev_out),
          steps, arr, k, halo_radius, evs)
    return list(evs[:n_ev]) if want_events else []


def sy_chunk_energy_replay(q: int, p: StencilParams, u_prev, u_cur, u_next, chunks, c: int, halo_radius: int,
                           min_seconds: float = 1.0, min_reps: int = 20) -> dict:
    """Chunk c's step launch replayed alone in one metering window: measured J and device ms per
    launch, and the number of launches."""
    arr, k = _chunks(chunks)
    j, ms, n = C.c_double(), C.c_double(), C.c_int()
    _call("sy_chunk_energy_replay", q, C.byref(p), _ptr(u_prev), _ptr(u_cur), _ptr(u_next), arr, k, c, halo_radius,
          min_seconds, min_reps, C.byref(j), C.byref(ms), C.byref(n))
    return {"joules": j.value, "ms": ms.value, "reps": n.value}


def sy_stencil_multistep(q: int, p: StencilParams, T: int, u_prev, u_cur, out_prev, out_cur, chunks,
                         halo_radius: int, want_events: bool = False) -> list[int]:
    arr, k = _chunks(chunks)
    evs = (C.c_uint64 * max(1, k))()
    _call("sy_stencil_multistep", q, C.byref(p), T, _ptr(u_prev), _ptr(u_cur), _ptr(out_prev), _ptr(out_cur), arr,
          k, halo_radius, evs if want_events else None)
    return list(evs[:k]) if want_events else []


def sy_stencil_default_variant(radius: int, dtype: int) -> int:
    v = C.c_int()
    _call("sy_stencil_default_variant", radius, dtype, C.byref(v))
    return v.value


def sy_stencil_variant_count(radius: int, dtype: int) -> int:
    n = C.c_int()
    _call("sy_stencil_variant_count", radius, dtype, C.byref(n))
    return n.value


def sy_stencil_variant_info(radius: int, dtype: int, variant: int) -> tuple[int, int, int]:
    r, c, t = C.c_int(), C.c_int(), C.c_int()
    _call("sy_stencil_variant_info", radius, dtype, variant, C.byref(r), C.byref(c), C.byref(t))
    return r.value, c.value, t.value


def sy_wave_energy(q: int, p: StencilParams, u_new, u_old) -> tuple[float, float, float]:
    e, k, pot = C.c_double(), C.c_double(), C.c_double()
    _call("sy_wave_energy", q, C.byref(p), _ptr(u_new), _ptr(u_old), C.byref(e), C.byref(k), C.byref(pot))
    return e.value, k.value, pot.value


# ---------------------------------------------------------------------------
# Convenience: a queue object bound to torch's current stream
# ---------------------------------------------------------------------------

class Queue:
    """sy_queue on a CUDA device; borrows `stream` (a torch.cuda.Stream or raw
    cudaStream_t) or torch's current stream when None."""

    def __init__(self, device: int = 0, stream=None):
        import torch

        if stream is None:
            stream = torch.cuda.current_stream(device)
        raw = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        # torch reports its default (legacy) stream as handle 0; NULL would ask the
        # library for a private stream, so name the legacy stream explicitly.
        self.handle = sy_queue_create(device, raw if raw else SY_STREAM_LEGACY)
        self.device = device

    def close(self) -> None:
        if self.handle:
            sy_queue_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sync(self) -> None:
        sy_queue_sync(self.handle)

    @property
    def launches(self) -> int:
        return sy_queue_launch_count(self.handle)


# ---- energy targets by frequency scaling ------------------------------------------

def sy_clock_choose(target: int, points) -> int:
    """Index of the (sm_mhz, seconds, joules) point minimising the target's objective."""
    arr = (FreqPoint * max(1, len(points)))(*[FreqPoint(int(f), float(t), float(j)) for f, t, j in points])
    idx = C.c_int(-1)
    _call("sy_clock_choose", int(target), arr, len(points), C.byref(idx))
    return idx.value


def sy_clock_nvml_index(cuda_device: int) -> int:
    out = C.c_uint32(0)
    _call("sy_clock_nvml_index", int(cuda_device), C.byref(out))
    return out.value


def sy_clock_supported(nvml_index: int) -> tuple[int, list[int]]:
    """(memory clock, supported SM clocks highest first), read-only."""
    mem, n = C.c_uint32(0), C.c_int(0)
    _call("sy_clock_supported", int(nvml_index), C.byref(mem), None, 0, C.byref(n))
    buf = (C.c_uint32 * max(1, n.value))()
    _call("sy_clock_supported", int(nvml_index), C.byref(mem), buf, n.value, C.byref(n))
    return mem.value, list(buf[: n.value])


def sy_clock_current(nvml_index: int) -> tuple[int, int]:
    cur, mx = C.c_uint32(0), C.c_uint32(0)
    _call("sy_clock_current", int(nvml_index), C.byref(cur), C.byref(mx))
    return cur.value, mx.value


def sy_clock_lock(nvml_index: int, sm_mhz: int) -> None:
    _call("sy_clock_lock", int(nvml_index), int(sm_mhz))


def sy_clock_unlock(nvml_index: int) -> None:
    _call("sy_clock_unlock", int(nvml_index))


def sy_clock_sweep(nvml_index: int, candidates, measure, target: int = SY_TARGET_MIN_EDP):
    """Lock each candidate SM clock in turn, call measure(sm_mhz) -> (seconds, joules), release
    the lock, and choose by target.  Returns (best index, [(sm_mhz, seconds, joules), ...])."""
    def cb(_ctx, mhz, t_out, j_out):
        try:
            t, j = measure(int(mhz))
            t_out[0], j_out[0] = float(t), float(j)
            return 0
        except Exception:  # reported to the library as a failed measurement
            return 1

    fn = MEASURE_FN(cb)
    n = len(candidates)
    freqs = (C.c_uint32 * max(1, n))(*[int(f) for f in candidates])
    pts = (FreqPoint * max(1, n))()
    best = C.c_int(-1)
    _call("sy_clock_sweep", int(nvml_index), freqs, n, fn, None, int(target), pts, C.byref(best))
    return best.value, [(p.sm_mhz, p.seconds, p.joules) for p in pts[:n]]


# ---- 3D leapfrog (chunks of planes) --------------------------------------------------

def stencil3d_params(nz: int, ny: int, nx: int, radius: int, c2: float, dtype: str = "f32", pitch: int | None = None,
                     plane: int | None = None, variant: int = 0) -> Stencil3dParams:
    pitch = nx if pitch is None else pitch
    plane = ny * pitch if plane is None else plane
    return Stencil3dParams(nz, ny, nx, pitch, plane, radius, DTYPE_CODES[dtype], c2, variant)


def sy_stencil3d_step(q: int, p: Stencil3dParams, u_prev, u_cur, u_next, chunks, halo_radius: int,
                      want_events: bool = False) -> list[int]:
    arr, k = _chunks(chunks)
    evs = (C.c_uint64 * max(1, k))()
    _call("sy_stencil3d_step", q, C.byref(p), _ptr(u_prev), _ptr(u_cur), _ptr(u_next), arr, k, halo_radius,
          evs if want_events else None)
    return list(evs[:k]) if want_events else []


def sy_stencil3d_start(q: int, p: Stencil3dParams, u0, u_m1, chunks, halo_radius: int,
                       want_events: bool = False) -> list[int]:
    arr, k = _chunks(chunks)
    evs = (C.c_uint64 * max(1, k))()
    _call("sy_stencil3d_start", q, C.byref(p), _ptr(u0), _ptr(u_m1), arr, k, halo_radius,
          evs if want_events else None)
    return list(evs[:k]) if want_events else []


def sy_stencil3d_step_planes(q: int, p: Stencil3dParams, u_prev, u_cur, u_next, plane_begin: int, plane_end: int,
                             halo_radius: int, start: bool = False) -> None:
    _call("sy_stencil3d_step_planes", q, C.byref(p), _ptr(u_prev), _ptr(u_cur), _ptr(u_next), int(plane_begin),
          int(plane_end), halo_radius, 1 if start else 0, None)


def sy_wave3d_run(q: int, p: Stencil3dParams, u0, u_a, u_b, steps: int, chunks, halo_radius: int,
                  want_events: bool = False):
    """Start + `steps` steps as one cached graph: (prev_ptr, cur_ptr, events), as sy_wave_run."""
    arr, k = _chunks(chunks)
    n_ev = (steps + 1) * k
    evs = (C.c_uint64 * max(1, n_ev))() if want_events else None
    pv, cv = C.c_void_p(), C.c_void_p()
    _call("sy_wave3d_run", q, C.byref(p), _ptr(u0), _ptr(u_a), _ptr(u_b), steps, arr, k, halo_radius, evs,
          C.byref(pv), C.byref(cv))
    return pv.value, cv.value, (list(evs[:n_ev]) if want_events else [])


def sy_wave3d_energy(q: int, p: Stencil3dParams, u_new, u_old) -> tuple[float, float, float]:
    """(E, kinetic, potential) of the 3D scheme, FP64, fixed reduction shape."""
    e, k, pt = C.c_double(), C.c_double(), C.c_double()
    _call("sy_wave3d_energy", q, C.byref(p), _ptr(u_new), _ptr(u_old), C.byref(e), C.byref(k), C.byref(pt))
    return e.value, k.value, pt.value


def sy_stencil3d_variant_count(radius: int, dtype: str = "f32") -> int:
    n = C.c_int(0)
    _call("sy_stencil3d_variant_count", radius, DTYPE_CODES[dtype], C.byref(n))
    return n.value


def sy_stencil3d_variant_info(radius: int, dtype: str, variant: int) -> tuple[int, int]:
    rows, thr = C.c_int(0), C.c_int(0)
    _call("sy_stencil3d_variant_info", radius, DTYPE_CODES[dtype], variant, C.byref(rows), C.byref(thr))
    return rows.value, thr.value


# ---- range mappers on boxes ---------------------------------------------------------

def _mk_box(b) -> Box:
    (l0, l1, l2), (h0, h1, h2) = b
    return Box((C.c_int64 * 3)(l0, l1, l2), (C.c_int64 * 3)(h0, h1, h2))


def _unbox(b: Box) -> tuple:
    return (tuple(b.lo), tuple(b.hi))


def range_mapper(kind: int, radius=(0, 0, 0), dim: int = 0, fixed=((0, 0, 0), (0, 0, 0))) -> RangeMapper:
    return RangeMapper(kind, dim, (C.c_int64 * 3)(*radius), _mk_box(fixed))


def sy_rm_box(rm: RangeMapper, chunk, extent) -> tuple:
    out = Box()
    _call("sy_rm_box", C.byref(rm), C.byref(_mk_box(chunk)), (C.c_int64 * 3)(*extent), C.byref(out))
    return _unbox(out)


def sy_rm_box_transfers(rm: RangeMapper, chunks, extent) -> list:
    """[(src, dst, box)] in dst-major, src-minor order."""
    arr = (Box * max(1, len(chunks)))(*[_mk_box(c) for c in chunks])
    n = C.c_int(0)
    ext = (C.c_int64 * 3)(*extent)
    L = lib()
    rc = L.sy_rm_box_transfers(C.byref(rm), arr, len(chunks), ext, None, 0, C.byref(n))
    if rc not in (0, 1) or (rc == 1 and n.value == 0):
        raise SyError(rc, L.sy_last_error().decode(errors="replace"))
    out = (BoxTransfer * max(1, n.value))()
    _call("sy_rm_box_transfers", C.byref(rm), arr, len(chunks), ext, out, n.value, C.byref(n))
    return [(t.src, t.dst, _unbox(t.box)) for t in out[: n.value]]


SY_TUNE_SAXPY, SY_TUNE_STENCIL, SY_TUNE_STENCIL3D = 0, 1, 2


def sy_tune_exhaustive(q: int, kind: int, params, n: int, in0, in1, out_buf, chunk_counts, reps: int = 3):
    """Every candidate of one kernel kind timed on the caller's buffers: (records, best index),
    records as (variant, tile_rows, tile_cols, threads, chunks, ms)."""
    counts = (C.c_int * max(1, len(chunk_counts)))(*chunk_counts)
    cap = 64 * max(1, len(chunk_counts))
    recs = (TuneRecord * cap)()
    n_out, best = C.c_int(0), C.c_int(-1)
    _call("sy_tune_exhaustive", q, int(kind), None if params is None else C.byref(params), int(n), _ptr(in0),
          _ptr(in1), _ptr(out_buf), counts, len(chunk_counts), int(reps), recs, cap, C.byref(n_out), C.byref(best))
    return [(r.variant, r.tile_rows, r.tile_cols, r.threads, r.chunks, r.ms) for r in recs[: n_out.value]], best.value


def sy_mlp_backward(m, d_X, d_T, B: int, want_loss: bool = True):
    loss = C.c_float(0.0)
    _call("sy_mlp_backward", m, _ptr(d_X), _ptr(d_T), int(B), C.byref(loss) if want_loss else None)
    return loss.value if want_loss else None


class ChunkStats(C.Structure):
    _fields_ = [("ms", C.c_double), ("bytes", C.c_double), ("joules", C.c_double), ("updates", C.c_double)]


def sy_chunk_stats_read(q: int, p: StencilParams, chunks, events) -> list[dict]:
    """Per chunk: device ms, algorithmic bytes, joules (-1 outside a closed metering window), updates."""
    arr, k = _chunks(chunks)
    evs = (C.c_uint64 * max(1, k))(*events)
    out = (ChunkStats * max(1, k))()
    _call("sy_chunk_stats_read", q, C.byref(p), arr, evs, k, out)
    return [{"ms": s.ms, "bytes": s.bytes, "joules": s.joules, "updates": s.updates} for s in out[:k]]


def sy_checkpoint_save(q: int, path: str, p: StencilParams, u_prev, u_cur, step: int) -> None:
    _call("sy_checkpoint_save", q, path.encode(), C.byref(p), _ptr(u_prev), _ptr(u_cur), int(step))


def sy_checkpoint_load(q: int, path: str, p: StencilParams, u_prev, u_cur) -> int:
    step = C.c_int64(0)
    _call("sy_checkpoint_load", q, path.encode(), C.byref(p), _ptr(u_prev), _ptr(u_cur), C.byref(step))
    return step.value
