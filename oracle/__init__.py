"""Python face of the CPU oracle (liboracle.so, built from oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and by
the CPU-baseline leg of bench.py.  The product package never imports it.

All arrays are numpy, C-contiguous.  Storage dtypes for the precision mirror are
numpy float32 (FP32) or uint16 bit patterns (BF16, FP16).  See oracle.c for the
definitions and the paper passages each routine follows.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

F32, BF16, F16 = 0, 1, 2
DTYPES = {"f32": F32, "bf16": BF16, "f16": F16}

_lib = None

_p = C.c_void_p
_i64 = C.c_int64


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        sig = {
            "oracle_threads": (C.c_int, []),
            "oracle_set_threads": (None, [C.c_int]),
            "oracle_saxpy_f32": (None, [_i64, C.c_float, _p, _p, _p]),
            "oracle_saxpy_f64": (None, [_i64, C.c_double, _p, _p, _p]),
            "oracle_split_rows": (C.c_int, [_i64, C.c_int, _p]),
            "oracle_rm_one_to_one": (None, [_i64, _i64, _p, _p]),
            "oracle_rm_neighbourhood": (None, [_i64, _i64, C.c_int, _i64, _p, _p]),
            "oracle_chunks_valid": (C.c_int, [_i64, _p, C.c_int]),
            "oracle_d2_weights": (C.c_int, [C.c_int, _p]),
            "oracle_wave_step_f64": (C.c_int, [_i64, _i64, C.c_int, C.c_double, _p, _p, _p]),
            "oracle_wave_start_f64": (C.c_int, [_i64, _i64, C.c_int, C.c_double, _p, _p]),
            "oracle_wave_run_f64": (C.c_int, [_i64, _i64, C.c_int, C.c_double, _i64, _p, _p, _p]),
            "oracle_f32_to_bf16": (C.c_uint16, [C.c_float]),
            "oracle_bf16_to_f32": (C.c_float, [C.c_uint16]),
            "oracle_f32_to_f16": (C.c_uint16, [C.c_float]),
            "oracle_f16_to_f32": (C.c_float, [C.c_uint16]),
            "oracle_wave_step_mirror": (C.c_int, [C.c_int, _i64, _i64, C.c_int, C.c_float, _p, _p, _p]),
            "oracle_wave_start_mirror": (C.c_int, [C.c_int, _i64, _i64, C.c_int, C.c_float, _p, _p]),
            "oracle_wave_run_mirror": (C.c_int, [C.c_int, _i64, _i64, C.c_int, C.c_float, _i64, _p, _p, _p]),
            "oracle_wave_energy_f64": (C.c_double, [_i64, _i64, C.c_int, C.c_double, _p, _p, _p, _p, _p]),
            "oracle_mlp_param_count": (_i64, [C.c_int, C.c_int, C.c_int]),
            "oracle_mlp_forward": (C.c_int, [_i64, C.c_int, C.c_int, C.c_int, _p, _p, _p]),
            "oracle_mlp_loss_grad": (C.c_double, [_i64, C.c_int, C.c_int, C.c_int, _p, _p, _p, _p]),
            "oracle_wave3d_step_f64": (C.c_int, [_i64, _i64, _i64, C.c_int, C.c_double, _p, _p, _p]),
            "oracle_wave3d_start_f64": (C.c_int, [_i64, _i64, _i64, C.c_int, C.c_double, _p, _p]),
            "oracle_wave3d_run_f64": (C.c_int, [_i64, _i64, _i64, C.c_int, C.c_double, _i64, _p, _p, _p]),
            "oracle_wave3d_step_mirror": (C.c_int, [C.c_int, _i64, _i64, _i64, C.c_int, C.c_float, _p, _p, _p]),
            "oracle_wave3d_start_mirror": (C.c_int, [C.c_int, _i64, _i64, _i64, C.c_int, C.c_float, _p, _p]),
            "oracle_wave3d_run_mirror": (C.c_int, [C.c_int, _i64, _i64, _i64, C.c_int, C.c_float, _i64, _p, _p,
                                                   _p]),
            "oracle_wave3d_energy_f64": (C.c_double, [_i64, _i64, _i64, C.c_int, C.c_double, _p, _p, _p, _p]),
            "oracle_rm_box": (C.c_int, [C.c_int, _p, C.c_int, _p, _p, _p, _p]),
            "oracle_rm_box_transfers": (C.c_int, [C.c_int, _p, C.c_int, _p, _p, C.c_int, _p, _p, C.c_int]),
            "oracle_adam_step": (None, [_i64, _p, _p, _p, _p, _i64, C.c_double, C.c_double, C.c_double,
                                        C.c_double]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    return a.ctypes.data


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


def threads() -> int:
    return lib().oracle_threads()


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


# --- 1. SAXPY (paper §2 Listing 1) -----------------------------------------

def saxpy_f32(alpha: float, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float32)
    y = np.ascontiguousarray(y, np.float32)
    z = np.empty_like(x)
    lib().oracle_saxpy_f32(x.size, float(np.float32(alpha)), _ptr(x), _ptr(y), _ptr(z))
    return z


def saxpy_f64(alpha: float, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    z = np.empty_like(x)
    lib().oracle_saxpy_f64(x.size, float(alpha), _ptr(x), _ptr(y), _ptr(z))
    return z


# --- 2. Range mappers (paper §3) -------------------------------------------

def split_rows(ny: int, k: int) -> list[tuple[int, int]]:
    out = np.zeros(2 * k, np.int64)
    _check(lib().oracle_split_rows(ny, k, _ptr(out)), "split_rows")
    return [(int(out[2 * c]), int(out[2 * c + 1])) for c in range(k)]


def rm_one_to_one(a: int, b: int) -> tuple[int, int]:
    lo, hi = C.c_int64(), C.c_int64()
    lib().oracle_rm_one_to_one(a, b, C.addressof(lo), C.addressof(hi))
    return lo.value, hi.value


def rm_neighbourhood(a: int, b: int, r: int, ny: int) -> tuple[int, int]:
    lo, hi = C.c_int64(), C.c_int64()
    lib().oracle_rm_neighbourhood(a, b, r, ny, C.addressof(lo), C.addressof(hi))
    return lo.value, hi.value


def chunks_valid(ny: int, chunks) -> bool:
    arr = np.asarray(chunks, np.int64).reshape(-1)
    return bool(lib().oracle_chunks_valid(ny, _ptr(np.ascontiguousarray(arr)), len(arr) // 2))


# --- 3. Weights --------------------------------------------------------------

def d2_weights(r: int) -> np.ndarray:
    """[w_0, w_1, ..., w_r] of the order-2r central second difference."""
    w = np.zeros(5, np.float64)
    _check(lib().oracle_d2_weights(r, _ptr(w)), "d2_weights")
    return w[: r + 1].copy()


# --- 4. FP64 wave -------------------------------------------------------------

def wave_step_f64(u_prev: np.ndarray, u_cur: np.ndarray, r: int, c2: float) -> np.ndarray:
    up = np.ascontiguousarray(u_prev, np.float64)
    uc = np.ascontiguousarray(u_cur, np.float64)
    ny, nx = uc.shape
    un = np.empty_like(uc)
    _check(lib().oracle_wave_step_f64(ny, nx, r, c2, _ptr(up), _ptr(uc), _ptr(un)), "wave_step_f64")
    return un


def wave_start_f64(u0: np.ndarray, r: int, c2: float) -> np.ndarray:
    u0 = np.ascontiguousarray(u0, np.float64)
    ny, nx = u0.shape
    um1 = np.empty_like(u0)
    _check(lib().oracle_wave_start_f64(ny, nx, r, c2, _ptr(u0), _ptr(um1)), "wave_start_f64")
    return um1


def wave_run_f64(u0: np.ndarray, steps: int, r: int, c2: float) -> tuple[np.ndarray, np.ndarray]:
    """Taylor start and `steps` leapfrog steps: returns (u^{steps-1}, u^{steps})."""
    u0 = np.ascontiguousarray(u0, np.float64)
    ny, nx = u0.shape
    prev = np.empty_like(u0)
    cur = np.empty_like(u0)
    _check(lib().oracle_wave_run_f64(ny, nx, r, c2, steps, _ptr(u0), _ptr(prev), _ptr(cur)), "wave_run_f64")
    return prev, cur


# --- 5. Precision mirror -------------------------------------------------------

def _storage(a: np.ndarray, dtype: int) -> np.ndarray:
    want = np.float32 if dtype == F32 else np.uint16
    if a.dtype != want:
        raise TypeError(f"mirror storage for dtype {dtype} must be {np.dtype(want).name}, got {a.dtype}")
    return np.ascontiguousarray(a)


def wave_step_mirror(dtype: int, u_prev: np.ndarray, u_cur: np.ndarray, r: int, c2: float) -> np.ndarray:
    up, uc = _storage(u_prev, dtype), _storage(u_cur, dtype)
    ny, nx = uc.shape
    un = np.empty_like(uc)
    _check(lib().oracle_wave_step_mirror(dtype, ny, nx, r, c2, _ptr(up), _ptr(uc), _ptr(un)), "wave_step_mirror")
    return un


def wave_start_mirror(dtype: int, u0: np.ndarray, r: int, c2: float) -> np.ndarray:
    u0 = _storage(u0, dtype)
    ny, nx = u0.shape
    um1 = np.empty_like(u0)
    _check(lib().oracle_wave_start_mirror(dtype, ny, nx, r, c2, _ptr(u0), _ptr(um1)), "wave_start_mirror")
    return um1


def wave_run_mirror(dtype: int, u0: np.ndarray, steps: int, r: int, c2: float) -> tuple[np.ndarray, np.ndarray]:
    u0 = _storage(u0, dtype)
    ny, nx = u0.shape
    prev = np.empty_like(u0)
    cur = np.empty_like(u0)
    _check(lib().oracle_wave_run_mirror(dtype, ny, nx, r, c2, steps, _ptr(u0), _ptr(prev), _ptr(cur)),
           "wave_run_mirror")
    return prev, cur


def f32_to_bf16(values: np.ndarray) -> np.ndarray:
    L = lib()
    flat = np.asarray(values, np.float32).reshape(-1)
    return np.array([L.oracle_f32_to_bf16(float(v)) for v in flat], np.uint16).reshape(np.shape(values))


def f32_to_f16(values: np.ndarray) -> np.ndarray:
    L = lib()
    flat = np.asarray(values, np.float32).reshape(-1)
    return np.array([L.oracle_f32_to_f16(float(v)) for v in flat], np.uint16).reshape(np.shape(values))


def bf16_to_f32(bits: np.ndarray) -> np.ndarray:
    L = lib()
    flat = np.asarray(bits, np.uint16).reshape(-1)
    return np.array([L.oracle_bf16_to_f32(int(b)) for b in flat], np.float32).reshape(np.shape(bits))


def f16_to_f32(bits: np.ndarray) -> np.ndarray:
    L = lib()
    flat = np.asarray(bits, np.uint16).reshape(-1)
    return np.array([L.oracle_f16_to_f32(int(b)) for b in flat], np.float32).reshape(np.shape(bits))


def storage_to_f64(a: np.ndarray, dtype: int) -> np.ndarray:
    """Widen a mirror storage array to float64 (exact)."""
    if dtype == F32:
        return a.astype(np.float64)
    if dtype == BF16:
        return (a.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    return f16_bits_to_f64_fast(a)


def f16_bits_to_f64_fast(a: np.ndarray) -> np.ndarray:
    """Exact widening of binary16 bit patterns, by the format's definition."""
    a = np.asarray(a, np.uint16)
    sign = np.where((a >> 15) & 1, -1.0, 1.0)
    E = ((a >> 10) & 0x1F).astype(np.int64)
    mant = (a & 0x3FF).astype(np.float64)
    normal = np.ldexp(1.0 + mant / 1024.0, (E - 15).astype(np.int32))
    sub = np.ldexp(mant, -24)
    v = np.where(E == 0, sub, normal)
    v = np.where(E == 31, np.where(mant > 0, np.nan, np.inf), v)
    return sign * v


# --- 6. Energy -----------------------------------------------------------------

def wave_energy_f64(u_new: np.ndarray, u_old: np.ndarray, r: int, c2: float) -> dict:
    un = np.ascontiguousarray(u_new, np.float64)
    uo = np.ascontiguousarray(u_old, np.float64)
    ny, nx = un.shape
    kin, pot, mag = C.c_double(), C.c_double(), C.c_double()
    E = lib().oracle_wave_energy_f64(ny, nx, r, c2, _ptr(un), _ptr(uo), C.addressof(kin), C.addressof(pot),
                                     C.addressof(mag))
    return {"E": E, "kin": kin.value, "pot": pot.value, "abs_sum": mag.value}


# --- 8. 3D leapfrog --------------------------------------------------------------

def wave3d_step_f64(u_prev: np.ndarray, u_cur: np.ndarray, r: int, c2: float) -> np.ndarray:
    up = np.ascontiguousarray(u_prev, np.float64)
    uc = np.ascontiguousarray(u_cur, np.float64)
    nz, ny, nx = uc.shape
    un = np.empty_like(uc)
    _check(lib().oracle_wave3d_step_f64(nz, ny, nx, r, c2, _ptr(up), _ptr(uc), _ptr(un)), "wave3d_step_f64")
    return un


def wave3d_start_f64(u0: np.ndarray, r: int, c2: float) -> np.ndarray:
    u0 = np.ascontiguousarray(u0, np.float64)
    nz, ny, nx = u0.shape
    um1 = np.empty_like(u0)
    _check(lib().oracle_wave3d_start_f64(nz, ny, nx, r, c2, _ptr(u0), _ptr(um1)), "wave3d_start_f64")
    return um1


def wave3d_run_f64(u0: np.ndarray, steps: int, r: int, c2: float) -> tuple[np.ndarray, np.ndarray]:
    u0 = np.ascontiguousarray(u0, np.float64)
    nz, ny, nx = u0.shape
    prev, cur = np.empty_like(u0), np.empty_like(u0)
    _check(lib().oracle_wave3d_run_f64(nz, ny, nx, r, c2, steps, _ptr(u0), _ptr(prev), _ptr(cur)), "wave3d_run_f64")
    return prev, cur


def wave3d_step_mirror(dtype: int, u_prev: np.ndarray, u_cur: np.ndarray, r: int, c2: float) -> np.ndarray:
    up, uc = _storage(u_prev, dtype), _storage(u_cur, dtype)
    nz, ny, nx = uc.shape
    un = np.empty_like(uc)
    _check(lib().oracle_wave3d_step_mirror(dtype, nz, ny, nx, r, c2, _ptr(up), _ptr(uc), _ptr(un)),
           "wave3d_step_mirror")
    return un


def wave3d_start_mirror(dtype: int, u0: np.ndarray, r: int, c2: float) -> np.ndarray:
    u0 = _storage(u0, dtype)
    nz, ny, nx = u0.shape
    um1 = np.empty_like(u0)
    _check(lib().oracle_wave3d_start_mirror(dtype, nz, ny, nx, r, c2, _ptr(u0), _ptr(um1)), "wave3d_start_mirror")
    return um1


def wave3d_run_mirror(dtype: int, u0: np.ndarray, steps: int, r: int, c2: float) -> tuple[np.ndarray, np.ndarray]:
    u0 = _storage(u0, dtype)
    nz, ny, nx = u0.shape
    prev, cur = np.empty_like(u0), np.empty_like(u0)
    _check(lib().oracle_wave3d_run_mirror(dtype, nz, ny, nx, r, c2, steps, _ptr(u0), _ptr(prev), _ptr(cur)),
           "wave3d_run_mirror")
    return prev, cur


def wave3d_energy_f64(u_new: np.ndarray, u_old: np.ndarray, r: int, c2: float) -> dict:
    un = np.ascontiguousarray(u_new, np.float64)
    uo = np.ascontiguousarray(u_old, np.float64)
    nz, ny, nx = un.shape
    kin, pot = C.c_double(), C.c_double()
    E = lib().oracle_wave3d_energy_f64(nz, ny, nx, r, c2, _ptr(un), _ptr(uo), C.addressof(kin), C.addressof(pot))
    return {"E": E, "kin": kin.value, "pot": pot.value}


# --- 9. Range mappers on boxes ---------------------------------------------------

RM_ONE_TO_ONE, RM_NEIGHBOURHOOD, RM_SLICE, RM_ALL, RM_FIXED = 0, 1, 2, 3, 4


def _box(b) -> np.ndarray:
    """((lo0, lo1, lo2), (hi0, hi1, hi2)) -> int64[6]."""
    (l0, l1, l2), (h0, h1, h2) = b
    return np.array([l0, l1, l2, h0, h1, h2], np.int64)


def _unbox(a) -> tuple:
    return (tuple(int(v) for v in a[:3]), tuple(int(v) for v in a[3:6]))


def rm_box(kind: int, chunk, extent, radius=(0, 0, 0), dim: int = 0, fixed=((0, 0, 0), (0, 0, 0))) -> tuple:
    rad = np.array(radius, np.int64)
    fx, ch, out = _box(fixed), _box(chunk), np.zeros(6, np.int64)
    ext = np.array(extent, np.int64)
    _check(lib().oracle_rm_box(kind, _ptr(rad), dim, _ptr(fx), _ptr(ch), _ptr(ext), _ptr(out)), "rm_box")
    return _unbox(out)


def rm_box_transfers(kind: int, chunks, extent, radius=(0, 0, 0), dim: int = 0,
                     fixed=((0, 0, 0), (0, 0, 0))) -> list:
    """[(src, dst, box)] in dst-major, src-minor order."""
    rad = np.array(radius, np.int64)
    fx = _box(fixed)
    ch = np.ascontiguousarray(np.concatenate([_box(c) for c in chunks]) if chunks else np.zeros(6, np.int64))
    ext = np.array(extent, np.int64)
    cap = max(1, len(chunks) * len(chunks))
    out = np.zeros(8 * cap, np.int64)
    n = lib().oracle_rm_box_transfers(kind, _ptr(rad), dim, _ptr(fx), _ptr(ch), len(chunks), _ptr(ext), _ptr(out),
                                      cap)
    if n < 0:
        raise ValueError("oracle rm_box_transfers failed")
    return [(int(out[8 * t]), int(out[8 * t + 1]), _unbox(out[8 * t + 2: 8 * t + 8])) for t in range(n)]


# --- 7. MLP --------------------------------------------------------------------

def mlp_param_count(F: int, H: int, O: int) -> int:
    return int(lib().oracle_mlp_param_count(F, H, O))


def mlp_forward(X: np.ndarray, params: np.ndarray, F: int, H: int, O: int) -> np.ndarray:
    X = np.ascontiguousarray(X, np.float64)
    p = np.ascontiguousarray(params, np.float64)
    B = X.shape[0]
    Y = np.empty((B, O), np.float64)
    _check(lib().oracle_mlp_forward(B, F, H, O, _ptr(X), _ptr(p), _ptr(Y)), "mlp_forward")
    return Y


def mlp_loss_grad(X: np.ndarray, T: np.ndarray, params: np.ndarray, F: int, H: int, O: int):
    X = np.ascontiguousarray(X, np.float64)
    T = np.ascontiguousarray(T, np.float64)
    p = np.ascontiguousarray(params, np.float64)
    g = np.empty_like(p)
    loss = lib().oracle_mlp_loss_grad(X.shape[0], F, H, O, _ptr(X), _ptr(T), _ptr(p), _ptr(g))
    return float(loss), g


def adam_step(params, grad, m, v, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8) -> None:
    """In place on float64 arrays params, m, v."""
    for a in (params, m, v):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    g = np.ascontiguousarray(grad, np.float64)
    lib().oracle_adam_step(params.size, _ptr(params), _ptr(g), _ptr(m), _ptr(v), t, lr, beta1, beta2, eps)


def lib_path() -> str:
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "liboracle.so")
