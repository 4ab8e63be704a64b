"""Helpers for the GPU parity tests: upload/download of seeded inputs and a
driver for multi-step wave runs through the C ABI (argument marshalling only)."""
from __future__ import annotations

import numpy as np
import pytest

import paper_2505_06022_gb300 as sy


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("a test marked gpu ran without a CUDA device")
    return torch


def to_device(a: np.ndarray, pitch: int | None = None, fill=None):
    """Upload a 2D float32 or uint16 array; optional padded pitch (padding = fill bits)."""
    torch = torch_cuda()
    if a.dtype == np.uint16:
        host = torch.from_numpy(a.view(np.int16).copy())
    else:
        host = torch.from_numpy(np.ascontiguousarray(a))
    if a.ndim == 2 and pitch is not None and pitch != a.shape[1]:
        buf = torch.empty((a.shape[0], pitch), dtype=host.dtype)
        if fill is not None:
            buf.fill_(fill)
        else:
            buf.zero_()
        buf[:, : a.shape[1]] = host
        host = buf
    return host.cuda()


def to_host(t, shape=None, storage=np.float32) -> np.ndarray:
    a = t.cpu().numpy()
    if storage == np.uint16:
        a = a.view(np.uint16)
    if shape is not None and a.ndim == 2 and a.shape[1] != shape[1]:
        a = np.ascontiguousarray(a[:, : shape[1]])
    return a


def wave_run(q, u0: np.ndarray, steps: int, r: int, c2: float, dtype: str, chunks, variant: int = 0,
             halo: int | None = None, pitch: int | None = None):
    """Taylor start + `steps` leapfrog steps on the GPU; returns (u^{steps-1}, u^{steps}) on the host."""
    torch = torch_cuda()
    ny, nx = u0.shape
    cur = to_device(u0, pitch)
    prev = torch.empty_like(cur)
    p = sy.stencil_params(ny, nx, r, c2, dtype, pitch=pitch or nx, variant=variant)
    halo = r if halo is None else halo
    sy.sy_stencil_start(q, p, cur, prev, chunks, halo)
    for _ in range(steps):
        sy.sy_stencil_step(q, p, prev, cur, prev, chunks, halo)
        prev, cur = cur, prev
    torch.cuda.synchronize()
    st = np.uint16 if dtype != "f32" else np.float32
    return to_host(prev, u0.shape, st), to_host(cur, u0.shape, st)


def bits(a: np.ndarray) -> np.ndarray:
    return a.view(np.uint32) if a.dtype == np.float32 else a.view(np.uint16)
