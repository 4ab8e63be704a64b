"""Chunks on separate ranks (one per GPU): the paper's split of a kernel across
devices (§3) with the data transfers inferred from the neighbourhood range
mapper.

Rank k holds chunk k of the row split (of the plane split, for the 3D grid) in a
buffer of its own (the split-buffer layout: halo_lo rows or planes before its
own, halo_hi after).  Before every step the
halo rows of u^n are exchanged with point-to-point messages
(torch.distributed batch_isend_irecv: NCCL between GPUs, gloo between CPU
processes); which rows go where is `sy_rm_transfers`, the same inference the
single-GPU split-buffer mode uses.  The step itself is the library's kernel on
the rank's own rows (`sy_stencil_step_rows`).
"""
from __future__ import annotations

from typing import Callable

from . import (stencil3d_params, stencil_params, sy_rm_transfers, sy_split_layout, sy_split_rows,
               sy_stencil3d_step_planes, sy_stencil_step_rows)


class RankChunk:
    """Halo exchange and stepping for this rank's chunk of an ny x nx grid."""

    def __init__(self, ny: int, nx: int, radius: int, halo: int, rank: int, world: int, pitch: int | None = None):
        if halo < radius:
            raise ValueError("halo radius must be >= stencil radius")
        self.ny, self.nx, self.radius, self.halo = ny, nx, radius, halo
        self.rank, self.world = rank, world
        self.pitch = pitch or nx
        self.chunks = sy_split_rows(ny, world)
        self.layout = [sy_split_layout(ny, self.chunks, halo, c) for c in range(world)]
        self.halo_lo, self.halo_hi, self.rows = self.layout[rank]
        self.own = (self.halo_lo, self.halo_lo + self.chunks[rank][1] - self.chunks[rank][0])
        self.transfers = sy_rm_transfers(ny, self.chunks, halo)

    def local_row(self, chunk: int, global_row: int) -> int:
        return global_row - self.chunks[chunk][0] + self.layout[chunk][0]

    def exchange(self, local, dist) -> None:
        """Fill this rank's halo rows of `local` (rows x pitch tensor) from their owners
        and send the rows others need."""
        ops = []
        for src, dst, r0, r1 in self.transfers:
            if src == self.rank and dst != self.rank:
                a = self.local_row(src, r0)
                ops.append(dist.P2POp(dist.isend, local[a: a + (r1 - r0)].contiguous(), dst))
            elif dst == self.rank and src != self.rank:
                a = self.local_row(dst, r0)
                ops.append(dist.P2POp(dist.irecv, local[a: a + (r1 - r0)], src))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()

    def step(self, prev, cur, nxt, dist, step_fn: Callable | None = None, start: bool = False) -> None:
        """One leapfrog step (or the Taylor start) of this rank's rows: exchange the halos of
        `cur`, then step.  step_fn(prev, cur, nxt, row_begin, row_end, start) replaces the
        GPU kernel when given (CPU tests of the exchange)."""
        self.exchange(cur, dist)
        if step_fn is not None:
            step_fn(prev, cur, nxt, self.own[0], self.own[1], start)
            return
        raise RuntimeError("use GpuRankChunk for the GPU step")


class GpuRankChunk(RankChunk):
    """RankChunk stepping with the library's CUDA kernel on this rank's GPU.

    The queue must issue on torch's current stream (what sy.Queue borrows by default):
    the exchange's NCCL sends are ordered after the work already on that stream, and
    waiting on its receives orders that stream after them, so the step's kernel reads
    the new halo rows and the next exchange sends finished ones."""

    def __init__(self, queue, c2: float, dtype: str = "f32", **kw):
        super().__init__(**kw)
        self.q = queue
        self.params = stencil_params(self.rows, self.nx, self.radius, c2, dtype, pitch=self.pitch)

    def step(self, prev, cur, nxt, dist, step_fn=None, start: bool = False) -> None:
        self.exchange(cur, dist)
        sy_stencil_step_rows(self.q.handle, self.params, None if start else prev, cur, nxt, self.own[0],
                             self.own[1], self.halo, start=start)


class GpuRankChunk3d(RankChunk):
    """The 3D grid split into chunks of planes, one per rank: the same exchange along
    dimension 0 (whole planes), stepping with the library's 3D kernel on this rank's
    planes.  Local buffers are (planes, ny, pitch) tensors.  The queue issues on torch's
    current stream, as for GpuRankChunk."""

    def __init__(self, queue, nz: int, ny: int, nx: int, radius: int, halo: int, rank: int, world: int, c2: float,
                 dtype: str = "f32", pitch: int | None = None):
        super().__init__(ny=nz, nx=nx, radius=radius, halo=halo, rank=rank, world=world, pitch=pitch)
        self.nz, self.ny3 = nz, ny
        self.q = queue
        self.params = stencil3d_params(self.rows, ny, nx, radius, c2, dtype, pitch=self.pitch)

    def step(self, prev, cur, nxt, dist, step_fn=None, start: bool = False) -> None:
        self.exchange(cur, dist)
        if step_fn is not None:
            step_fn(prev, cur, nxt, self.own[0], self.own[1], start)
            return
        sy_stencil3d_step_planes(self.q.handle, self.params, None if start else prev, cur, nxt, self.own[0],
                                 self.own[1], self.halo, start=start)
