"""Data transfers inferred from the neighbourhood range mapper (paper §3), and the
rank-per-chunk halo exchange run as gloo processes on the CPU.

The exchange test holds each rank's chunk in the split-buffer layout and steps it
with the oracle (a CPU stand-in for the GPU kernel, injected by the test); after
the steps the ranks' own rows must equal the oracle run on the whole grid bit for
bit -- which holds only if every halo row arrived from the right owner."""
import os
import socket

import numpy as np
import pytest

import oracle
import paper_2505_06022_gb300 as sy
from paper_2505_06022_gb300 import inputs


def brute_transfers(ny, chunks, h):
    """{(dst, global row) -> src}: every row a chunk reads (oracle range mapper) but does not own."""
    want = {}
    for c, (a, b) in enumerate(chunks):
        lo, hi = oracle.rm_neighbourhood(a, b, h, ny)
        for row in range(lo, hi):
            if not (a <= row < b):
                want[(c, row)] = next(s for s, (x, y) in enumerate(chunks) if x <= row < y)
    return want


@pytest.mark.parametrize("ny,chunks,h", [
    (20, [(0, 5), (5, 12), (12, 20)], 1),
    (20, [(0, 5), (5, 12), (12, 20)], 3),
    (7, [(0, 2), (2, 4), (4, 6), (6, 7)], 2),      # chunks shorter than the halo
    (9, [(0, 1), (1, 2), (2, 9)], 4),
    (10, [(0, 10)], 2),                            # one chunk: nothing to move
    (8192, sy.sy_split_rows(8192, 4), 1),
])
def test_transfers_match_brute_force(ny, chunks, h):
    got = sy.sy_rm_transfers(ny, chunks, h)
    cover = {}
    for src, dst, r0, r1 in got:
        assert r0 < r1 and chunks[src][0] <= r0 and r1 <= chunks[src][1]  # one owner per transfer
        for row in range(r0, r1):
            assert (dst, row) not in cover
            cover[(dst, row)] = src
    assert cover == brute_transfers(ny, chunks, h)
    for c in range(len(chunks)):
        lo, hi, rows = sy.sy_split_layout(ny, chunks, h, c)
        a, b = chunks[c]
        assert lo == min(h, a) and hi == min(h, ny - b) and rows == lo + (b - a) + hi


def test_transfers_errors():
    with pytest.raises(sy.SyError) as e:
        sy.sy_rm_transfers(10, [(0, 4), (5, 10)], 1)
    assert e.value.name == "SY_ERR_BAD_CHUNKS"


# ---- rank-per-chunk exchange over gloo --------------------------------------------

def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, ny, nx, r, h, steps, out_dir):
    import torch
    import torch.distributed as dist

    from paper_2505_06022_gb300.distributed import RankChunk

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    rc = RankChunk(ny=ny, nx=nx, radius=r, halo=h, rank=rank, world=world)
    u0 = inputs.to_storage(inputs.gaussian_pulse(ny, nx, 3.0) + 0.1 * inputs.random_field(7, ny, nx), "f32")
    a, b = rc.chunks[rank]
    cur = torch.zeros(rc.rows, nx, dtype=torch.float32)
    cur[rc.own[0]: rc.own[1]] = torch.from_numpy(u0[a:b])
    prev = torch.zeros_like(cur)

    def oracle_step(p_, c_, n_, r0, r1, start):
        # CPU stand-in for the GPU kernel: the oracle on the local buffer, own rows kept
        if start:
            full = oracle.wave_start_mirror(oracle.F32, c_.numpy().copy(), r, 0.25)
        else:
            full = oracle.wave_step_mirror(oracle.F32, p_.numpy().copy(), c_.numpy().copy(), r, 0.25)
        n_[r0:r1] = torch.from_numpy(full[r0:r1])

    rc.step(None, cur, prev, dist, oracle_step, start=True)
    for _ in range(steps):
        rc.step(prev, cur, prev, dist, oracle_step)
        prev, cur = cur, prev
    np.save(os.path.join(out_dir, f"rank{rank}.npy"), cur[rc.own[0]: rc.own[1]].numpy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,ny,nx,r,h,steps", [(2, 23, 17, 1, 1, 9), (3, 37, 29, 2, 3, 7), (4, 7, 11, 2, 2, 5)])
def test_gloo_rank_chunks_equal_whole_grid(tmp_path, world, ny, nx, r, h, steps):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    port = _free_port()
    mp.start_processes(_rank_main, args=(world, port, ny, nx, r, h, steps, str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    got = np.concatenate([np.load(tmp_path / f"rank{k}.npy") for k in range(world)])
    u0 = inputs.to_storage(inputs.gaussian_pulse(ny, nx, 3.0) + 0.1 * inputs.random_field(7, ny, nx), "f32")
    _, want = oracle.wave_run_mirror(oracle.F32, u0, steps, r, 0.25)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


# ---- the 3D grid split into chunks of planes ---------------------------------------

def _rank_main_3d(rank, world, port, nz, ny, nx, r, h, steps, out_dir):
    import torch
    import torch.distributed as dist

    from paper_2505_06022_gb300.distributed import GpuRankChunk3d

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    rc = GpuRankChunk3d(None, nz, ny, nx, r, h, rank, world, 0.125)  # no GPU: the oracle steps (below)
    u0 = inputs.to_storage(inputs.gaussian_pulse_3d(nz, ny, nx, 2.0) + 0.1 * inputs.random_field_3d(7, nz, ny, nx),
                           "f32")
    a, b = rc.chunks[rank]
    cur = torch.zeros(rc.rows, ny, nx, dtype=torch.float32)
    cur[rc.own[0]: rc.own[1]] = torch.from_numpy(u0[a:b])
    prev = torch.zeros_like(cur)

    def oracle_step(p_, c_, n_, z0, z1, start):
        # CPU stand-in for the 3D kernel on the local buffer, own planes kept
        if start:
            full = oracle.wave3d_start_mirror(oracle.F32, c_.numpy().copy(), r, 0.125)
        else:
            full = oracle.wave3d_step_mirror(oracle.F32, p_.numpy().copy(), c_.numpy().copy(), r, 0.125)
        n_[z0:z1] = torch.from_numpy(full[z0:z1])

    rc.step(None, cur, prev, dist, oracle_step, start=True)
    for _ in range(steps):
        rc.step(prev, cur, prev, dist, oracle_step)
        prev, cur = cur, prev
    np.save(os.path.join(out_dir, f"rank{rank}.npy"), cur[rc.own[0]: rc.own[1]].numpy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,nz,ny,nx,r,h,steps", [(2, 9, 7, 6, 1, 1, 6), (3, 11, 5, 9, 2, 3, 5),
                                                      (4, 6, 6, 5, 2, 2, 4)])
def test_gloo_plane_chunks_equal_whole_grid(tmp_path, world, nz, ny, nx, r, h, steps):
    pytest.importorskip("torch")
    import torch.multiprocessing as mp

    port = _free_port()
    mp.start_processes(_rank_main_3d, args=(world, port, nz, ny, nx, r, h, steps, str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    got = np.concatenate([np.load(tmp_path / f"rank{k}.npy") for k in range(world)])
    u0 = inputs.to_storage(inputs.gaussian_pulse_3d(nz, ny, nx, 2.0) + 0.1 * inputs.random_field_3d(7, nz, ny, nx),
                           "f32")
    _, want = oracle.wave3d_run_mirror(oracle.F32, u0, steps, r, 0.125)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
