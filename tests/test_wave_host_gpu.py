"""sy_wave_run_host: a whole simulation from host memory, the runtime moving the
data (paper §2 Listing 1 and §3: accessors name the data, the runtime makes it
present on the device).

Bar: the host result is bit-identical to sy_wave_run on device buffers and to
the oracle's precision mirror; consecutive calls (which overlap their copies
with each other's simulations) each give their own input's result; feeding a
result straight back in as the next input is safe; bad arguments launch
nothing."""
import numpy as np
import pytest

import oracle
import paper_2505_06022_gb300 as sy
from paper_2505_06022_gb300 import inputs

from gpu_helpers import bits, torch_cuda

pytestmark = pytest.mark.gpu

DT = {"f32": oracle.F32, "bf16": oracle.BF16, "f16": oracle.F16}


@pytest.fixture(scope="module")
def q():
    torch_cuda()
    with sy.Queue(0) as queue:
        yield queue.handle


def field(ny, nx, dtype, seed):
    a = inputs.gaussian_pulse(ny, nx, max(2.0, min(ny, nx) / 6.0)) + 0.05 * inputs.random_field(seed, ny, nx)
    return inputs.to_storage(a, dtype)


def as_torch_host(a, pinned):
    torch = torch_cuda()
    t = torch.from_numpy(a.view(np.int16) if a.dtype == np.uint16 else a).clone()
    return t.pin_memory() if pinned else t


@pytest.mark.parametrize("dtype,r,variant", [("f32", 1, 0), ("bf16", 2, 0), ("f16", 4, 0), ("f32", 3, 0),
                                             ("bf16", 3, 15)])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_run_equals_device_run_and_mirror(q, dtype, r, pinned, variant):
    torch = torch_cuda()
    ny, nx, steps = 77, 304, 9
    u0 = field(ny, nx, dtype, seed=r)
    chunks = sy.sy_split_rows(ny, 3)
    p = sy.stencil_params(ny, nx, r, 0.25, dtype, variant=variant)
    h_in = as_torch_host(u0, pinned)
    h_out, h_prev = torch.empty_like(h_in), torch.empty_like(h_in)
    if pinned:
        h_out, h_prev = h_out.pin_memory(), h_prev.pin_memory()
    sy.sy_wave_run_host(q, p, h_in, h_out, steps, chunks, r, host_prev_out=h_prev)
    sy.sy_queue_sync(q)
    # the same run on device buffers
    d0 = h_in.cuda()
    ua, ub = torch.empty_like(d0), torch.empty_like(d0)
    pv, cv, _ = sy.sy_wave_run(q, p, d0, ua, ub, steps, chunks, r)
    torch.cuda.synchronize()
    byptr = {d0.data_ptr(): d0, ua.data_ptr(): ua, ub.data_ptr(): ub}
    assert torch.equal(h_out, byptr[cv].cpu()) and torch.equal(h_prev, byptr[pv].cpu())
    op, oc = oracle.wave_run_mirror(DT[dtype], u0, steps, r, 0.25)
    st = oc.dtype
    assert np.array_equal(bits(h_out.numpy().view(st)), bits(oc))
    assert np.array_equal(bits(h_prev.numpy().view(st)), bits(op))


def test_consecutive_calls_each_give_their_own_result(q):
    """Four calls in a row (rotating work sets, copies overlapping the neighbouring
    simulations), a padded pitch, numpy host arrays, one sync at the end."""
    torch_cuda()
    ny, nx, pitch, steps, r = 64, 250, 264, 6, 1
    p = sy.stencil_params(ny, nx, r, 0.25, "f32", pitch=pitch)
    chunks = sy.sy_split_rows(ny, 4)
    ins, outs = [], []
    for k in range(4):
        u = np.zeros((ny, pitch), np.float32)
        u[:, :nx] = field(ny, nx, "f32", seed=10 + k)
        ins.append(u)
        outs.append(np.full((ny, pitch), np.nan, np.float32))
    for k in range(4):
        sy.sy_wave_run_host(q, p, ins[k], outs[k], steps, chunks, r)
    sy.sy_queue_sync(q)
    for k in range(4):
        _, want = oracle.wave_run_mirror(oracle.F32, np.ascontiguousarray(ins[k][:, :nx]), steps, r, 0.25)
        assert np.array_equal(bits(np.ascontiguousarray(outs[k][:, :nx])), bits(want)), k


def test_result_fed_back_in_is_read_after_it_is_written(q):
    """host_u0 = host_out, three calls in a row: each restarts (zero velocity) from the
    previous result, which must be complete before it is copied in."""
    torch_cuda()
    ny, nx, steps, r = 40, 512, 5, 2
    p = sy.stencil_params(ny, nx, r, 0.25, "bf16")
    chunks = sy.sy_split_rows(ny, 2)
    u = field(ny, nx, "bf16", seed=4)
    buf = as_torch_host(u, pinned=True)
    for _ in range(3):
        sy.sy_wave_run_host(q, p, buf, buf, steps, chunks, r)
    sy.sy_queue_sync(q)
    want = u
    for _ in range(3):
        _, want = oracle.wave_run_mirror(oracle.BF16, want, steps, r, 0.25)
    assert np.array_equal(buf.numpy().view(np.uint16), want)


def test_host_run_rejects_bad_arguments(q):
    torch_cuda()
    ny, nx = 16, 64
    p = sy.stencil_params(ny, nx, 1, 0.25, "f32")
    u = np.zeros((ny, nx), np.float32)
    out = np.zeros((ny, nx), np.float32)
    chunks = sy.sy_split_rows(ny, 2)
    cases = [
        (lambda: sy.sy_wave_run_host(q, p, None, out, 3, chunks, 1), "SY_ERR_NULL_POINTER"),
        (lambda: sy.sy_wave_run_host(q, p, u, None, 3, chunks, 1), "SY_ERR_NULL_POINTER"),
        (lambda: sy.sy_wave_run_host(q, p, u, out, 3, chunks, 1, host_prev_out=out), "SY_ERR_ALIAS"),
        (lambda: sy.sy_wave_run_host(q, p, u, out, -1, chunks, 1), "SY_ERR_INVALID_ARGUMENT"),
        (lambda: sy.sy_wave_run_host(q, p, u, out, 3, [(0, 5), (6, 16)], 1), "SY_ERR_BAD_CHUNKS"),
        (lambda: sy.sy_wave_run_host(q, p, u, out, 3, chunks, 0), "SY_ERR_HALO_TOO_SMALL"),
    ]
    for call, name in cases:
        with pytest.raises(sy.SyError) as e:
            call()
        assert e.value.name == name
    with pytest.raises(ValueError):
        sy.sy_wave_run_host(q, p, u[:, ::2], out, 3, chunks, 1)


def test_host_run_zero_steps_growing_grids_and_events(q):
    """steps = 0 returns u^0 and u^-1 (the Taylor start); a larger grid after a smaller one
    reallocates the work sets (waiting for the calls still using them); per-chunk events of a
    host run time every chunk launch."""
    torch_cuda()
    results = []
    for (ny, nx), steps in (((20, 64), 0), ((90, 520), 4), ((30, 128), 3)):
        u = field(ny, nx, "f32", seed=ny)
        out, prv = np.zeros_like(u), np.zeros_like(u)
        p = sy.stencil_params(ny, nx, 1, 0.25, "f32")
        chunks = sy.sy_split_rows(ny, 3)
        ev = sy.sy_wave_run_host(q, p, u, out, steps, chunks, 1, host_prev_out=prv, want_events=True)
        results.append((u, out, prv, steps, ev))
    sy.sy_queue_sync(q)
    for u, out, prv, steps, ev in results:
        if steps == 0:
            assert np.array_equal(bits(out), bits(u))
            want_prev = oracle.wave_start_mirror(oracle.F32, u, 1, 0.25)
        else:
            want_prev, want = oracle.wave_run_mirror(oracle.F32, u, steps, 1, 0.25)
            assert np.array_equal(bits(out), bits(want))
        assert np.array_equal(bits(prv), bits(want_prev))
        assert len(ev) == (steps + 1) * 3
    # the last call's events are still valid: every chunk launch timed
    ms = sy.sy_events_elapsed(q, results[-1][4])
    assert all(m > 0 for m in ms)


def test_results_fed_back_two_and_three_calls_later(q):
    """Interleaved chains: every call's input is the output of the call two back (chains
    A and B alternate) or three back (chains A, B, C rotate), so the input copy must wait
    for a copy-out of a call that used another work set."""
    torch_cuda()
    ny, nx, steps, r = 48, 256, 4, 1
    p = sy.stencil_params(ny, nx, r, 0.25, "f32")
    chunks = sy.sy_split_rows(ny, 2)
    for n_chains in (2, 3):
        starts = [field(ny, nx, "f32", seed=20 + c) for c in range(n_chains)]
        bufs = [as_torch_host(u, pinned=True) for u in starts]
        rounds = 4
        for _ in range(rounds):
            for c in range(n_chains):
                sy.sy_wave_run_host(q, p, bufs[c], bufs[c], steps, chunks, r)
        sy.sy_queue_sync(q)
        for c in range(n_chains):
            want = starts[c]
            for _ in range(rounds):
                _, want = oracle.wave_run_mirror(oracle.F32, want, steps, r, 0.25)
            assert np.array_equal(bits(bufs[c].numpy()), bits(want)), (n_chains, c)
