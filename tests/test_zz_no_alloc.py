"""The allocation-free energy entry point (sy_wave_energy_static) against the
allocating one (sy_wave_energy).

Some callers cannot allocate device memory where they need the energy (work
issued during graph capture, applications whose allocator owns all device
memory, loops that must not synchronise the device); the static entry point
serves them from a fixed module-scope array.  This file is collected last so
that a run stopping at the first failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest

import oracle
import paper_2505_06022_gb300 as sy
from paper_2505_06022_gb300 import inputs

pytestmark = pytest.mark.gpu


def _field(ny, nx, dtype, seed):
    return inputs.to_storage(inputs.random_field(seed, ny, nx).astype(np.float64), dtype)


def test_static_energy_matches_allocating_entry_point_on_two_calls():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available(), "a test marked gpu ran without a CUDA device"
    L = sy.lib()
    out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream  # 0 = legacy default stream
    with sy.Queue(0) as q:
        # Two calls in a row: first a grid on which every one of the reduction's 1024 x 256
        # threads has points, then one of 100k points, on which about 600 blocks have none.
        # Those blocks must still overwrite their partial sums, or the second call would add
        # the first call's leftovers.
        for dtype, r, (ny, nx), seed in [("f32", 1, (700, 1030), 3), ("bf16", 4, (100, 1000), 8)]:
            code = oracle.DTYPES[dtype]
            un, uo = _field(ny, nx, dtype, seed), _field(ny, nx, dtype, seed + 1)
            to_dev = (lambda a: torch.from_numpy(a.view(np.int16) if a.dtype == np.uint16 else a).cuda())
            dn, do = to_dev(un), to_dev(uo)
            p = sy.stencil_params(ny, nx, r, 0.25, dtype)
            want = sy.sy_wave_energy(q.handle, p, dn, do)
            torch.cuda.synchronize()
            free_before = torch.cuda.mem_get_info()[0]
            rc = L.sy_wave_energy_static(C.c_void_p(stream or None), C.byref(p), C.c_void_p(dn.data_ptr()),
                                         C.c_void_p(do.data_ptr()), C.c_void_p(out.data_ptr()))
            assert rc == 0, L.sy_last_error().decode()
            torch.cuda.synchronize()
            assert torch.cuda.mem_get_info()[0] == free_before, "the allocation-free entry point allocated"
            got = out.cpu().tolist()
            # same kernels, same fixed reduction shape and order as the allocating entry point
            assert got == list(want), (dtype, got, want)
            # and the FP64 oracle, within two summation orders of N terms: <= 2 N eps sum|terms|
            ref = oracle.wave_energy_f64(oracle.storage_to_f64(un, code), oracle.storage_to_f64(uo, code), r, 0.25)
            tol = 2 * ny * nx * 2.0 ** -53 * ref["abs_sum"]
            assert abs(got[0] - ref["E"]) <= tol, (dtype, got[0], ref["E"])


def test_static_energy_rejects_bad_arguments():
    torch = pytest.importorskip("torch")
    L = sy.lib()
    a = torch.zeros(8, 64, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    bad = sy.stencil_params(8, 64, 5, 0.25, "f32")
    assert L.sy_wave_energy_static(None, C.byref(bad), a.data_ptr(), a.data_ptr(), out.data_ptr()) == 1
    ok = sy.stencil_params(8, 64, 1, 0.25, "f32")
    assert L.sy_wave_energy_static(None, C.byref(ok), a.data_ptr(), a.data_ptr(), None) == 2
    empty = sy.stencil_params(0, 0, 1, 0.25, "f32")
    out.fill_(7.0)
    assert L.sy_wave_energy_static(None, C.byref(empty), None, None, out.data_ptr()) == 0
    torch.cuda.synchronize()
    assert out.cpu().tolist() == [0.0, 0.0, 0.0]
