"""The stated accuracy of each storage type (paper_2505_06022_gb300.accuracy) against
what the oracle measures on the 8192^2 / 200-step wave workload.

The fixture tests/golden/precision_error_8192.txt is written by the oracle alone
(tests/golden/make_precision_error.py); here it is recomputed, and every stated
bound must hold the measured error with a margin of at most 2x (a looser bound would
state nothing).  The GPU side of the same bounds is tests/test_precision_gpu.py."""
import importlib.util
import os

import pytest

from paper_2505_06022_gb300 import accuracy

HERE = os.path.dirname(os.path.abspath(__file__))


def _maker():
    spec = importlib.util.spec_from_file_location("make_precision_error",
                                                  os.path.join(HERE, "golden", "make_precision_error.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_bounds_hold_the_measured_error_with_a_stated_margin():
    fixture = _maker().read()
    for dtype, bounds in accuracy.TOLERANCE.items():
        for k, bound in bounds.items():
            v = abs(fixture[dtype][k])
            assert v <= bound <= 2.0 * v, (dtype, k, v, bound)
    assert accuracy.TOLERANCE["f32"]["max_rel"] == 1e-5  # the workload's own bar


def test_usable_storage_types_conserve_energy_within_a_quarter():
    fixture = _maker().read()
    for dtype, ok in accuracy.USABLE.items():
        assert ok == (abs(fixture[dtype]["energy_drift"]) < 0.25), dtype


def test_fixture_is_what_the_oracle_computes():
    mk = _maker()
    stored, fresh = mk.read(), mk.measure()
    for dtype in ("f32", "bf16", "f16"):
        for k, v in stored[dtype].items():
            # rel 1e-6: the Gaussian's FP64 exp may differ in the last bit between numpy builds
            assert fresh[dtype][k] == pytest.approx(v, rel=1e-6, abs=0.0), (dtype, k)


def test_check_reports_each_bound():
    res = accuracy.check("f16", {"max_abs": 0.01, "max_rel": 0.5, "energy_drift": -0.1})
    assert res["max_abs"][2] and not res["max_rel"][2] and res["energy_drift"][2]
    assert "l2_rel" not in res
