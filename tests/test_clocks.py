"""Energy targets by frequency scaling (paper §4, MIN_EDP), on the CPU.

The choice of an operating point is checked against brute force.  Clock control
runs against a fake NVML (tests/fake_nvml.c, loaded through SY_NVML_LIB), never
a real device: each scenario runs in a fresh process (the library loads NVML once
per process) and checks what the fake saw -- which clocks were locked, in which
order, and that the lock is always released."""
import json
import os
import random
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, ROOT)

import paper_2505_06022_gb300 as sy  # noqa: E402

TARGETS = {sy.SY_TARGET_MIN_TIME: lambda t, j: t, sy.SY_TARGET_MIN_ENERGY: lambda t, j: j,
           sy.SY_TARGET_MIN_EDP: lambda t, j: j * t, sy.SY_TARGET_MIN_ED2P: lambda t, j: j * t * t}


def brute_choice(target, points):
    f = TARGETS[target]
    best = 0
    for i, (mhz, t, j) in enumerate(points):
        ob, oi = f(points[best][1], points[best][2]), f(t, j)
        if oi < ob or (oi == ob and mhz > points[best][0]):
            best = i
    return best


@pytest.mark.parametrize("seed", range(20))
def test_choose_matches_brute_force(seed):
    rng = random.Random(seed)
    n = rng.randint(1, 12)
    pts = [(rng.choice([990, 1200, 1410, 1755, 2070]), rng.uniform(1e-4, 1.0), rng.choice([0.0, rng.uniform(0, 50)]))
           for _ in range(n)]
    if seed % 4 == 0 and n > 1:  # exact ties in every objective: the higher clock wins
        pts[-1] = (pts[0][0] + 15, pts[0][1], pts[0][2])
    for target in TARGETS:
        assert sy.sy_clock_choose(target, pts) == brute_choice(target, pts)


def test_choose_edp_interior_minimum():
    # t = 1 + 2070/f (memory part fixed, SM part scales), P = 100 + 300 (f/2070)^3: the EDP minimum
    # lies strictly inside the clock range, the time minimum at the top and the energy minimum below it.
    clocks = [2070 - 105 * k for k in range(11)]
    pts = [(f, 1 + 2070 / f, (100 + 300 * (f / 2070) ** 3) * (1 + 2070 / f)) for f in clocks]
    assert clocks[sy.sy_clock_choose(sy.SY_TARGET_MIN_TIME, pts)] == 2070
    edp = clocks[sy.sy_clock_choose(sy.SY_TARGET_MIN_EDP, pts)]
    en = clocks[sy.sy_clock_choose(sy.SY_TARGET_MIN_ENERGY, pts)]
    assert 1020 < edp < 2070 and en <= edp


@pytest.mark.parametrize("pts,target", [([], 2), ([(2070, 0.0, 1.0)], 2), ([(2070, 1.0, -1.0)], 2),
                                        ([(2070, float("nan"), 1.0)], 2), ([(2070, 1.0, float("inf"))], 2),
                                        ([(2070, 1.0, 1.0)], 4), ([(2070, 1.0, 1.0)], -1)])
def test_choose_rejects(pts, target):
    with pytest.raises(sy.SyError) as e:
        sy.sy_clock_choose(target, pts)
    assert e.value.name == "SY_ERR_INVALID_ARGUMENT"


# ---- clock control against the fake NVML, one process per scenario -----------------

@pytest.fixture(scope="module")
def fake_lib(tmp_path_factory):
    out = tmp_path_factory.mktemp("nvml") / "libfake_nvml.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", os.path.join(HERE, "fake_nvml.c"), "-o", str(out)],
                   check=True, capture_output=True)
    return str(out)


def run_scenario(name, fake, control):
    env = dict(os.environ)
    env.pop("SY_FAULT", None)
    env["SY_NVML_LIB"] = fake
    env.pop("SY_CLOCK_CONTROL", None)
    if control:
        env["SY_CLOCK_CONTROL"] = "1"
    r = subprocess.run([sys.executable, os.path.abspath(__file__), name], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    return json.loads(r.stdout.strip().splitlines()[-1])


def _fake():
    import ctypes as C

    F = C.CDLL(os.environ["SY_NVML_LIB"])
    F.fake_nvml_log.restype = C.c_char_p
    return F


def _raises(name, fn, *args):
    try:
        fn(*args)
    except sy.SyError as e:
        return e.name == name
    return False


def scenario_gate_off():
    F = _fake()
    ok = [_raises("SY_ERR_UNSUPPORTED", sy.sy_clock_lock, 0, 1755),
          _raises("SY_ERR_UNSUPPORTED", sy.sy_clock_unlock, 0),
          _raises("SY_ERR_UNSUPPORTED", sy.sy_clock_sweep, 0, [2070, 1755], lambda f: (1.0, 1.0))]
    mem, clocks = sy.sy_clock_supported(0)  # reading needs no permission
    return {"ok": all(ok), "log": F.fake_nvml_log().decode(), "mem": mem, "clocks": clocks}


def scenario_read_only():
    mem, clocks = sy.sy_clock_supported(0)
    cur = sy.sy_clock_current(0)
    bad = _raises("SY_ERR_NVML", sy.sy_clock_supported, 7)
    F = _fake()
    F.fake_nvml_set_mem_clock(405)  # an idle memory clock NVML does not list: the highest listed one is used
    mem_idle, clocks_idle = sy.sy_clock_supported(0)
    return {"mem": mem, "clocks": clocks, "cur": list(cur), "bad_index": bad, "mem_idle": mem_idle,
            "clocks_idle": clocks_idle, "log": F.fake_nvml_log().decode()}


def scenario_lock_unlock():
    import ctypes as C

    F = _fake()
    sy.sy_clock_lock(1, 1755)
    lo, hi = C.c_uint(), C.c_uint()
    F.fake_nvml_locked(1, C.byref(lo), C.byref(hi))
    cur = sy.sy_clock_current(1)
    sy.sy_clock_unlock(1)
    F.fake_nvml_locked(1, C.byref(lo), C.byref(hi))
    after = (lo.value, hi.value)
    unsupported = _raises("SY_ERR_INVALID_ARGUMENT", sy.sy_clock_lock, 1, 1000)
    F.fake_nvml_fail(b"nvmlDeviceSetGpuLockedClocks", 4)  # no permission
    refused = _raises("SY_ERR_NVML", sy.sy_clock_lock, 1, 2070)
    return {"cur": list(cur), "after": list(after), "unsupported": unsupported, "refused": refused,
            "log": F.fake_nvml_log().decode()}


def _model(f):
    t = 1 + 2070 / f
    return t, (100 + 300 * (f / 2070) ** 3) * t


def scenario_sweep():
    F = _fake()
    res = {}
    _, clocks = sy.sy_clock_supported(0)
    for target in TARGETS:
        F.fake_nvml_clear()
        seen = []

        def measure(mhz):
            seen.append((mhz, sy.sy_clock_current(0)[0]))  # the clock is locked while measuring
            return _model(mhz)

        best, pts = sy.sy_clock_sweep(0, clocks, measure, target)
        res[str(target)] = {"best": best, "pts": pts, "seen": seen, "log": F.fake_nvml_log().decode()}
    return {"clocks": clocks, "res": res}


def scenario_sweep_failures():
    F = _fake()
    out = {}
    calls = []

    def measure(mhz):
        calls.append(mhz)
        if len(calls) == 3:
            raise RuntimeError("measurement failed")
        return _model(mhz)

    out["measure_fails"] = _raises("SY_ERR_INVALID_ARGUMENT", sy.sy_clock_sweep, 0, [2070, 1860, 1650, 1440],
                                   measure)
    out["log_measure"] = F.fake_nvml_log().decode()
    F.fake_nvml_clear()
    out["bad_candidate"] = _raises("SY_ERR_INVALID_ARGUMENT", sy.sy_clock_sweep, 0, [2070, 1000], _model)
    out["log_bad"] = F.fake_nvml_log().decode()
    F.fake_nvml_clear()
    F.fake_nvml_fail(b"nvmlDeviceSetGpuLockedClocks", 4)
    out["lock_refused"] = _raises("SY_ERR_NVML", sy.sy_clock_sweep, 0, [2070, 1860], _model)
    out["log_refused"] = F.fake_nvml_log().decode()
    F.fake_nvml_fail(b"", 0)
    F.fake_nvml_clear()
    F.fake_nvml_fail(b"nvmlDeviceResetGpuLockedClocks", 4)
    out["unlock_refused"] = _raises("SY_ERR_NVML", sy.sy_clock_sweep, 0, [2070], _model)
    return out


def scenario_missing():
    return {"read": _raises("SY_ERR_NVML_UNAVAILABLE", sy.sy_clock_supported, 0),
            "lock": _raises("SY_ERR_NVML_UNAVAILABLE", sy.sy_clock_lock, 0, 2070)}


FAKE_CLOCKS = [2070, 1965, 1860, 1755, 1650, 1545, 1440, 1335, 1230, 1125, 1020]


def test_gate_off_refuses_before_any_nvml_call(fake_lib):
    r = run_scenario("gate_off", fake_lib, control=False)
    assert r["ok"] and r["log"] == ""
    assert r["mem"] == 3996 and r["clocks"] == FAKE_CLOCKS


def test_read_only_queries(fake_lib):
    r = run_scenario("read_only", fake_lib, control=False)
    assert r["mem"] == 3996 and r["clocks"] == FAKE_CLOCKS and r["cur"] == [2070, 2070]
    assert r["bad_index"]
    assert r["mem_idle"] == 3996 and r["clocks_idle"] == FAKE_CLOCKS
    assert r["log"] == ""


def test_lock_and_unlock(fake_lib):
    r = run_scenario("lock_unlock", fake_lib, control=True)
    assert r["cur"] == [1755, 2070] and r["after"] == [0, 0]
    assert r["unsupported"] and r["refused"]
    assert r["log"] == "lock:1:1755:1755;reset:1;lock:1:2070:2070;"


def test_sweep_locks_each_candidate_then_releases_and_chooses(fake_lib):
    r = run_scenario("sweep", fake_lib, control=True)
    clocks = r["clocks"]
    want_log = "".join(f"lock:0:{f}:{f};" for f in clocks) + "reset:0;"
    for target, got in r["res"].items():
        assert got["log"] == want_log
        assert got["seen"] == [[f, f] for f in clocks]
        pts = [tuple(p) for p in got["pts"]]
        assert [p[0] for p in pts] == clocks
        assert got["best"] == brute_choice(int(target), pts)
    assert clocks[r["res"][str(sy.SY_TARGET_MIN_TIME)]["best"]] == 2070
    assert 1020 < clocks[r["res"][str(sy.SY_TARGET_MIN_EDP)]["best"]] < 2070


def test_sweep_failures_always_release(fake_lib):
    r = run_scenario("sweep_failures", fake_lib, control=True)
    assert r["measure_fails"] and r["log_measure"] == "lock:0:2070:2070;lock:0:1860:1860;lock:0:1650:1650;reset:0;"
    assert r["bad_candidate"] and r["log_bad"] == ""  # validated before the first lock
    assert r["lock_refused"] and r["log_refused"] == "lock:0:2070:2070;reset:0;"
    assert r["unlock_refused"]


def test_missing_nvml(tmp_path):
    r = run_scenario("missing", str(tmp_path / "no_such_nvml.so"), control=True)
    assert r["read"] and r["lock"]


if __name__ == "__main__":
    print(json.dumps(globals()["scenario_" + sys.argv[1]]()))
