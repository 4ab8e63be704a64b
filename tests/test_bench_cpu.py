"""bench.py's reference arm (the CPU oracle timed on the host cores) prints one
well-formed JSON line; runs without a GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "updates/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["higher_is_better"] is True


def _bench():
    sys.path.insert(0, ROOT)
    import bench

    return bench


def test_clock_record_from_nvidia_smi_lines():
    import threading

    bench = _bench()

    class Proc:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    s = bench.ClockSampler(0)
    s.proc, s._t = Proc(), threading.Thread(target=lambda: None)
    s._t.start()
    t = "2026/01/02 03:04:05.100"
    s.lines = [f"{t}, 0, 2070, 2070, 650.1, 0x0, Not Active, Not Active, Not Active, Not Active",
               f"{t}, 0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
               f"{t}, 0, 2070, 2070, 700.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbage line", f"{t}, 0, [N/A], 2070, 1.0, 0x0, a, b, c, d"]
    rec = s.stop()
    assert rec["sm_mhz"] == 2070.0 and rec["sm_max_mhz"] == 2070.0 and rec["samples"] == 3
    assert rec["reasons"] == ["sw_power_cap"] and rec["power_w_median"] == 700.0
    s2 = bench.ClockSampler(0)
    s2.proc, s2._t = Proc(), threading.Thread(target=lambda: None)
    s2._t.start()
    s2.lines = [f"{t}, 0, 900, 2070, 300, 0x8, Not Active, Active, Not Active, Not Active"]
    assert s2.stop()["reasons"] == ["hw_thermal_slowdown"]


def test_clock_record_keeps_the_timed_region():
    """Samples stamped inside the timed region's wall-clock window are the record; idle
    samples before and after it are dropped (all samples count only when none is inside)."""
    import datetime

    bench = _bench()
    t0 = datetime.datetime(2026, 1, 2, 3, 4, 5).timestamp()

    def line(dt, mhz, watts, cap):
        ts = datetime.datetime.fromtimestamp(t0 + dt).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        return f"{ts}, 0, {mhz}, 2070, {watts}, 0x0, Not Active, Not Active, Not Active, {cap}"

    lines = [line(-0.5, 2070, 150.0, "Not Active"), line(0.1, 1995, 1100.0, "Active"),
             line(0.3, 2010, 1150.0, "Active"), line(0.5, 2000, 1120.0, "Active"),
             line(2.0, 2070, 160.0, "Not Active")]
    rec = bench.ClockSampler.parse(lines, (t0, t0 + 1.0))
    assert rec["samples"] == 3 and rec["samples_in_timed_region"] == 3
    assert rec["sm_mhz"] == 2000.0 and rec["power_w_median"] == 1120.0 and rec["reasons"] == ["sw_power_cap"]
    everything = bench.ClockSampler.parse(lines, (t0 + 5.0, t0 + 6.0))
    assert everything["samples"] == 5 and everything["samples_in_timed_region"] == 0


def test_clock_record_without_nvidia_smi():
    bench = _bench()
    s = bench.ClockSampler(0)
    s.proc = None
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_measured_peak_and_kernel_hash():
    bench = _bench()
    peaks = bench.measured_peaks()
    assert peaks["hbm_gbs"] > 0 and peaks["source"] in ("measured", "fallback")
    sha = bench.kernel_source_sha()
    assert len(sha) == 16 and sha == bench.kernel_source_sha()
    assert bench.ncu_traffic() in (None, float(json.load(open(os.path.join(ROOT, "profiles",
                                                                            "wave_f32_8192_traffic.json")))
                                                 ["dram_bytes_per_launch"]))
