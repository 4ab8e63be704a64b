"""Host-side logic of the cost model (no GPU): the held-out split, the regret
bookkeeping, the energy labels and the synthetic corpus shapes."""
import math

import numpy as np

from paper_2505_06022_gb300 import costmodel, inputs


def test_split_shapes_is_a_seeded_partition():
    for n in (1, 5, 220, 600):
        train, test = costmodel.split_shapes(n)
        assert len(np.intersect1d(train, test)) == 0
        assert np.array_equal(np.sort(np.concatenate([train, test])), np.arange(n))
        assert test.size == max(1, int(round(0.2 * n)))
        t2, s2 = costmodel.split_shapes(n)
        assert np.array_equal(train, t2) and np.array_equal(test, s2)
    assert not np.array_equal(costmodel.split_shapes(600, seed=1)[1], costmodel.split_shapes(600, seed=2)[1])


def _corpus():
    # shape 0: stencil with times 2, 1, 4 ms; shape 1: SAXPY with times 3, 6 ms; shape 2: stencil 5, 5
    shape = np.array([0, 0, 0, 1, 1, 2, 2])
    t = np.array([2.0, 1.0, 4.0, 3.0, 6.0, 5.0, 5.0])
    shapes = [{"kind": 1, "dtype": "f32", "radius": 1}, {"kind": 0, "dtype": "f32"},
              {"kind": 1, "dtype": "bf16", "radius": 2}]
    return shapes, {"shape": shape, "logt": np.log(t)}


def test_regret_of_the_best_and_the_worst_pick():
    shapes, corpus = _corpus()
    best = costmodel.regret(shapes, corpus, lambda sid, rows: int(np.argmin(corpus["logt"][rows])))
    assert best["mean"] == 0.0 and best["max"] == 0.0 and best["shapes"] == 3
    worst = costmodel.regret(shapes, corpus, lambda sid, rows: int(np.argmax(corpus["logt"][rows])))
    # shape 0: 4/1 - 1 = 3; shape 1: 6/3 - 1 = 1; shape 2: 0
    assert math.isclose(worst["mean"], 4.0 / 3.0) and math.isclose(worst["max"], 3.0)
    assert math.isclose(worst["mean_stencil"], 1.5) and math.isclose(worst["mean_saxpy"], 1.0)
    first = costmodel.regret(shapes, corpus, lambda sid, rows: 0)  # shape 0: 2/1 - 1 = 1
    assert math.isclose(first["mean"], (1.0 + 0.0 + 0.0) / 3.0)


def test_energy_labels_are_group_power_times_time():
    shapes, corpus = _corpus()
    power = {(1, "f32", 1): 500.0, (0, "f32", 0): 300.0, (1, "bf16", 2): 400.0}
    loge = costmodel.energy_labels(shapes, corpus, power)
    t_s = np.exp(corpus["logt"]) * 1e-3
    want = np.log(np.array([500.0, 500.0, 500.0, 300.0, 300.0, 400.0, 400.0]) * t_s)
    assert np.allclose(loge, want, rtol=0, atol=1e-12)


def test_corpus_shapes_ranges_and_determinism():
    shapes = inputs.cost_corpus_shapes(n_stencil=300, n_saxpy=40)
    assert shapes == inputs.cost_corpus_shapes(n_stencil=300, n_saxpy=40)
    sten = [s for s in shapes if s["kind"] == 1]
    sax = [s for s in shapes if s["kind"] == 0]
    assert len(sten) == 300 and len(sax) == 40
    assert all(512 <= s["ny"] <= 16384 and 512 <= s["nx"] <= 16384 for s in sten)
    assert {s["radius"] for s in sten} == {1, 2, 3, 4} and {s["dtype"] for s in sten} == {"f32", "bf16"}
    assert all((1 << 16) <= s["n"] <= (1 << 28) for s in sax)
    # log-uniform sides: about half of them below the geometric mean of the range
    below = sum(s["ny"] < math.sqrt(512 * 16384) for s in sten)
    assert 0.35 * 300 < below < 0.65 * 300


def test_power_model_recovers_a_known_power_law_and_beats_the_group_label():
    """Synthetic metered candidates whose power is the group's times exp(0.3 - 0.1 log2 points):
    the fitted model (features from the library's host-side feature code) predicts held-out
    candidates far better than the group label, and orders their energies correctly."""
    z = inputs.splitmix64(3, 4 * 60)
    rows = []
    for i in range(60):
        dt = ("f32", "bf16")[int(z[4 * i] % 2)]
        r = 1 + int(z[4 * i + 1] % 4)
        side = (2048, 4096, 8192)[int(z[4 * i + 2] % 3)]
        v = 1 + int(z[4 * i + 3] % 12)
        k = (1, 4)[int((z[4 * i + 3] >> 32) % 2)]
        ms = 1e-3 * side * side / 6e8 * (1.0 + 0.05 * (v % 3))
        label = 1000.0 * ms * 1e-3
        meas = label * math.exp(0.3 - 0.1 * math.log2(side * side))
        rows.append({"dtype": dt, "radius": r, "side": side, "variant": v, "chunks": k, "ms": ms,
                     "j_measured": meas, "j_label": label})
    fit = costmodel.fit_power_model({"candidates": rows, "group_power_w": {}}, ridge=1e-6)
    assert fit["loo_abs_log_error"]["max"] < 0.02
    assert fit["group_label_abs_log_error"]["median"] > 1.0
    o = fit["energy_order_loo"]
    assert o["pairs"] > 0 and o["agree"] == o["pairs"]
