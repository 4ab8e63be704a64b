"""Learned cost model: corpus, training and regret.

The library measures its own kernels (sy_tune_stencil / sy_tune_saxpy: every
candidate configuration, device timestamps), turns each candidate into features
(sy_cost_features), trains its own MLP on the GPU (sy_mlp_train: the library's
forward/backward/Adam kernels) to predict (log time, log energy), and is judged
by regret against the exhaustive tuner on held-out shapes:

    regret(shape) = t(candidate the model picks) / t(best measured candidate) - 1

Energy labels: NVML's energy counter ticks every ~100 ms, far coarser than one
kernel, so each group of kernels with the same kind, storage type and radius gets
its busy power P from a >= 1 s burst of a representative launch, and a
candidate's energy is P x its time (the same attribution sy_kernel_energy uses).

Run:  python -m paper_2505_06022_gb300.costmodel [--stencil N] [--saxpy N] [--out corpus.npz]
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import (DTYPE_CODES, Queue, SyError, inputs, stencil_params, sy_cost_features, sy_cost_model_predict,
               sy_meter_begin, sy_meter_end, sy_mlp_create, sy_mlp_destroy, sy_mlp_save, sy_mlp_train,
               sy_saxpy_variant_info, sy_stencil_step, sy_stencil_variant_info, sy_saxpy, sy_tune_saxpy,
               sy_tune_stencil)

CHUNK_COUNTS = (1, 2, 4, 8)
F = 13


def default_candidate(kind: int, dtype: str, radius: int = 1) -> tuple[int, int, int, int]:
    """(tile_rows, tile_cols, threads, chunks) the library uses without the model."""
    if kind == 1:
        rows, cols, thr = sy_stencil_variant_info(radius, DTYPE_CODES[dtype], 0)
        return rows, cols, thr, 1
    thr, waves = sy_saxpy_variant_info(0)
    return waves, 4, thr, 1


def _pitch(s: dict) -> int:
    """Row pitch padded to 16 bytes, as an application allocating for the vector kernel would."""
    v = 4 if s["dtype"] == "f32" else 8
    return (s["nx"] + v - 1) // v * v


def measure(q: Queue, shapes: list[dict], reps: int = 3, log=None) -> dict:
    """Tune every shape exhaustively; returns feature rows, log-time labels and ids."""
    import torch

    st_pts = max([s["ny"] * _pitch(s) for s in shapes if s["kind"] == 1] or [1])
    sx_n = max([s["n"] for s in shapes if s["kind"] == 0] or [1])
    bufs = [torch.zeros(max(st_pts, sx_n) + 64, dtype=torch.float32, device="cuda") for _ in range(3)]
    feats, logt, shape_id, meta = [], [], [], []
    t0 = time.time()
    for i, s in enumerate(shapes):
        if s["kind"] == 1:
            p = stencil_params(s["ny"], s["nx"], s["radius"], 0.25, s["dtype"], pitch=_pitch(s))
            recs = sy_tune_stencil(q.handle, p, bufs[0], bufs[1], bufs[2], CHUNK_COUNTS, reps)
            dt = DTYPE_CODES[s["dtype"]]
            for r in recs:
                feats.append(sy_cost_features(1, dt, s["radius"], s["ny"], s["nx"], r["tile_rows"], r["tile_cols"],
                                              r["threads"], r["chunks"]))
                logt.append(math.log(r["ms"]))
                shape_id.append(i)
                meta.append((r["tile_rows"], r["tile_cols"], r["threads"], r["chunks"]))
        else:
            recs = sy_tune_saxpy(q.handle, s["n"], bufs[0], bufs[1], bufs[2], CHUNK_COUNTS, reps)
            for r in recs:
                feats.append(sy_cost_features(0, 0, 0, 1, s["n"], r["tile_rows"], r["tile_cols"], r["threads"],
                                              r["chunks"]))
                logt.append(math.log(r["ms"]))
                shape_id.append(i)
                meta.append((r["tile_rows"], r["tile_cols"], r["threads"], r["chunks"]))
        if log and (i + 1) % 50 == 0:
            log(f"tuned {i + 1}/{len(shapes)} shapes, {len(logt)} rows, {time.time() - t0:.1f} s")
    del bufs
    return {"X": np.asarray(feats, np.float32), "logt": np.asarray(logt, np.float64),
            "shape": np.asarray(shape_id, np.int64), "cand": np.asarray(meta, np.int64)}


def _fields(dt: str, n: int, seed: int = 5) -> list:
    """Three n x n device fields of storage `dt` holding uniform values in [-1, 1) (switching
    power depends on the data: zeros would understate it)."""
    import torch

    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    tdt = torch.float32 if dt == "f32" else torch.bfloat16
    out = []
    for _ in range(3):
        t = torch.rand(n * n + 64, generator=g, device="cuda", dtype=torch.float32).mul_(2.0).sub_(1.0)
        out.append(t.to(tdt))
    return out


def group_power(q: Queue, seconds: float = 1.0) -> dict:
    """Busy device power (W) per (kind, dtype, radius) group from >= `seconds` bursts."""
    import torch

    out = {}
    n = 8192
    fields = {dt: _fields(dt, n) for dt in ("f32", "bf16")}
    for dt in ("f32", "bf16"):
        for r in (1, 2, 3, 4):
            p = stencil_params(n, n, r, 0.25, dt)
            a, b, c = fields[dt]
            out[(1, dt, r)] = _burst(q, lambda: sy_stencil_step(q.handle, p, a, b, c, [(0, n)], r), seconds)
    big = 1 << 27
    x, y, z = (torch.zeros(big, dtype=torch.float32, device="cuda") for _ in range(3))
    out[(0, "f32", 0)] = _burst(q, lambda: sy_saxpy(q.handle, big, 1.5, x, y, z), seconds)
    return out


def _burst(q: Queue, fn, seconds: float) -> float:
    import torch

    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    sy_meter_begin(q.handle)
    t0 = time.time()
    while time.time() - t0 < seconds:
        for _ in range(20):
            fn()
        torch.cuda.synchronize()
    joules, secs = sy_meter_end(q.handle)
    return joules / secs


def energy_labels(shapes, corpus, power: dict) -> np.ndarray:
    """log J per row = log(P_group * t)."""
    out = np.empty_like(corpus["logt"])
    for k, sid in enumerate(corpus["shape"]):
        s = shapes[sid]
        key = (s["kind"], s["dtype"], s.get("radius", 0))
        out[k] = math.log(power[key]) + corpus["logt"][k] - math.log(1e3)
    return out


def energy_check(q: Queue, n_cands: int = 96, seconds: float = 1.0, seed: int = 21) -> dict:
    """Meters a seeded subset of stencil candidates one by one, each repeated in its own
    >= `seconds` NVML window, and compares the measured joules per step with the label the
    corpus gives it (group busy power x its own time).  Candidates span both storage types,
    radius 1..4, every tile variant and chunk counts {1, 4}, on grids of 2048^2 to 8192^2.
    Returns per-candidate rows and summary statistics (correlation of log J, the spread of
    measured / label, and within each (storage, radius, grid) group whether the energy
    order of the candidates is their time order)."""
    import torch

    from . import sy_stencil_variant_count, sy_split_rows, DTYPE_CODES as CODES

    power = group_power(q, seconds)
    z = inputs.splitmix64(seed, 4 * n_cands)
    sides = (2048, 4096, 8192)
    fields = {dt: _fields(dt, 8192) for dt in ("f32", "bf16")}
    rows = []
    for i in range(n_cands):
        dt = ("f32", "bf16")[int(z[4 * i] % 2)]
        r = 1 + int(z[4 * i + 1] % 4)
        side = sides[int(z[4 * i + 2] % 3)]
        nv = sy_stencil_variant_count(r, CODES[dt])
        v = 1 + int(z[4 * i + 3] % nv)
        k = (1, 4)[int((z[4 * i + 3] >> 32) % 2)]
        p = stencil_params(side, side, r, 0.25, dt, variant=v)
        chunks = sy_split_rows(side, k)
        a, b, c = fields[dt]
        fn = lambda: sy_stencil_step(q.handle, p, a, b, c, chunks, r)  # noqa: E731
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        sy_meter_begin(q.handle)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps, t0 = 0, time.time()
        e0.record()
        while reps < 20 or time.time() - t0 < seconds:
            for _ in range(20):
                fn()
            reps += 20
            torch.cuda.synchronize()
        e1.record()
        torch.cuda.synchronize()
        joules, _ = sy_meter_end(q.handle)
        ms = e0.elapsed_time(e1) / reps
        label = power[(1, dt, r)] * ms * 1e-3
        rows.append({"dtype": dt, "radius": r, "side": side, "variant": v, "chunks": k, "ms": ms,
                     "j_measured": joules / reps, "j_label": label})
    del fields
    lm = np.log([x["j_measured"] for x in rows])
    ll = np.log([x["j_label"] for x in rows])
    ratio = np.exp(lm - ll)
    agree, groups = 0, 0
    keyf = lambda x: (x["dtype"], x["radius"], x["side"])  # noqa: E731
    for key in sorted({keyf(x) for x in rows}):
        g = [x for x in rows if keyf(x) == key]
        for a in range(len(g)):
            for b in range(a + 1, len(g)):
                dt_ = g[a]["ms"] - g[b]["ms"]
                de_ = g[a]["j_measured"] - g[b]["j_measured"]
                if abs(dt_) > 0.02 * max(g[a]["ms"], g[b]["ms"]):  # pairs whose times differ by > 2 %
                    groups += 1
                    agree += int((dt_ > 0) == (de_ > 0))
    return {"candidates": rows, "corr_log_j": float(np.corrcoef(lm, ll)[0, 1]),
            "ratio_measured_over_label": {"median": float(np.median(ratio)), "p10": float(np.quantile(ratio, 0.1)),
                                          "p90": float(np.quantile(ratio, 0.9)), "min": float(ratio.min()),
                                          "max": float(ratio.max())},
            "pairs_time_order_equals_energy_order": {"pairs": groups, "agree": agree},
            "group_power_w": {f"{k[1]}/r{k[2]}": v for k, v in power.items() if k[0] == 1}}


def _power_design(rows: list[dict]) -> np.ndarray:
    """Design matrix of the power model: a bias, the 13 cost features of each candidate, and a
    one-hot of its (storage, radius) group."""
    from . import DTYPE_CODES as CODES, sy_stencil_variant_info

    out = []
    for x in rows:
        code = CODES[x["dtype"]]
        tr, tc, thr = sy_stencil_variant_info(x["radius"], code, x["variant"])
        f = sy_cost_features(1, code, x["radius"], x["side"], x["side"], tr, tc, thr, x["chunks"])
        onehot = np.zeros(8)
        onehot[(0 if x["dtype"] == "f32" else 4) + x["radius"] - 1] = 1.0
        out.append(np.concatenate([[1.0], f.astype(np.float64), onehot]))
    return np.asarray(out)


def fit_power_model(check: dict, ridge: float = 1e-2) -> dict:
    """Least-squares (ridge) model of log(measured power / group power) on the candidates an
    energy_check metered one by one: log P = log P_group + design . beta.  Also reports its
    leave-one-out error against the group-power labels' own error on the same candidates."""
    rows = check["candidates"]
    X = _power_design(rows)
    y = np.log([x["j_measured"] / x["j_label"] for x in rows])  # = log(P_measured / P_group)
    A = X.T @ X + ridge * np.eye(X.shape[1])
    beta = np.linalg.solve(A, X.T @ y)
    loo_pred = []
    for i in range(len(rows)):
        m = np.ones(len(rows), bool)
        m[i] = False
        b = np.linalg.solve(X[m].T @ X[m] + ridge * np.eye(X.shape[1]), X[m].T @ y[m])
        loo_pred.append(float(X[i] @ b))
    loo_pred = np.asarray(loo_pred)
    loo = np.abs(loo_pred - y)

    def order_agreement(log_e_pred):
        """Pairs of one (storage, radius, grid) group whose measured energies differ by > 2 %:
        how many the predicted energies order the same way."""
        agree = pairs = 0
        lm = np.log([x["j_measured"] for x in rows])
        key = [(x["dtype"], x["radius"], x["side"]) for x in rows]
        for a in range(len(rows)):
            for b in range(a + 1, len(rows)):
                if key[a] != key[b] or abs(lm[a] - lm[b]) < 0.02:
                    continue
                pairs += 1
                agree += int((lm[a] > lm[b]) == (log_e_pred[a] > log_e_pred[b]))
        return {"pairs": pairs, "agree": agree}

    log_label = np.log([x["j_label"] for x in rows])
    return {"beta": beta.tolist(), "group_power_w": check["group_power_w"], "candidates": len(rows),
            "loo_abs_log_error": {"median": float(np.median(loo)), "p90": float(np.quantile(loo, 0.9)),
                                  "max": float(loo.max())},
            "group_label_abs_log_error": {"median": float(np.median(np.abs(y))),
                                          "p90": float(np.quantile(np.abs(y), 0.9)), "max": float(np.abs(y).max())},
            "energy_order_loo": order_agreement(log_label + loo_pred),
            "energy_order_group_label": order_agreement(log_label)}


def energy_labels_measured(shapes, corpus, power: dict, model: dict) -> np.ndarray:
    """log J per row = log(P_group * t) + the power model's correction for that candidate (stencils;
    SAXPY rows keep the group label)."""
    out = energy_labels(shapes, corpus, power)
    beta = np.asarray(model["beta"])
    for k, sid in enumerate(corpus["shape"]):
        s = shapes[sid]
        if s["kind"] != 1:
            continue
        onehot = np.zeros(8)
        onehot[(0 if s["dtype"] == "f32" else 4) + s["radius"] - 1] = 1.0
        out[k] += float(np.concatenate([[1.0], corpus["X"][k].astype(np.float64), onehot]) @ beta)
    return out


def split_shapes(n_shapes: int, seed: int = 11, test_fraction: float = 0.2) -> tuple[np.ndarray, np.ndarray]:
    """Held-out shapes never seen in training: a seeded permutation of the shape ids."""
    order = np.argsort(inputs.splitmix64(seed, n_shapes))
    n_test = max(1, int(round(test_fraction * n_shapes)))
    return np.sort(order[n_test:]), np.sort(order[:n_test])


def regret(shapes, corpus, pick) -> dict:
    """Mean/median/max regret of `pick(rows) -> index into rows` over the shapes in corpus."""
    regs = []
    by_kind = {0: [], 1: []}
    for sid in np.unique(corpus["shape"]):
        rows = np.nonzero(corpus["shape"] == sid)[0]
        t = np.exp(corpus["logt"][rows])
        k = pick(sid, rows)
        r = t[k] / t.min() - 1.0
        regs.append(r)
        by_kind[shapes[sid]["kind"]].append(r)
    regs = np.asarray(regs)
    return {"mean": float(regs.mean()), "median": float(np.median(regs)), "p90": float(np.quantile(regs, 0.9)),
            "max": float(regs.max()), "shapes": int(regs.size),
            "mean_stencil": float(np.mean(by_kind[1])) if by_kind[1] else None,
            "mean_saxpy": float(np.mean(by_kind[0])) if by_kind[0] else None}


def predict(models, X: np.ndarray) -> np.ndarray:
    """Predicted (log time, log energy) of candidates X: one model's, or the mean over an
    ensemble of models trained from different seeds (their ranking is steadier than any one's)."""
    if isinstance(models, (list, tuple)):
        return np.mean([sy_cost_model_predict(m, X) for m in models], axis=0)
    return sy_cost_model_predict(models, X)


def evaluate(q: Queue, model, shapes, corpus, test_ids) -> dict:
    mask = np.isin(corpus["shape"], test_ids)
    sub = {k: v[mask] for k, v in corpus.items()}
    pred = predict(model, sub["X"])

    def model_pick(sid, rows):
        return int(np.argmin(pred[rows, 0]))

    def default_pick(sid, rows):
        s = shapes[sid]
        want = default_candidate(s["kind"], s["dtype"], s.get("radius", 1))
        for j, r in enumerate(rows):
            if tuple(sub["cand"][r]) == want:
                return j
        raise KeyError(want)

    def mean_pick(sid, rows):  # expected regret of a uniformly random candidate, as a reference
        return None

    res = {"model": regret(shapes, sub, model_pick), "default": regret(shapes, sub, default_pick)}
    # the held-out shapes the model chooses worst for: the shape, its pick and the best candidate
    # (tile rows, tile cols, threads, chunks) with their measured times
    worst = []
    for sid in np.unique(sub["shape"]):
        rows = np.nonzero(sub["shape"] == sid)[0]
        t = np.exp(sub["logt"][rows])
        k, b = model_pick(sid, rows), int(np.argmin(t))
        worst.append((float(t[k] / t[b] - 1.0), int(sid), [int(x) for x in sub["cand"][rows[k]]], float(t[k]),
                      [int(x) for x in sub["cand"][rows[b]]], float(t[b])))
    worst.sort(reverse=True)
    res["worst_picks"] = [{"regret": w[0], "shape": {k: v for k, v in shapes[w[1]].items()}, "pick": w[2],
                           "pick_ms": w[3], "best": w[4], "best_ms": w[5]} for w in worst[:6]]
    # the same picks as whole-corpus throughput: work of every held-out shape (grid points of one
    # step, or SAXPY elements) over the summed measured time of the chosen configurations
    totals = {}
    for kind, name in ((1, "stencil"), (0, "saxpy")):
        work = t_model = t_default = t_best = 0.0
        for sid in np.unique(sub["shape"]):
            s = shapes[sid]
            if s["kind"] != kind:
                continue
            rows = np.nonzero(sub["shape"] == sid)[0]
            t = np.exp(sub["logt"][rows]) * 1e-3
            work += s["ny"] * s["nx"] if kind == 1 else s["n"]
            t_model += t[model_pick(sid, rows)]
            t_default += t[default_pick(sid, rows)]
            t_best += t.min()
        if work:
            totals[name] = {"per_s_model": work / t_model, "per_s_default": work / t_default,
                            "per_s_best": work / t_best, "model_over_default": t_default / t_model}
    res["held_out_totals"] = totals
    # expected regret of a random candidate
    rr = []
    for sid in np.unique(sub["shape"]):
        t = np.exp(sub["logt"][sub["shape"] == sid])
        rr.append(float(np.mean(t / t.min() - 1.0)))
    res["random_expected_mean"] = float(np.mean(rr))
    # log-time prediction error on held-out rows
    res["held_out_rmse_log_time"] = float(np.sqrt(np.mean((pred[:, 0] - sub["logt"]) ** 2)))
    return res


def train_ensemble(q: Queue, corpus, train_ids, n: int = 3, epochs: int = 300, log_energy=None) -> list:
    """n models on the same rows from seeds 7, 8, ... (initial weights and minibatch order)."""
    return [train(q, corpus, train_ids, epochs=epochs, seed=7 + i, log_energy=log_energy) for i in range(n)]


def train(q: Queue, corpus, train_ids, epochs: int = 300, batch: int = 256, lr: float = 2e-3, seed: int = 7,
          log_energy: np.ndarray | None = None) -> int:
    mask = np.isin(corpus["shape"], train_ids)
    X = corpus["X"][mask]
    T = np.stack([corpus["logt"][mask], log_energy[mask] if log_energy is not None else corpus["logt"][mask]], 1)
    model = sy_mlp_create(q.handle, F, 64, 2, seed=seed)
    sy_mlp_train(model, X, T.astype(np.float32), epochs=epochs, batch=batch, lr=lr, seed=seed)
    return model


def tile_sweep(q: Queue, n: int = 8192, reps: int = 5) -> list[dict]:
    """Every tile variant of the 2D step on one n x n chunk, per storage type and radius, with the
    library's exhaustive tuner (device timestamps, median of `reps`): GB/s of algorithmic bytes
    (3 x element size per point) for each variant and the fastest."""
    import torch

    out = []
    for dtype in ("f32", "bf16", "f16"):
        tdt = torch.float32 if dtype == "f32" else torch.int16
        a, b, c = (torch.zeros(n, n, dtype=tdt, device="cuda") for _ in range(3))
        b.copy_(torch.from_numpy(inputs.to_storage(inputs.gaussian_pulse(n, n, 64.0), dtype)
                                 .view(np.float32 if dtype == "f32" else np.int16)).cuda())
        es = 4 if dtype == "f32" else 2
        for r in (1, 2, 3, 4):
            p = stencil_params(n, n, r, 0.25, dtype)
            recs = sy_tune_stencil(q.handle, p, a, b, c, chunk_counts=(1,), reps=reps)
            gbs = {rec["variant"]: 3 * es * n * n / (rec["ms"] * 1e-3) / 1e9 for rec in recs}
            best = max(recs, key=lambda rec: gbs[rec["variant"]])
            out.append({"dtype": dtype, "radius": r, "gb_per_s": gbs, "best_variant": best["variant"],
                        "best_tile": [best["tile_rows"], best["threads"]], "best_gb_per_s": gbs[best["variant"]],
                        "default_tile": list(sy_stencil_variant_info(r, DTYPE_CODES[dtype], 0)[::2])})
        del a, b, c
    return out


def main() -> None:
    import torch

    ap = argparse.ArgumentParser()
    ap.add_argument("--tile-sweep", type=int, default=0, metavar="N",
                    help="only sweep the 2D tile variants on an N x N chunk and print one JSON line per case")
    ap.add_argument("--energy-check", type=int, default=0, metavar="N",
                    help="only meter N stencil candidates one by one (>= 1 s NVML window each) and compare "
                         "their measured energy with the corpus labels (group power x time); one JSON line")
    ap.add_argument("--energy-measured", type=int, default=0, metavar="N",
                    help="label energy with a power model fitted on N candidates metered one by one "
                         "(instead of group power x time alone)")
    ap.add_argument("--stencil", type=int, default=560)
    ap.add_argument("--saxpy", type=int, default=40)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--epochs", type=int, default=300)
    ap.add_argument("--ensemble", type=int, default=3, help="models averaged (different seeds)")
    ap.add_argument("--out", default=None, help="save the corpus (npz) here")
    ap.add_argument("--model", default=None, help="save the trained model here")
    args = ap.parse_args()
    torch.cuda.set_device(0)
    q = Queue(0)
    if args.tile_sweep:
        for rec in tile_sweep(q, args.tile_sweep):
            print(json.dumps(rec), flush=True)
        return
    if args.energy_check:
        print(json.dumps(energy_check(q, args.energy_check)), flush=True)
        return
    shapes = inputs.cost_corpus_shapes(n_stencil=args.stencil, n_saxpy=args.saxpy)
    t0 = time.time()
    corpus = measure(q, shapes, reps=args.reps, log=lambda m: print(m, flush=True))
    t_measure = time.time() - t0
    power = group_power(q)
    loge = energy_labels(shapes, corpus, power)
    pmodel = None
    if args.energy_measured:
        pmodel = fit_power_model(energy_check(q, args.energy_measured))
        loge = energy_labels_measured(shapes, corpus, power, pmodel)
    train_ids, test_ids = split_shapes(len(shapes))
    t1 = time.time()
    models = train_ensemble(q, corpus, train_ids, n=args.ensemble, epochs=args.epochs, log_energy=loge)
    t_train = time.time() - t1
    res = evaluate(q, models, shapes, corpus, test_ids)
    res["single_model"] = {k: evaluate(q, models[0], shapes, corpus, test_ids)[k] for k in ("model",)}
    model = models[0]
    res.update({"rows": int(corpus["X"].shape[0]), "shapes": len(shapes), "train_shapes": int(train_ids.size),
                "test_shapes": int(test_ids.size), "measure_s": t_measure, "train_s": t_train,
                "group_power_w": {f"{k[0]}/{k[1]}/r{k[2]}": v for k, v in power.items()}})
    if pmodel is not None:
        res["power_model"] = {k: v for k, v in pmodel.items() if k != "beta"}
    if args.out:
        np.savez(args.out, loge=loge, **corpus)
    if args.model:
        sy_mlp_save(model, args.model)
    for m in models:
        sy_mlp_destroy(m)
    print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
