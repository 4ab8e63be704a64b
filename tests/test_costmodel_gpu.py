"""Exhaustive tuner and the learned cost model (a reduced corpus measured by the
library, an MLP trained on the GPU by the library's kernels), judged by regret on
shapes held out from training -- and compared with the method without the model
(the library's default configuration)."""
import numpy as np
import pytest

import paper_2505_06022_gb300 as sy
from paper_2505_06022_gb300 import costmodel, inputs

from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def queue():
    torch_cuda()
    q = sy.Queue(0)
    yield q
    q.close()


def test_tuner_records_are_complete_and_sane(queue):
    torch = torch_cuda()
    ny, nx = 1024, 2048
    a, b, c = (torch.zeros(ny, nx, device="cuda") for _ in range(3))
    p = sy.stencil_params(ny, nx, 2, 0.25, "f32")
    recs = sy.sy_tune_stencil(queue.handle, p, a, b, c, (1, 4), reps=3)
    assert len(recs) == 2 * sy.sy_stencil_variant_count(2, sy.SY_F32)
    assert all(r["ms"] > 0 for r in recs)
    assert {r["chunks"] for r in recs} == {1, 4}
    x, y, z = (torch.zeros(1 << 22, device="cuda") for _ in range(3))
    srec = sy.sy_tune_saxpy(queue.handle, 1 << 22, x, y, z, (1, 2), reps=2)
    assert len(srec) == 2 * sy.sy_saxpy_variant_count() and all(r["ms"] > 0 for r in srec)
    # every SAXPY variant computes the same bits
    xv, yv = inputs.saxpy_inputs(100003, seed=1)
    xd, yd = torch.from_numpy(xv).cuda(), torch.from_numpy(yv).cuda()
    ref = None
    for v in range(0, sy.sy_saxpy_variant_count() + 1):
        zd = torch.empty_like(xd)
        sy.sy_saxpy_config(queue.handle, xv.size, 2.5, xd, yd, zd, v, sy.sy_split_rows(xv.size, 3))
        torch.cuda.synchronize()
        got = zd.cpu().numpy().view(np.uint32)
        ref = got if ref is None else ref
        assert np.array_equal(got, ref)


def test_features_are_finite_and_distinguish_candidates():
    f1 = sy.sy_cost_features(1, sy.SY_F32, 2, 1000, 3000, 4, 128, 256, 1)
    f2 = sy.sy_cost_features(1, sy.SY_F32, 2, 1000, 3000, 8, 128, 256, 4)
    f3 = sy.sy_cost_features(0, sy.SY_F32, 0, 1, 1 << 20, 1, 4, 256, 1)
    assert f1.shape == (sy.SY_COST_FEATURES,) and np.isfinite(np.stack([f1, f2, f3])).all()
    assert not np.array_equal(f1, f2) and f3[0] == 0 and f1[0] == 1


def test_learned_model_beats_the_default_on_held_out_shapes(queue):
    shapes = inputs.cost_corpus_shapes(n_stencil=200, n_saxpy=20, side_hi=8192, n_hi=1 << 26)
    corpus = costmodel.measure(queue, shapes, reps=3)
    train_ids, test_ids = costmodel.split_shapes(len(shapes))
    models = costmodel.train_ensemble(queue, corpus, train_ids, n=3, epochs=250)
    try:
        res = costmodel.evaluate(queue, models, shapes, corpus, test_ids)
        one = costmodel.evaluate(queue, models[0], shapes, corpus, test_ids)
    finally:
        for m in models:
            sy.sy_mlp_destroy(m)
    assert one["model"]["mean"] <= 0.10, one  # each model alone is already a good chooser
    # the model's pick is close to the exhaustive optimum and better than the fixed default
    assert res["model"]["mean"] <= 0.10, res
    assert res["model"]["mean"] < res["default"]["mean"], res
    assert res["model"]["mean"] < 0.1 * res["random_expected_mean"], res
    # and as whole-corpus throughput: the model's picks beat the default's over the held-out stencils
    tot = res["held_out_totals"]["stencil"]
    assert tot["per_s_model"] > tot["per_s_default"] and tot["per_s_model"] <= tot["per_s_best"] * (1 + 1e-12), tot


def test_exhaustive_tuner_every_kind(queue):
    """sy_tune_exhaustive: the complete candidate list of each kind (SAXPY, 2D step, 3D step) and
    the index of the fastest record."""
    torch = torch_cuda()
    x, y, z = (torch.zeros(1 << 20, device="cuda") for _ in range(3))
    recs, best = sy.sy_tune_exhaustive(queue.handle, sy.SY_TUNE_SAXPY, None, 1 << 20, x, y, z, (1, 2), reps=2)
    assert len(recs) == 2 * sy.sy_saxpy_variant_count()
    ny, nx = 512, 1024
    a, b, c = (torch.zeros(ny, nx, device="cuda") for _ in range(3))
    p = sy.stencil_params(ny, nx, 1, 0.25, "f32")
    recs2, best2 = sy.sy_tune_exhaustive(queue.handle, sy.SY_TUNE_STENCIL, p, 0, a, b, c, (1, 4), reps=2)
    assert len(recs2) == 2 * sy.sy_stencil_variant_count(1, sy.SY_F32)
    n3 = 128
    a3, b3, c3 = (torch.zeros(n3 * n3 * n3, device="cuda") for _ in range(3))
    p3 = sy.stencil3d_params(n3, n3, n3, 1, 0.125, "f32")
    recs3, best3 = sy.sy_tune_exhaustive(queue.handle, sy.SY_TUNE_STENCIL3D, p3, 0, a3, b3, c3, (1, 4), reps=2)
    assert len(recs3) == 2 * sy.sy_stencil3d_variant_count(1, "f32")
    assert {(r[0], r[4]) for r in recs3} == {(v, k) for v in range(1, 11) for k in (1, 4)}
    for rs, bi in ((recs, best), (recs2, best2), (recs3, best3)):
        assert all(r[5] > 0 for r in rs)
        assert rs[bi][5] == min(r[5] for r in rs)
    with pytest.raises(sy.SyError) as e:
        sy.sy_tune_exhaustive(queue.handle, 7, None, 1, x, y, z, (1,), reps=1)
    assert e.value.name == "SY_ERR_INVALID_ARGUMENT"
