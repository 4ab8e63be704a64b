"""The cost model's MLP kernels (FP32, on the GPU) against the FP64 oracle:
forward, loss, gradients (checked against the oracle's backpropagation, itself
pinned by central differences), Adam; plus training, save/load and choice."""
import numpy as np
import pytest

import oracle
import paper_2505_06022_gb300 as sy
from paper_2505_06022_gb300 import inputs

from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu

F, H, O = 13, 64, 2


@pytest.fixture(scope="module")
def q():
    torch_cuda()
    with sy.Queue(0) as queue:
        yield queue.handle


def case(B, seed=1, scale=0.4):
    P = oracle.mlp_param_count(F, H, O)
    p = inputs.uniform_pm1_f32(seed, P) * np.float32(scale)
    X = inputs.uniform_pm1_f32(seed + 1, B * F).reshape(B, F) * np.float32(2.0)
    T = inputs.uniform_pm1_f32(seed + 2, B * O).reshape(B, O)
    return p, X, T


@pytest.mark.parametrize("B", [1, 7, 300, 5000])
def test_forward_and_gradients_match_oracle(q, B):
    torch = torch_cuda()
    p, X, T = case(B)
    m = sy.sy_mlp_create(q, F, H, O)
    try:
        sy.sy_mlp_set_params(m, p)
        dX, dT = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
        dY = torch.empty(B, O, device="cuda")
        sy.sy_mlp_forward(m, dX, B, dY)
        torch.cuda.synchronize()
        p64, X64, T64 = p.astype(np.float64), X.astype(np.float64), T.astype(np.float64)
        Y64 = oracle.mlp_forward(X64, p64, F, H, O)
        assert np.max(np.abs(dY.cpu().numpy() - Y64)) <= 1e-5 * max(1.0, np.max(np.abs(Y64)))
        loss = sy.sy_mlp_loss_grad(m, dX, dT, B)
        g = sy.sy_mlp_get_grad(m)
        loss64, g64 = oracle.mlp_loss_grad(X64, T64, p64, F, H, O)
        assert abs(loss - loss64) <= 1e-5 * max(1.0, loss64)
        # FP32 sums of B products against FP64: error ~ sqrt(B) * 2^-24 relative to the
        # largest gradient; 1e-4 of max|g| holds with margin up to B = 5000.
        assert np.max(np.abs(g - g64)) <= 1e-4 * np.max(np.abs(g64))
        for name, lo, hi in [("W1", 0, H * F), ("b1", H * F, H * F + H), ("W2", H * F + H, H * F + H + H * H),
                             ("W3", H * F + 2 * H + H * H, H * F + 2 * H + H * H + O * H)]:
            seg, seg64 = g[lo:hi], g64[lo:hi]
            assert np.max(np.abs(seg - seg64)) <= 1e-4 * max(np.max(np.abs(seg64)), 1e-12), name
        # fixed-shape reductions: bit-reproducible (also under the backward pass's own name)
        sy.sy_mlp_loss_grad(m, dX, dT, B, want_loss=False)
        assert np.array_equal(sy.sy_mlp_get_grad(m).view(np.uint32), g.view(np.uint32))
        assert sy.sy_mlp_backward(m, dX, dT, B) == loss
        assert np.array_equal(sy.sy_mlp_get_grad(m).view(np.uint32), g.view(np.uint32))
    finally:
        sy.sy_mlp_destroy(m)


def test_adam_matches_oracle(q):
    """Three Adam steps: the GPU's gradient at each step is applied by the GPU kernel and
    by the oracle's FP64 Adam to the same starting parameters and moments."""
    torch = torch_cuda()
    B = 64
    p, X, T = case(B, seed=9)
    m = sy.sy_mlp_create(q, F, H, O)
    try:
        sy.sy_mlp_set_params(m, p)  # also zeroes Adam's moments and step count
        dX, dT = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
        p64 = p.astype(np.float64)
        m64, v64 = np.zeros_like(p64), np.zeros_like(p64)
        for t in range(1, 4):
            sy.sy_mlp_loss_grad(m, dX, dT, B, want_loss=False)
            g = sy.sy_mlp_get_grad(m).astype(np.float64)
            sy.sy_mlp_adam_step(m, 1e-2)
            oracle.adam_step(p64, g, m64, v64, t, 1e-2)
            got = sy.sy_mlp_get_params(m)
            assert np.max(np.abs(got - p64)) <= 2e-6 * max(1.0, np.max(np.abs(p64))), t
    finally:
        sy.sy_mlp_destroy(m)


def smooth_target(X):
    return np.stack([np.log1p((X[:, :4] ** 2).sum(1)), np.sin(X[:, 4]) * X[:, 5]], 1).astype(np.float32)


def test_training_reduces_held_out_loss_and_save_load(q, tmp_path):
    n = 6000
    X = inputs.uniform_pm1_f32(31, n * F).reshape(n, F) * np.float32(2.0)
    T = smooth_target(X)
    Xtr, Ttr, Xte, Tte = X[:5000], T[:5000], X[5000:], T[5000:]
    m = sy.sy_mlp_create(q, F, H, O, seed=3)
    try:
        sy.sy_mlp_train(m, Xtr, Ttr, epochs=0, batch=256, lr=1e-3)  # fit normalisation only
        before = np.mean((sy.sy_cost_model_predict(m, Xte) - Tte) ** 2)
        sy.sy_mlp_train(m, Xtr, Ttr, epochs=150, batch=256, lr=2e-3, seed=5)
        pred = sy.sy_cost_model_predict(m, Xte)
        after = np.mean((pred - Tte) ** 2)
        assert after < 0.05 * before, (before, after)
        path = str(tmp_path / "model.bin")
        sy.sy_mlp_save(m, path)
        m2 = sy.sy_mlp_load(q, path)
        try:
            assert np.array_equal(sy.sy_cost_model_predict(m2, Xte).view(np.uint32), pred.view(np.uint32))
            k = sy.sy_cost_model_choose(m2, Xte[:50], objective=0)
            assert k == int(np.argmin(pred[:50, 0]))
            k2 = sy.sy_cost_model_choose(m2, Xte[:50], objective=2)
            assert k2 == int(np.argmin(pred[:50, 0] + pred[:50, 1]))
        finally:
            sy.sy_mlp_destroy(m2)
    finally:
        sy.sy_mlp_destroy(m)


def test_mlp_errors(q):
    with pytest.raises(sy.SyError) as e:
        sy.sy_mlp_create(q, 33, 64, 2)
    assert e.value.name == "SY_ERR_INVALID_ARGUMENT"
    with pytest.raises(sy.SyError) as e:
        sy.sy_mlp_create(q, 4, 65, 2)
    assert e.value.name == "SY_ERR_INVALID_ARGUMENT"
    m = sy.sy_mlp_create(q, 4, 8, 1)
    try:
        with pytest.raises(sy.SyError) as e:
            sy.sy_cost_model_choose(m, np.zeros((3, 4)), objective=1)  # needs an energy output
        assert e.value.name == "SY_ERR_INVALID_ARGUMENT"
        with pytest.raises(sy.SyError) as e:
            sy.sy_mlp_set_params(m, np.zeros(5))
        assert e.value.name == "SY_ERR_INVALID_ARGUMENT"
        with pytest.raises(sy.SyError) as e:
            sy.sy_mlp_load(q, "/nonexistent/model.bin")
        assert e.value.name == "SY_ERR_IO"
    finally:
        sy.sy_mlp_destroy(m)
