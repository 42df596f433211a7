"""The CPU reference of the surrogate network against finite differences of
its own loss (the gradient) and against torch's bfloat16 conversion (the
rounding helper).  No GPU."""
import numpy as np
import pytest

from oracle import mlp_oracle as mo


def test_param_count():
    assert mo.N_PARAMS == 69639


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    theta = mo.init_params(1) + rng.normal(0, 0.05, mo.N_PARAMS)
    x = np.column_stack([rng.normal(size=(32, 6)), np.ones(32)])
    t = rng.normal(size=(32, 7))
    L, g = mo.loss_and_grad(theta, x, t)
    idx = np.concatenate([rng.choice(np.arange(0, 1792), 6, replace=False),     # W1
                          rng.choice(np.arange(1792, 2048), 3, replace=False),  # b1
                          rng.choice(np.arange(2048, 67584), 8, replace=False), # W2
                          rng.choice(np.arange(67584, 67840), 3, replace=False),# b2
                          rng.choice(np.arange(67840, 69632), 6, replace=False),# W3
                          np.arange(69632, 69639)])                             # b3
    h = 1e-5
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mo.loss_and_grad(tp, x, t)[0] - mo.loss_and_grad(tm, x, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(g[i]), (i, fd, g[i])


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    a = np.concatenate([rng.normal(size=5000) * 10.0 ** rng.integers(-8, 8, 5000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.01171875, -3.0078125]])
    ours = mo.bf16_round(a)
    ref = torch.tensor(a.astype(np.float32)).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)
    assert np.array_equal(ours, ref)


def test_forward_shapes_and_tanh_bounds():
    theta = mo.init_params(3)
    x = np.column_stack([np.linspace(-2, 2, 10)[:, None].repeat(6, 1), np.ones(10)])
    y, (h1, h2) = mo.forward(theta, x)
    assert y.shape == (10, 7) and h1.shape == (10, 256) and np.all(np.abs(h2) < 1)
