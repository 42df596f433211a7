"""The CPU reference of the surrogate network against finite differences of
its own loss (the gradient), against torch's bfloat16 conversion (the
rounding helper), and its forward pass against two formulations that share
nothing with it: torch's float64 linear layers, and the network's sums
written out neuron by neuron.  No GPU."""
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


def _asymmetric_theta(seed):
    """Weights with no symmetry a transposed matrix could hide behind: W2 is
    far from symmetric (its transpose differs in every entry)."""
    rng = np.random.default_rng(seed)
    th = mo.init_params(seed) + rng.normal(0, 0.05, mo.N_PARAMS)
    P = mo.unflatten(th)
    P["W2"] = P["W2"] + np.triu(np.full((256, 256), 0.02), 1)  # W2 - W2^T has no zero off the diagonal
    P["b1"] = rng.normal(0, 0.3, 256)
    P["b2"] = rng.normal(0, 0.3, 256)
    P["b3"] = rng.normal(0, 0.3, 7)
    assert np.min(np.abs(P["W2"] - P["W2"].T)[np.triu_indices(256, 1)]) > 0
    return mo.flatten(P), P


def test_forward_matches_torch_linear_layers():
    """y = linear(tanh(linear(tanh(linear(x, W1, b1)), W2, b2)), W3, b3), with
    torch's convention linear(x, W, b) = x W^T + b for W of shape [out, in]."""
    torch = pytest.importorskip("torch")
    import torch.nn.functional as F
    th, P = _asymmetric_theta(11)
    rng = np.random.default_rng(12)
    x = np.column_stack([rng.normal(size=(40, 6)), np.ones(40)])
    T = {k: torch.tensor(v, dtype=torch.float64) for k, v in P.items()}
    xt = torch.tensor(x, dtype=torch.float64)
    y = F.linear(torch.tanh(F.linear(torch.tanh(F.linear(xt, T["W1"], T["b1"])), T["W2"], T["b2"])),
                 T["W3"], T["b3"]).numpy()
    ours, _ = mo.forward(th, x)
    assert np.allclose(ours, y, rtol=1e-12, atol=1e-12)
    # a transposed W2 changes the outputs grossly: the check can fail
    P2 = dict(P)
    P2["W2"] = P["W2"].T
    bad, _ = mo.forward(mo.flatten(P2), x)
    assert np.max(np.abs(bad - y)) > 1e-2


def test_forward_matches_neuron_by_neuron_sums():
    """For two inputs, every unit's value as its defining sum, loop by loop:
    h1_i = tanh(b1_i + sum_m W1[i, m] x_m), h2_j = tanh(b2_j + sum_i W2[j, i] h1_i),
    y_k = b3_k + sum_j W3[k, j] h2_j."""
    import math
    th, P = _asymmetric_theta(13)
    rng = np.random.default_rng(14)
    xs = np.column_stack([rng.normal(size=(2, 6)), np.ones(2)])
    ours, _ = mo.forward(th, xs)
    for r in range(2):
        x = [float(v) for v in xs[r]]
        h1 = [math.tanh(P["b1"][i] + sum(P["W1"][i, m] * x[m] for m in range(7))) for i in range(256)]
        h2 = [math.tanh(P["b2"][j] + sum(P["W2"][j, i] * h1[i] for i in range(256))) for j in range(256)]
        y = [P["b3"][k] + sum(P["W3"][k, j] * h2[j] for j in range(256)) for k in range(7)]
        assert np.allclose(ours[r], y, rtol=1e-12, atol=1e-12)
