"""The surrogate network's CUDA forward, loss and gradient against the CPU
reference (same weights, the same BF16 rounding points), and training on the
GPU.  Tolerances: outputs and loss within 2e-4 relative to their scale, every
gradient block within 2e-3 of its largest entry (FP32 accumulation order)."""
import numpy as np
import pytest

from oracle import mlp_oracle as mo
from paper_2407_11349_gb300.hawkes import MLP

pytestmark = pytest.mark.gpu

BLOCKS = [(0, 1792), (1792, 2048), (2048, 67584), (67584, 67840), (67840, 69632), (69632, 69639)]


@pytest.mark.parametrize("B", [64, 192, 1024])
def test_forward_backward_match_reference(B):
    rng = np.random.default_rng(B)
    theta = (mo.init_params(5) + rng.normal(0, 0.02, mo.N_PARAMS)).astype(np.float32)
    x = np.column_stack([rng.normal(size=(B, 6)), np.ones(B)]).astype(np.float32)
    t = rng.normal(size=(B, 7)).astype(np.float32)
    net = MLP(0, seed=1)
    try:
        net.set_params(theta)
        assert np.array_equal(net.get_params(), theta)
        L, g, Y = net.loss_grad(x, t)
    finally:
        net.close()
    th64, x64, t64 = theta.astype(np.float64), x.astype(np.float64), t.astype(np.float64)
    yref, _ = mo.forward(th64, x64, bf16=True)
    Lref, gref = mo.loss_and_grad(th64, x64, t64, bf16=True)
    assert np.max(np.abs(Y - yref)) <= 2e-4 * np.max(np.abs(yref))
    assert abs(L - Lref) <= 2e-4 * Lref
    for a, b in BLOCKS:
        scale = np.max(np.abs(gref[a:b]))
        assert np.max(np.abs(g[a:b] - gref[a:b])) <= 2e-3 * scale, (a, b)


def test_training_fits_a_smooth_function():
    rng = np.random.default_rng(7)
    n = 4000
    centre = np.log([0.5, 20, 7, 0.3, 0.2, 2])
    spread = np.array([0.1, 0.2, 0.3, 0.1, 0.2, 0.4])
    X = rng.normal(size=(n, 6)) * spread + centre

    def f(X):  # a smooth log-likelihood surface and its gradient
        z = (X - centre) / spread
        ell = -1e6 + 500 * np.sum(z, 1) - 300 * np.sum(z ** 2, 1)
        grad = (500 - 600 * z) / spread
        return np.column_stack([ell, grad])

    Y = f(X)
    net = MLP(0, seed=3)
    try:
        net.set_data(X, Y)
        st = net.stats()
        assert np.allclose(st[:6], X.mean(0)) and np.allclose(st[6:12], X.std(0))
        l0 = net.train(1, batch=256, lr=1e-3, seed=1)
        l1 = net.train(3000, batch=256, lr=1e-3, seed=1)
        assert l1 < 0.05 * l0 and l1 < 5e-3
        torch = pytest.importorskip("torch")
        q = rng.normal(size=(100, 6)) * spread + centre
        dq = torch.tensor(q, dtype=torch.float64, device="cuda")
        dout = torch.zeros((100, 7), dtype=torch.float64, device="cuda")
        net.predict(dq.data_ptr(), 100, dout.data_ptr())
        net.wait()
        pred = dout.cpu().numpy()
        true = f(q)
        err = np.abs(pred - true) / Y.std(0)
        assert np.median(err) < 0.05
    finally:
        net.close()


@pytest.mark.parametrize("feature", [False, True])
def test_predict_matches_reference_element_by_element(feature):
    """hawkes_mlp_predict against the reference forward pass after the same
    standardisation: inputs (q - mean_in) / sd_in with the seventh input
    appended (the constant 1, or the standardised feature (f - mean_f) /
    sd_f), outputs mean_out + sd_out * y, with the network's stored weights
    and the GPU's BF16 rounding points; every element within 2e-4 of its
    column's output scale (sd_out)."""
    torch = pytest.importorskip("torch")
    from paper_2407_11349_gb300.hawkes import HawkesError
    rng = np.random.default_rng(17)
    X = rng.normal(size=(500, 6)) * np.array([0.1, 0.2, 0.3, 0.1, 0.2, 0.4]) + np.log([0.5, 20, 7, 0.3, 0.2, 2])
    Y = np.column_stack([rng.normal(-1e6, 300.0, 500), rng.normal(0, 50.0, (500, 6))])
    F = rng.normal(-1e6, 40.0, 500) if feature else None
    net = MLP(0, seed=9)
    try:
        net.set_data(X, Y, F)
        net.train(200, batch=128, lr=1e-3, seed=2)
        theta = net.get_params().astype(np.float64)
        st = net.stats()
        q = X[:77] + rng.normal(0, 0.05, (77, 6))
        f = F[:77] + rng.normal(0, 5.0, 77) if feature else None
        dq = torch.tensor(q, dtype=torch.float64, device="cuda")
        df = torch.tensor(f, dtype=torch.float64, device="cuda") if feature else None
        dout = torch.zeros((77, 7), dtype=torch.float64, device="cuda")
        with pytest.raises(HawkesError):  # the feature must be given exactly when trained with one
            net.predict(dq.data_ptr(), 77, dout.data_ptr(), 0 if feature else dq.data_ptr())
        net.predict(dq.data_ptr(), 77, dout.data_ptr(), df.data_ptr() if feature else 0)
        net.wait()
        got = dout.cpu().numpy()
    finally:
        net.close()
    if feature:
        assert abs(st[26] - F.mean()) < 1e-9 * abs(F.mean()) and abs(st[27] - F.std()) < 1e-6 * F.std()
    else:
        assert st[26] == 0.0 and st[27] == 1.0
    xs = (q - st[:6]) / st[6:12]
    z = ((f - st[26]) / st[27]).astype(np.float32).astype(np.float64) if feature else np.ones(77)
    xin = np.column_stack([xs.astype(np.float32).astype(np.float64), z])
    y, _ = mo.forward(theta, xin, bf16=True)
    want = st[12:19] + st[19:26] * y
    err = np.abs(got - want) / st[19:26]
    assert np.max(err) <= 2e-4, np.max(err, axis=0)
