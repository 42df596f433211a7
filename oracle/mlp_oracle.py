"""CPU reference of the surrogate network: a 7 -> 256 -> 256 -> 7 multilayer
perceptron with tanh hidden units, its mean-squared-error loss and the
gradient of that loss in every weight, in float64 numpy.

TEST INFRASTRUCTURE: only the tests compare the CUDA network against it.

The GPU network stores its weights in bfloat16 for the two tensor-core
products and rounds the activations that enter them to bfloat16; with
``bf16=True`` this reference rounds the same quantities at the same points
(weights of the 256 x 256 layer, the first hidden activations, the second
layer's error signal), so the two differ only by float32 accumulation order.

Parameters (flattened in this order, the layout of the CUDA library):
  W1 [256, 7], b1 [256], W2 [256, 256], b2 [256], W3 [7, 256], b3 [7]
Forward:   h1 = tanh(x W1^T + b1), h2 = tanh(h1 W2^T + b2), y = h2 W3^T + b3
Loss:      L = mean over the batch and the 7 outputs of (y - t)^2
"""
import numpy as np

D_IN, D_H, D_OUT = 7, 256, 7
SHAPES = [("W1", (D_H, D_IN)), ("b1", (D_H,)), ("W2", (D_H, D_H)), ("b2", (D_H,)),
          ("W3", (D_OUT, D_H)), ("b3", (D_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unflatten(theta):
    out, k = {}, 0
    for name, shp in SHAPES:
        m = int(np.prod(shp))
        out[name] = np.asarray(theta[k:k + m], dtype=np.float64).reshape(shp)
        k += m
    return out


def flatten(parts):
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def bf16_round(a):
    """Round float64 values to the nearest bfloat16 (ties to even), via float32."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(theta, x, bf16=False):
    P = unflatten(theta)
    r = bf16_round if bf16 else (lambda a: a)
    z1 = x @ P["W1"].T + P["b1"]
    h1 = np.tanh(z1)
    z2 = r(h1) @ r(P["W2"]).T + P["b2"]
    h2 = np.tanh(z2)
    y = h2 @ P["W3"].T + P["b3"]
    return y, (h1, h2)


def loss_and_grad(theta, x, t, bf16=False):
    """MSE loss and its gradient (flattened like theta)."""
    P = unflatten(theta)
    r = bf16_round if bf16 else (lambda a: a)
    y, (h1, h2) = forward(theta, x, bf16)
    B = x.shape[0]
    diff = y - t
    L = np.mean(diff ** 2)
    dy = 2.0 * diff / (B * D_OUT)
    g = {}
    g["W3"] = dy.T @ h2
    g["b3"] = dy.sum(axis=0)
    dz2 = (dy @ P["W3"]) * (1.0 - h2 ** 2)
    g["W2"] = r(dz2).T @ r(h1)
    g["b2"] = dz2.sum(axis=0)
    dz1 = (r(dz2) @ r(P["W2"])) * (1.0 - h1 ** 2)
    g["W1"] = dz1.T @ x
    g["b1"] = dz1.sum(axis=0)
    return L, flatten(g)


def init_params(seed):
    """Glorot-uniform weights, zero biases (a reference initialisation)."""
    rng = np.random.default_rng(seed)
    parts = {}
    for name, shp in SHAPES:
        if name.startswith("W"):
            lim = np.sqrt(6.0 / (shp[0] + shp[1]))
            parts[name] = rng.uniform(-lim, lim, size=shp)
        else:
            parts[name] = np.zeros(shp)
    return flatten(parts)
