"""Learned CG initial guess: the per-node MLP (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The network maps 16 per-node features to a 3-component correction of the
standard Newmark predictor (dt v + dt^2/2 a):

    features  x = [du_{s-1}, du_{s-2}, du_{s-3}, du_{s-4}] / sigma  (12 values)
                  ++ [Vs / 1000, Vp / 3000, rho / 2000, h / 0.05] of the node's layer
    sigma     = RMS over all DOF of du_{s-1}
    network   h1 = relu(x W1 + b1) (64), h2 = relu(h1 W2 + b2) (64), o = h2 W3 + b3 (3)
    guess     du0 = dt v + dt^2/2 a + sigma * o
    target    (du_s - dt v - dt^2/2 a) / sigma, loss = mean over the batch of |o - target|^2

Parameters are packed in one vector: W1 [16,64], b1 [64], W2 [64,64], b2 [64],
W3 [64,3], b3 [3] (row-major), 5,443 values.  Training uses Adam
(beta1 0.9, beta2 0.999, eps 1e-8).
"""
import numpy as np

SHAPES = [("W1", (16, 64)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("W3", (64, 3)), ("b3", (3,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = theta[o:o + n].reshape(shape)
        o += n
    return out


def init(seed):
    """He-uniform weights (fan-in), zero biases."""
    rng = np.random.default_rng(seed)
    theta = np.zeros(N_PARAMS)
    p = unpack(theta)
    for name, shape in SHAPES:
        if name.startswith("W"):
            lim = np.sqrt(6.0 / shape[0])
            p[name][...] = rng.uniform(-lim, lim, size=shape)
    if True:  # small last layer: the initial network is close to the plain predictor
        p["W3"][...] *= 0.01
    return theta


def forward(theta, X):
    p = unpack(theta)
    z1 = X @ p["W1"] + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"] + p["b2"]
    h2 = np.maximum(z2, 0.0)
    o = h2 @ p["W3"] + p["b3"]
    return o, (X, z1, h1, z2, h2)


def loss_grad(theta, X, Y):
    """Mean squared error over the batch and its analytic gradient (backprop)."""
    p = unpack(theta)
    o, (X, z1, h1, z2, h2) = forward(theta, X)
    B = X.shape[0]
    diff = o - Y
    loss = float((diff ** 2).sum() / B)
    d3 = 2.0 * diff / B
    g = {}
    g["W3"] = h2.T @ d3
    g["b3"] = d3.sum(axis=0)
    d2 = (d3 @ p["W3"].T) * (z2 > 0)
    g["W2"] = h1.T @ d2
    g["b2"] = d2.sum(axis=0)
    d1 = (d2 @ p["W2"].T) * (z1 > 0)
    g["W1"] = X.T @ d1
    g["b1"] = d1.sum(axis=0)
    grad = np.concatenate([g[name].ravel() for name, _ in SHAPES])
    return loss, grad


def adam(theta, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (t counts from 1); returns new (theta, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def bf16(x):
    """Round float64 values to bfloat16 (round to nearest even) and back."""
    a = np.asarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_bf16(theta, X):
    """Inference as the tensor-core kernel computes it: features, weights and
    hidden activations rounded to bfloat16, biases and sums in higher precision."""
    p = unpack(theta)
    h = bf16(X)
    h = bf16(np.maximum(h @ bf16(p["W1"]) + p["b1"], 0.0))
    h = bf16(np.maximum(h @ bf16(p["W2"]) + p["b2"], 0.0))
    return h @ bf16(p["W3"]) + p["b3"]
