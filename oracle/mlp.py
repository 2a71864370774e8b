"""Learned CG initial guess: the per-node MLP and its data path (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The network maps 16 per-node features to a 3-component correction of a base
initial guess for step s (the method's spec form (4): the network
predicts each step's CG initial guess from the previous steps' increments):

    differences  D_k = k-th backward difference of the increments at s-1:
                 D_k = sum_j (-1)^j C(k, j) du_{s-1-j},  k = 0..3
    features  x = [D_0 / s_0, D_1 / s_1, D_2 / s_2, D_3 / s_3]  (12 values)
                  ++ [Vs / 1000, Vp / 3000, rho / 2000, h / 0.05] of the node's layer
                  (the lowest layer index among the elements touching the node)
    s_k       = RMS over all DOF of D_k (1 if that is zero)
    network   h1 = relu(x W1 + b1) (64), h2 = relu(h1 W2 + b2) (64), o = h2 W3 + b3 (3)
    base      the Newmark predictor dt v + dt^2/2 a (guess order 0), or the
              degree-k polynomial through the last k+1 increments evaluated one
              step ahead (guess order k, once k+1 increments exist)
    scale     the RMS of the previous step's correction du_{s-1} - base_{s-1}
              (s_0 if that is zero)
    guess     du0 = base + scale * o
    target    of training step s: (du_s - base_s) / RMS(du_s - base_s);
              loss = mean over the batch of |o - target|^2

Differences rather than the increments themselves: the correction is a
nearly cancelling combination of nearly equal increments, which features
rounded to bfloat16 (8 significant bits) could not resolve; each difference
normalised by its own RMS keeps its leading digits.

Training samples of step s, Adam iteration i, batch slot j are nodes
hash(seed, s, i, j) mod N, with the counter-based hash built from Wellons'
"lowbias32" integer mixer (see :func:`sample_nodes`).

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


# ----------------------------------------------------------------------------
# Data path of the learned guess: features, base guess, scale, targets
# ----------------------------------------------------------------------------


def layer_features(mesh, mat):
    """[N, 4] layer features of each node: (Vs/1000, Vp/3000, rho/2000, h/0.05)
    of the lowest layer index among the elements touching it (layer 0 for a
    node in no element)."""
    n = mesh["xyz"].shape[0]
    conn = np.asarray(mesh["conn"], dtype=np.int64)
    em = np.asarray(mesh["elem_mat"], dtype=np.int64)
    big = np.iinfo(np.int64).max
    lay = np.full(n, big, dtype=np.int64)
    for k in range(conn.shape[1]):
        np.minimum.at(lay, conn[:, k], em)
    lay[lay == big] = 0
    m = np.asarray(mat, dtype=np.float64)[lay]
    return np.stack([m[:, 1] / 1000.0, m[:, 0] / 3000.0, m[:, 2] / 2000.0, m[:, 3] / 0.05], axis=1)


def rms(x):
    x = np.asarray(x, dtype=np.float64).ravel()
    return float(np.sqrt(np.mean(x * x)))


def backward_differences(history):
    """D_k = sum_j (-1)^j C(k, j) history[j], k = 0..3 (history[0] the latest)."""
    from math import comb

    return [sum((-1) ** j * comb(k, j) * np.asarray(history[j], dtype=np.float64) for j in range(k + 1))
            for k in range(4)]


def features(history, nodef):
    """Features [N, 16] and the scales s_k [4] from ``history`` = [du_{s-1},
    du_{s-2}, du_{s-3}, du_{s-4}] (each [N, 3], latest first) and layer
    features [N, 4]."""
    D = backward_differences(history)
    sig = np.array([rms(d) for d in D])
    sig[sig == 0.0] = 1.0
    X = np.concatenate([d.reshape(-1, 3) / sg for d, sg in zip(D, sig)]
                       + [np.asarray(nodef, dtype=np.float64)], axis=1)
    return X, sig


def extrapolate(increments, k):
    """Degree-k polynomial through the last k+1 increments, one step ahead.

    ``increments[j]`` is the increment j steps back (j = 0 the latest, at
    t = 0; increment j sits at t = -j).  The polynomial is written in
    Lagrange form and evaluated at t = 1."""
    t = -np.arange(k + 1, dtype=np.float64)
    out = np.zeros_like(np.asarray(increments[0], dtype=np.float64))
    for j in range(k + 1):
        L = 1.0
        for m in range(k + 1):
            if m != j:
                L *= (1.0 - t[m]) / (t[j] - t[m])
        out = out + L * np.asarray(increments[j], dtype=np.float64)
    return out


def base_guess(v, a, dt, increments, k):
    """Base initial guess of a step: the polynomial extrapolation of order k
    when k > 0 and k+1 increments exist, else the Newmark predictor."""
    if k > 0 and len(increments) >= k + 1:
        return extrapolate(increments, k)
    return dt * np.asarray(v, dtype=np.float64) + 0.5 * dt * dt * np.asarray(a, dtype=np.float64)


def correction_scale(du, base, fallback):
    """RMS of the correction du - base, or ``fallback`` when it is zero."""
    r = rms(np.asarray(du, dtype=np.float64).ravel() - np.asarray(base, dtype=np.float64).ravel())
    return r if r > 0.0 else fallback


def targets(du, base, scale):
    """Training targets (du - base) / scale, [N, 3]."""
    return ((np.asarray(du, dtype=np.float64).ravel() - np.asarray(base, dtype=np.float64).ravel())
            / scale).reshape(-1, 3)


def learned_guess(theta, X, base, scale):
    """du0 = base + scale * o, o from the BF16 inference (:func:`forward_bf16`)."""
    return np.asarray(base, dtype=np.float64).reshape(-1, 3) + scale * forward_bf16(theta, X)


_M32 = np.uint64(0xFFFFFFFF)


def lowbias32(x):
    """Wellons' "lowbias32" 32-bit integer hash (xorshift-multiply, constants
    0x7feb352d and 0x846ca68b), on uint64 arrays holding 32-bit values."""
    x = np.asarray(x, dtype=np.uint64) & _M32
    x = x ^ (x >> np.uint64(16))
    x = (x * np.uint64(0x7FEB352D)) & _M32
    x = x ^ (x >> np.uint64(15))
    x = (x * np.uint64(0x846CA68B)) & _M32
    x = x ^ (x >> np.uint64(16))
    return x


def sample_nodes(n_nodes, batch, seed, step, it):
    """Node index of each training sample: h mod N with
    h = H(seed ^ H(step * 0x9E3779B9 ^ H(it * 0x85EBCA6B ^ j))), H = lowbias32,
    products taken modulo 2^32."""
    j = np.arange(batch, dtype=np.uint64)
    inner = lowbias32(((np.uint64(it) * np.uint64(0x85EBCA6B)) & _M32) ^ j)
    mid = lowbias32(((np.uint64(step) * np.uint64(0x9E3779B9)) & _M32) ^ inner)
    h = lowbias32(np.uint64(seed) ^ mid)
    return (h % np.uint64(n_nodes)).astype(np.int64)


def loss_grad_bf16(theta, X, Y, rnd=None):
    """Loss and gradient as the tensor-core training kernel computes them.

    Every matrix product takes its operands rounded by ``rnd`` (bfloat16,
    :func:`bf16`, by default) and sums exactly (the kernel accumulates in
    FP32): features, weights and the stored activations h1, h2 of the
    forward pass; the output error 2 (o - y) / B; the back-propagated
    dz2 = (d3 W3^T) * [z2 > 0] and dz1 = (dz2 W2^T) * [z1 > 0].  Biases and
    bias gradients are not rounded.  With ``rnd`` the identity this is
    :func:`loss_grad`."""
    r = bf16 if rnd is None else rnd
    p = unpack(theta)
    W1, W2, W3 = r(p["W1"]), r(p["W2"]), r(p["W3"])
    x = r(X)
    z1 = x @ W1 + p["b1"]
    h1 = r(np.maximum(z1, 0.0))
    z2 = h1 @ W2 + p["b2"]
    h2 = r(np.maximum(z2, 0.0))
    o = h2 @ W3 + p["b3"]
    B = X.shape[0]
    diff = o - Y
    loss = float((diff ** 2).sum() / B)
    d3 = 2.0 * diff / B
    g = {"b3": d3.sum(axis=0)}
    d3r = r(d3)
    g["W3"] = h2.T @ d3r
    dz2 = (d3r @ W3.T) * (z2 > 0)
    g["b2"] = dz2.sum(axis=0)
    dz2r = r(dz2)
    g["W2"] = h1.T @ dz2r
    dz1 = (dz2r @ W2.T) * (z1 > 0)
    g["b1"] = dz1.sum(axis=0)
    g["W1"] = x.T @ r(dz1)
    grad = np.concatenate([g[name].ravel() for name, _ in SHAPES])
    return loss, grad
