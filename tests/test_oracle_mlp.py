"""Pins of the learned-guess oracle: analytic backprop vs central finite
differences; Adam against closed forms over five steps; BF16 inference against
exact arithmetic on representable values and hand-made rounding cases; the
polynomial extrapolation against polynomials; features, layer features,
targets and scales against hand-built histories; the sampling hash against
its inverse."""
import numpy as np

from oracle import mlp
from synth import configs


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(0)
    theta = mlp.init(3)
    theta += 0.05 * rng.standard_normal(theta.size)  # leave the near-zero last layer
    X = rng.standard_normal((40, 16))
    Y = rng.standard_normal((40, 3))
    loss, g = mlp.loss_grad(theta, X, Y)
    idx = rng.choice(theta.size, 60, replace=False)
    for i in idx:
        e = np.zeros_like(theta)
        h = 1e-6 * max(1.0, abs(theta[i]))
        e[i] = h
        fd = (mlp.loss_grad(theta + e, X, Y)[0] - mlp.loss_grad(theta - e, X, Y)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, i
    assert mlp.N_PARAMS == 5443


def test_adam_first_step_is_lr_times_sign():
    g = np.array([0.3, -2.0, 1e-3])
    th, m, v = mlp.adam(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    np.testing.assert_allclose(th, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 3.14159265, -2.5e-3])
    r = mlp.bf16(x)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2 ** -7  # tie to even, exact
    assert abs(r[3] - 3.140625) < 1e-12
    assert np.all(np.abs(r - x) <= np.abs(x) * 2 ** -8)


def test_adam_closed_form_over_five_steps():
    """Adam over t = 1..5 against closed forms.  Constant gradient g: m_t = (1 - b1^t) g,
    v_t = (1 - b2^t) g^2, so every bias-corrected step is lr g / (|g| + eps).  Alternating
    gradient (-1)^t g: m_t = (1 - b1) g (-1)^t (1 - (-b1)^t) / (1 + b1) (a geometric sum),
    v_t as before, so the step depends on b1 and on both bias corrections."""
    b1, b2, eps, lr = 0.9, 0.999, 1e-8, 0.01
    g = np.array([0.3, -2.0, 1e-3, 7.5])
    th, m, v = np.zeros(4), np.zeros(4), np.zeros(4)
    for t in range(1, 6):
        th, m, v = mlp.adam(th, g, m, v, t, lr)
        np.testing.assert_allclose(m, (1 - b1 ** t) * g, rtol=1e-13)
        np.testing.assert_allclose(v, (1 - b2 ** t) * g * g, rtol=1e-13)
        np.testing.assert_allclose(th, -t * lr * g / (np.abs(g) + eps), rtol=1e-12)
    th, m, v = np.zeros(4), np.zeros(4), np.zeros(4)
    expect = np.zeros(4)
    for t in range(1, 6):
        gt = (-1) ** t * g
        th, m, v = mlp.adam(th, gt, m, v, t, lr)
        m_ref = (1 - b1) * g * (-1) ** t * (1 - (-b1) ** t) / (1 + b1)
        np.testing.assert_allclose(m, m_ref, rtol=1e-12)
        np.testing.assert_allclose(v, (1 - b2 ** t) * g * g, rtol=1e-13)
        expect -= lr * (m_ref / (1 - b1 ** t)) / (np.abs(g) + eps)
        np.testing.assert_allclose(th, expect, rtol=1e-12)
    # the second step already differs from a sign step
    assert abs(expect[0]) < 2 * lr * 0.9


def _bf16_exact_net(rng):
    """Weights that are multiples of 1/4 with few nonzeros per column, so that with
    small-integer features every pre-activation is a multiple of 1/16 below 16 in
    magnitude: exactly representable in bfloat16 (8 significant bits)."""
    theta = np.zeros(mlp.N_PARAMS)
    p = mlp.unpack(theta)
    for name, (fan_in, fan_out) in (("W1", (16, 64)), ("W2", (64, 64)), ("W3", (64, 3))):
        for j in range(fan_out):
            rows = rng.choice(fan_in, 2, replace=False)
            p[name][rows, j] = rng.choice([-0.5, -0.25, 0.25, 0.5], 2)
    p["b1"][...] = rng.integers(-4, 5, 64) / 4.0
    p["b2"][...] = rng.integers(-4, 5, 64) / 4.0
    p["b3"][...] = rng.standard_normal(3)  # biases stay in higher precision
    return theta


def test_forward_bf16_equals_forward_on_representable_values():
    rng = np.random.default_rng(11)
    theta = _bf16_exact_net(rng)
    X = rng.integers(-3, 4, (50, 16)).astype(np.float64)
    o, (_, z1, _, z2, _) = mlp.forward(theta, X)
    for z in (z1, z2):
        assert np.array_equal(mlp.bf16(z), z)
    assert np.array_equal(mlp.forward_bf16(theta, X), o)


def test_forward_bf16_rounds_features_weights_and_activations():
    """One path through the network, values chosen so that each rounding stage shows."""
    theta = np.zeros(mlp.N_PARAMS)
    p = mlp.unpack(theta)
    p["W1"][0, 0] = 1.0
    p["b1"][0] = 2.0 ** -9          # z1 = x + 2^-9: the activation rounds back to x
    p["W2"][0, 0] = 1.0 + 2.0 ** -9  # the weight rounds to 1
    p["W3"][0, 0] = 1.0
    p["b3"][0] = 0.125
    X = np.zeros((2, 16))
    X[0, 0] = 1.0 + 2.0 ** -9       # the feature rounds to 1
    X[1, 0] = 3.0
    out = mlp.forward_bf16(theta, X)
    assert out[0, 0] == 1.0 + 0.125 and out[1, 0] == 3.0 + 0.125
    ref = mlp.forward(theta, X)[0]
    assert ref[0, 0] > 1.125 and ref[1, 0] > 3.125


def test_extrapolation_exact_on_polynomials():
    """The degree-k extrapolation reproduces every polynomial of degree <= k in the step
    index exactly, and misses degree k + 1 by (k+1)! times its leading coefficient."""
    rng = np.random.default_rng(3)
    for k in range(0, 7):
        coef = rng.standard_normal((k + 2, 5))
        poly = lambda t, d: sum(coef[i] * t ** i for i in range(d + 1))
        incs = [poly(-j, k) for j in range(k + 1)]
        np.testing.assert_allclose(mlp.extrapolate(incs, k), poly(1, k), rtol=1e-10, atol=1e-10)
        incs2 = [poly(-j, k + 1) for j in range(k + 1)]
        miss = poly(1, k + 1) - mlp.extrapolate(incs2, k)
        fact = np.prod(np.arange(1, k + 2, dtype=np.float64))
        np.testing.assert_allclose(miss, fact * coef[k + 1], rtol=1e-9, atol=1e-9)
    # order 0 repeats the latest increment; the predictor applies while history is short
    np.testing.assert_array_equal(mlp.extrapolate([np.arange(3.0)], 0), np.arange(3.0))
    v, a = np.ones(6), 2 * np.ones(6)
    np.testing.assert_allclose(mlp.base_guess(v, a, 0.1, [np.zeros(6)] * 2, 3), 0.1 + 0.01)


def test_features_are_normalised_backward_differences():
    """A cubic history du_{s-1-j} = (j + 1)^3 = 1, 8, 27, 64 has backward differences
    1, -7, 12, -6 (constant over the nodes), so every scaled difference is +-1: this
    pins the slot order, the difference formula and the per-difference scale."""
    N = 7
    hist = [np.full((N, 3), float((j + 1) ** 3)) for j in range(4)]
    nodef = np.arange(4 * N, dtype=np.float64).reshape(N, 4)
    X, sig = mlp.features(hist, nodef)
    np.testing.assert_array_equal(sig, [1.0, 7.0, 12.0, 6.0])
    np.testing.assert_array_equal(X[:, :12], np.repeat([1.0, -1.0, 1.0, -1.0], 3)[None].repeat(N, 0))
    np.testing.assert_array_equal(X[:, 12:], nodef)
    # a quadratic history has a zero third difference: its scale falls back to 1
    X, sig = mlp.features([np.full((N, 3), float((j + 1) ** 2)) for j in range(4)], nodef)
    assert sig[3] == 1.0 and np.abs(X[:, 9:12]).max() == 0.0
    # features do not change when all increments are scaled
    rng = np.random.default_rng(0)
    hist = [rng.standard_normal((N, 3)) for _ in range(4)]
    X1, s1 = mlp.features(hist, nodef)
    X2, s2 = mlp.features([-250.0 * h for h in hist], nodef)
    np.testing.assert_allclose(X2[:, :12], -X1[:, :12], rtol=1e-13)
    np.testing.assert_allclose(s2, 250.0 * s1, rtol=1e-13)
    # Newton's backward form: a cubic history f(tau) = (1 - tau)^3 (tau = 0 the latest
    # step, tau = -j the step j back) is extrapolated exactly by D_0 + ... + D_3 = f(1) = 0
    D = mlp.backward_differences([np.full(3, float((j + 1) ** 3)) for j in range(4)])
    np.testing.assert_allclose(sum(D), 0.0, atol=1e-12)


def test_layer_features_take_the_lowest_layer():
    cfg = configs.small_box(nx=3, ny=2, distort=False)
    mesh, mat = cfg["mesh"], cfg["mat"]
    F = mlp.layer_features(mesh, mat)
    depth = -mesh["xyz"][:, 2]
    itf = 12.0
    upper = depth <= itf + 1e-9  # interface nodes touch layer-0 elements
    np.testing.assert_allclose(F[upper], np.tile([mat[0, 1] / 1000, mat[0, 0] / 3000, mat[0, 2] / 2000,
                                                  mat[0, 3] / 0.05], (upper.sum(), 1)))
    np.testing.assert_allclose(F[~upper], np.tile([mat[1, 1] / 1000, mat[1, 0] / 3000, mat[1, 2] / 2000,
                                                   mat[1, 3] / 0.05], ((~upper).sum(), 1)))
    assert upper.any() and (~upper).any()


def test_targets_and_scale():
    rng = np.random.default_rng(4)
    du = rng.standard_normal((9, 3))
    base = du + 1e-3 * rng.standard_normal((9, 3))
    s = mlp.correction_scale(du, base, 5.0)
    np.testing.assert_allclose(s, np.sqrt(np.mean((du - base) ** 2)), rtol=1e-14)
    T = mlp.targets(du, base, s)
    np.testing.assert_allclose(np.sqrt(np.mean(T ** 2)), 1.0, rtol=1e-12)
    # an exact base: zero correction, zero targets, the scale falls back to sigma
    assert mlp.correction_scale(du, du, 5.0) == 5.0
    assert np.abs(mlp.targets(du, du, 5.0)).max() == 0.0


def test_sample_hash_is_a_bijection_and_spreads():
    """lowbias32 is a composition of invertible maps on 32-bit words (xorshifts and
    multiplications by odd constants): invert it step by step and recover the input."""
    x = np.arange(0, 1 << 16, dtype=np.uint64) * np.uint64(65537)
    h = mlp.lowbias32(x)
    M = (1 << 32) - 1

    def unxorshift(y, s):
        out = y.copy()
        for _ in range(32 // s + 1):
            out = y ^ (out >> np.uint64(s))
        return out

    y = unxorshift(h, 16)
    y = (y * np.uint64(pow(0x846CA68B, -1, 1 << 32))) & np.uint64(M)
    y = unxorshift(y, 15)
    y = (y * np.uint64(pow(0x7FEB352D, -1, 1 << 32))) & np.uint64(M)
    y = unxorshift(y, 16)
    np.testing.assert_array_equal(y, x)
    nodes = mlp.sample_nodes(1000, 65536, seed=7, step=3, it=1)
    assert nodes.min() >= 0 and nodes.max() < 1000
    counts = np.bincount(nodes, minlength=1000)
    assert counts.min() > 30 and counts.max() < 110  # 65.5 expected per node
    assert not np.array_equal(nodes, mlp.sample_nodes(1000, 65536, seed=7, step=4, it=1))


def test_bf16_gradient_is_the_exact_gradient_without_rounding_and_close_with_it():
    rng = np.random.default_rng(12)
    theta = mlp.init(4) + 0.05 * rng.standard_normal(mlp.N_PARAMS)
    X = rng.standard_normal((96, 16))
    Y = rng.standard_normal((96, 3))
    loss, g = mlp.loss_grad(theta, X, Y)
    loss_i, g_i = mlp.loss_grad_bf16(theta, X, Y, rnd=lambda a: np.asarray(a, dtype=np.float64))
    assert loss_i == loss and np.array_equal(g_i, g)
    loss_b, g_b = mlp.loss_grad_bf16(theta, X, Y)
    assert abs(loss_b - loss) <= 2e-2 * loss
    assert np.linalg.norm(g_b - g) <= 3e-2 * np.linalg.norm(g)
    # the rounding really happens: bf16 differs from the exact gradient
    assert np.linalg.norm(g_b - g) > 1e-5 * np.linalg.norm(g)


def test_bf16_gradient_rounds_the_back_propagated_error():
    """One-unit path: the output error 2 (o - y) / B is rounded before it multiplies
    the weights, so a weight gradient carries bfloat16 precision."""
    theta = np.zeros(mlp.N_PARAMS)
    p = mlp.unpack(theta)
    p["W1"][0, 0] = 1.0
    p["W2"][0, 0] = 1.0
    p["W3"][0, 0] = 1.0
    X = np.zeros((1, 16))
    X[0, 0] = 1.0
    Y = np.zeros((1, 3))
    Y[0, 0] = 1.0 - 2.0 ** -10  # o - y = 2^-10 exactly; 2(o - y) = 2^-9
    loss, g = mlp.loss_grad_bf16(theta, X, Y)
    W3 = mlp.unpack(g)["W3"]
    assert W3[0, 0] == 2.0 ** -9  # h2 = 1
    Y[0, 0] = 1.0 - 3.0 * 2.0 ** -12  # 2(o - y) = 1.5 * 2^-10, representable
    assert mlp.unpack(mlp.loss_grad_bf16(theta, X, Y)[1])["W3"][0, 0] == 1.5 * 2.0 ** -10
    Y[0, 0] = 1.0 - (1.0 + 2.0 ** -9) * 2.0 ** -11  # 2(o - y) = (1 + 2^-9) 2^-10 rounds to 2^-10
    assert mlp.unpack(mlp.loss_grad_bf16(theta, X, Y)[1])["W3"][0, 0] == 2.0 ** -10
    assert mlp.unpack(mlp.loss_grad(theta, X, Y)[1])["W3"][0, 0] == (1.0 + 2.0 ** -9) * 2.0 ** -10
