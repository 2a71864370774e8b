"""Pins of the oracle's input-wave estimation, ERR and selection (CPU only).

* the paper's worked example of Eq. (2): a 5 % amplitude error gives
  ERR = 0.05 (golden file with its citation);
* the inverse crime: observations synthesised from the Green's functions
  and known coefficients are reproduced exactly (c = c*, ERR ~ 0);
* optimality: the estimate satisfies the normal equations' orthogonality
  (weighted residual orthogonal to every shifted Green's function);
* the truncated pseudo-inverse against numpy's SVD-based pinv;
* selection by minimum ERR and by historical maximum, ties to the lowest index.
"""
import os

import numpy as np

from oracle import misfit

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "err_worked_example.txt")


def _random_G(n_rec=4, n_t=120, seed=0):
    rng = np.random.default_rng(seed)
    t = np.arange(n_t)
    G = np.zeros((n_rec, 3, 3, n_t))
    for k in range(n_rec):
        for i in range(3):
            for j in range(3):
                f = rng.uniform(0.02, 0.1)
                G[k, i, j] = rng.standard_normal() * np.sin(2 * np.pi * f * t + rng.uniform(0, 6)) * np.exp(-t / 60.0)
    return G


def test_worked_example_from_paper():
    rows = np.loadtxt(GOLDEN)
    rng = np.random.default_rng(1)
    obs = rng.standard_normal((9, 3, 200))
    for scale, expected in rows:
        assert abs(misfit.err(scale * obs, obs) - expected) < 1e-14


def test_inverse_crime_recovers_coefficients():
    G = _random_G()
    s, L = 7, 6
    rng = np.random.default_rng(2)
    c_true = rng.standard_normal((3, L))
    obs = misfit.superpose(G, c_true, s)
    e, c = misfit.estimate(G, obs, s, L, tau=1e-12)
    np.testing.assert_allclose(c, c_true, rtol=0, atol=1e-8)
    assert e < 1e-8


def test_estimate_satisfies_weighted_orthogonality():
    G = _random_G(seed=3)
    s, L = 5, 8
    obs = np.random.default_rng(4).standard_normal((4, 3, 120))
    e, c = misfit.estimate(G, obs, s, L, tau=1e-14)
    U = misfit.superpose(G, c, s)
    w = 1.0 / (obs ** 2).sum(axis=-1)
    # d/dc_jl of sum w (U - obs)^2 = 2 sum_{k,i} w_ki sum_n (U - obs)[n] G[k,i,j,n - l s]
    n_t = obs.shape[-1]
    grad = np.zeros((3, L))
    for j in range(3):
        for l in range(L):
            sh = l * s
            grad[j, l] = sum(w[k, i] * np.dot((U - obs)[k, i, sh:], G[k, i, j, :n_t - sh])
                             for k in range(4) for i in range(3))
    scale = sum(w[k, i] * np.dot(obs[k, i], obs[k, i]) for k in range(4) for i in range(3))
    assert np.abs(grad).max() < 1e-10 * scale
    # and ERR is Eq. (2) evaluated on that reproduction
    ref = np.mean([np.sqrt(((U - obs)[k, i] ** 2).sum()) / np.sqrt((obs[k, i] ** 2).sum())
                   for k in range(4) for i in range(3)])
    assert abs(e - ref) < 1e-14


def test_pinv_matches_numpy_and_truncates():
    rng = np.random.default_rng(5)
    B = rng.standard_normal((30, 12))
    A = B.T @ B
    np.testing.assert_allclose(misfit.pinv_sym(A, 1e-14), np.linalg.pinv(A, hermitian=True), rtol=1e-8, atol=1e-12)
    # rank-deficient: directions below tau * lambda_max are discarded, like an rcond-truncated pinv
    Q, _ = np.linalg.qr(rng.standard_normal((12, 12)))
    lam = np.array([1.0] * 6 + [1e-13] * 6)
    A2 = (Q * lam) @ Q.T
    np.testing.assert_allclose(misfit.pinv_sym(A2, 1e-10), np.linalg.pinv(A2, rcond=1e-10, hermitian=True), atol=1e-9)


def test_zero_energy_pairs_are_dropped():
    rng = np.random.default_rng(6)
    obs = rng.standard_normal((3, 3, 50))
    obs[1, 2] = 0.0
    U = 1.1 * obs
    assert abs(misfit.err(U, obs) - 0.1) < 1e-14


def test_selection_rules():
    ERR = np.array([[0.30, 0.10, 0.50],
                    [0.20, 0.40, 0.20],
                    [0.20, 0.35, 0.30],
                    [0.90, 0.05, 0.05]])
    best, hist = misfit.select(ERR)
    np.testing.assert_array_equal(best, [1, 3, 3])
    # historical maxima: m0 .3 .3 .5 ; m1 .2 .4 .4 ; m2 .2 .35 .35 ; m3 .9 .9 .9
    np.testing.assert_array_equal(hist, [1, 0, 2])
