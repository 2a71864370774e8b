"""Candidate pool from survey points (Section 3): IDW, Laplace smoothing, selection."""
import numpy as np

from synth import candidates as cd


def _pts():
    return cd.survey_points(n=40, L=600.0, seed=3)


def test_idw_exact_at_survey_points_and_convex():
    P, z = _pts()
    for M, q in [(1, 0.5), (7, 2.0), (40, 4.0)]:
        est = cd.idw(P, z, P[:, 0], P[:, 1], M, q)
        np.testing.assert_array_equal(est, z)  # d = 0 returns the point's own value
    rng = np.random.default_rng(1)
    X = rng.uniform(0, 600, 200)
    Y = rng.uniform(0, 600, 200)
    for M in (1, 5, 20):
        est = cd.idw(P, z, X, Y, M, 2.0)
        d = np.hypot(X[:, None] - P[None, :, 0], Y[:, None] - P[None, :, 1])
        near = np.argsort(d, axis=1, kind="stable")[:, :M]
        lo, hi = z[near].min(axis=1), z[near].max(axis=1)
        assert np.all(est >= lo - 1e-12) and np.all(est <= hi + 1e-12)  # convex combination of the M nearest
        if M == 1:
            np.testing.assert_allclose(est, z[near[:, 0]], rtol=1e-15)  # nearest-neighbour value


def test_idw_constant_and_sharp_limit():
    P, z = _pts()
    X, Y = np.meshgrid(np.linspace(0, 600, 13), np.linspace(0, 600, 13), indexing="ij")
    np.testing.assert_allclose(cd.idw(P, np.full(len(z), 17.5), X, Y, 12, 1.3), 17.5, rtol=1e-14)
    # q -> infinity: the nearest point's weight dominates wherever the second
    # nearest is clearly farther ((1/1.2)^200 ~ 1e-16)
    d = np.sort(np.hypot(X.ravel()[:, None] - P[None, :, 0], Y.ravel()[:, None] - P[None, :, 1]), axis=1)
    clear = (d[:, 1] > 1.2 * d[:, 0]).reshape(X.shape)
    assert clear.sum() > 50
    np.testing.assert_allclose(cd.idw(P, z, X, Y, 10, 200.0)[clear], cd.idw(P, z, X, Y, 1, 1.0)[clear], rtol=1e-12)
    # q -> 0 over all points: the plain mean
    np.testing.assert_allclose(cd.idw(P, z, X, Y, len(z), 1e-12), z.mean(), rtol=1e-9)


def test_laplace_smoothing_invariants():
    n = 20
    I, J = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    np.testing.assert_allclose(cd.laplace_smooth(np.full((n, n), 3.0), 5), 3.0, rtol=1e-15)
    lin = 2.0 * I - 0.5 * J + 1.0
    once = cd.laplace_smooth(lin, 1)
    np.testing.assert_allclose(once[1:-1, 1:-1], lin[1:-1, 1:-1], rtol=1e-14)  # mean of 4 neighbours
    rough = np.random.default_rng(2).standard_normal((n, n))
    sm = cd.laplace_smooth(rough, 5)
    assert np.abs(np.diff(sm, axis=0)).max() < np.abs(np.diff(rough, axis=0)).max()
    assert sm.max() <= rough.max() and sm.min() >= rough.min()  # averaging never leaves the data range


def test_pool_and_selection():
    P, z = _pts()
    assert len(cd.M_VALUES) * len(cd.Q_VALUES) == 2000
    assert cd.Q_VALUES[0] == 0.1 and cd.Q_VALUES[-1] == 4.0
    sub = [((M, q), cd.boundary(P, z, 8, 600.0, M, q)) for M in (1, 5, 20, 40) for q in (0.5, 2.0, 4.0)]
    ref = cd.boundary(P, z, 8, 600.0, 20, 2.0)
    keep, rms = cd.select_varied(sub, ref, 5)
    assert len(set(keep.tolist())) == 5
    assert np.all(np.diff(rms[keep]) <= 0)
    i_ref = [k for k, (mq, _) in enumerate(sub) if mq == (20, 2.0)][0]
    assert rms[i_ref] == 0.0 and i_ref not in keep


def test_candidate_config_builds_a_layered_mesh():
    P, z = _pts()
    cfg = cd.candidate_config(P, z, 20, 2.0, n=6, n_steps=10)
    mesh = cfg["mesh"]
    assert mesh["conn"].shape == (6 * 6 * 6 * 8, 10)
    assert set(np.unique(mesh["elem_mat"])) == {0, 1}
    assert cfg["rec_xy"].shape == (25, 2)
