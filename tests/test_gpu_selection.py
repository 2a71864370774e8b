"""End-to-end model selection on the GPU (Section 2 method, Section 3 workflow).

Candidates are seeded interface realisations of the two-layer box; one of
them is the hidden truth.  Each candidate is uploaded once; its Green's
functions (unit sin^2 pulse in x1, x2, x3; Section 3: three analyses per
model) are its three input-direction analyses, run for all candidates as one
GPU batch (gsw_run with dirs_mask 7).  Observations of three events are the
truth's responses to seeded input-coefficient sets, and the GPU misfit by
model id (device-resident Green's functions) estimates each candidate's input
and ERR (Eq. (2)).  The truth must reproduce the observations and be
selected, per event and by the historical maximum.
"""
import numpy as np
import pytest

from oracle import misfit, newmark
from synth import configs
from synth.waves import sin2_pulse

pytestmark = pytest.mark.gpu


def test_truth_is_selected_from_candidates():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_17754_gb300 import build, gsw

    build.build()
    ctx = gsw.Context(0)
    n_steps, s, L = 90, 10, 5
    seeds = [11, 12, 13, 14]
    truth = 2
    cfgs = [configs.config3_candidate(l, n_steps=n_steps, n_lateral=6) for l in seeds]
    t = cfgs[0]["dt"] * np.arange(1, n_steps + 1)
    pulse = sin2_pulse(t, 2 * s * cfgs[0]["dt"])
    models = []
    for cfg in cfgs:
        m = ctx.upload(cfg["mesh"], cfg["mat"], cfg["rec_xy"])
        m.set_time(cfg["dt"], n_steps, cfg["band"])
        m.set_solver(tol=1e-10, precision=1, inner_iters=15, batch_outer=12)
        for j in range(3):
            m.set_input(j, pulse)
        models.append(m)
    ctx.run(models, dirs_mask=7)
    G = [np.stack([m.waveforms(j) for j in range(3)], axis=2) for m in models]  # [rec, i, j, t]
    # one candidate's Green's functions against the oracle
    for j in range(3):
        ref = newmark.analysis(dict(cfgs[truth], p=pulse, dir=j), tol=1e-10)["wave"]
        assert np.linalg.norm(G[truth][:, :, j] - ref) <= 1e-6 * np.linalg.norm(ref)
    rng = np.random.default_rng(8)
    ERR = np.zeros((len(cfgs), 3))
    for e in range(3):
        c_true = rng.standard_normal((3, L)) * np.hanning(L + 2)[1:-1]
        obs = misfit.superpose(G[truth], c_true, s)
        for c, m in enumerate(models):
            err, c_est = m.misfit(obs, s, L, tau=1e-10)
            ERR[c, e] = err
            err_o, _ = misfit.estimate(G[c], obs, s, L, tau=1e-10)
            assert abs(err - err_o) <= 1e-9 * max(err_o, 1e-3)  # an exact fit leaves rounding noise (~1e-15)
            err_g, _ = ctx.misfit_green(G[c], obs, s, L, tau=1e-10)
            assert abs(err - err_g) <= 1e-12 * max(err_g, 1e-3)
            if c == truth:
                np.testing.assert_allclose(c_est, c_true, atol=1e-6 * np.abs(c_true).max())
    best, hist = misfit.select(ERR)
    assert ERR[truth].max() < 1e-6
    assert np.all(best == truth) and np.all(hist == truth)
    others = np.delete(ERR, truth, axis=0)
    assert others.min() > 100 * ERR[truth].max()
    # the misfit needs all three directions run since the last set-up
    models[0].set_input(1, 2.0 * pulse)
    with pytest.raises(gsw.GswError) as ei:
        models[0].misfit(obs, s, L)
    assert ei.value.status == gsw.E_STATE
    for m in models:
        m.free()
    ctx.close()
