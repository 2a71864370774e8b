"""Synthetic versions of the paper's experiments on the GPU (Section 3).

* Observation layouts: ERR per event from 1, 9 and 25 observation points
  (subsets of a 5 x 5 receiver grid), for two events inside the span of the
  shifted pulses and one random-phase event outside it; per-event and
  historical-maximum selection identical to the oracle's, the truth
  selected in every layout, and the input-wave recovery reported.
* Candidates from the paper's pool mechanics: IDW boundaries over seeded
  survey points (synth.candidates), the members farthest from the M = 20,
  q = 2.0 reference; the hidden member is selected by the GPU misfit.

Green's functions are the candidates' three input-direction analyses run as
one GPU batch (gsw_run with dirs_mask 7); ERR parity is against the oracle's
misfit on the same Green's functions.
"""
import numpy as np
import pytest

from oracle import misfit, newmark
from synth import candidates, configs
from synth.waves import random_phase, sin2_pulse

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_17754_gb300 import build, gsw

    build.build()
    c = gsw.Context(0)
    yield c
    c.close()


def _green(ctx, cfgs, pulse, n_steps):
    models = []
    for cfg in cfgs:
        m = ctx.upload(cfg["mesh"], cfg["mat"], cfg["rec_xy"])
        m.set_time(cfg["dt"], n_steps, cfg["band"])
        m.set_solver(tol=1e-10, precision=1, inner_iters=15, batch_outer=12)
        for j in range(3):
            m.set_input(j, pulse)
        models.append(m)
    ctx.run(models, dirs_mask=7)
    return models, [np.stack([m.waveforms(j) for j in range(3)], axis=2) for m in models]


def test_observation_layouts_and_out_of_span_event(ctx):
    n_steps, s, L = 120, 10, 11
    seeds, truth = [21, 22, 23, 24, 25], 1
    cfgs = [configs.config3_candidate(l, n_steps=n_steps, n_lateral=6) for l in seeds]
    dt = cfgs[0]["dt"]
    t = dt * np.arange(1, n_steps + 1)
    pulse = sin2_pulse(t, 2 * s * dt)
    models, G = _green(ctx, cfgs, pulse, n_steps)
    rng = np.random.default_rng(31)
    events = [misfit.superpose(G[truth], rng.standard_normal((3, L)) * np.hanning(L + 2)[1:-1], s) for _ in range(2)]
    # an event outside the span: the truth driven by a random-phase input in x1
    rp = random_phase(n_steps, dt, np.random.default_rng(77), t_window=1.0)
    mt = ctx.upload(cfgs[truth]["mesh"], cfgs[truth]["mat"], cfgs[truth]["rec_xy"])
    mt.set_time(dt, n_steps, cfgs[truth]["band"])
    mt.set_input(0, rp)
    mt.set_solver(tol=1e-10, precision=1, inner_iters=15)
    mt.run()
    events.append(mt.waveforms())
    mt.free()
    layouts = {1: [12], 9: [6, 7, 8, 11, 12, 13, 16, 17, 18], 25: list(range(25))}
    for name, rec in layouts.items():
        ERR = np.zeros((len(cfgs), len(events)))
        ERR_o = np.zeros_like(ERR)
        for e, obs in enumerate(events):
            for c in range(len(cfgs)):
                if name == 25:
                    err, c_est = models[c].misfit(obs, s, L, tau=1e-10)
                else:
                    err, c_est = ctx.misfit_green(G[c][rec], obs[rec], s, L, tau=1e-10)
                ERR[c, e] = err
                ERR_o[c, e] = misfit.estimate(G[c][rec], obs[rec], s, L, tau=1e-10)[0]
                assert abs(err - ERR_o[c, e]) <= 1e-9 * max(ERR_o[c, e], 1e-3)
                if e == 2 and c == truth:
                    est = sum(c_est[0, l] * sin2_pulse(t - l * s * dt, 2 * s * dt) for l in range(L))
                    recovery = np.linalg.norm(est - rp) / np.linalg.norm(rp)
        best, hist = misfit.select(ERR)
        best_o, hist_o = misfit.select(ERR_o)
        assert np.array_equal(best, best_o) and np.array_equal(hist, hist_o)
        assert np.all(best == truth) and np.all(hist == truth)
        assert ERR[truth, :2].max() < 1e-6
        margin = np.sort(ERR[:, 2])[1] - ERR[truth, 2]
        print("layout %2d points: out-of-span ERR truth %.4f, margin %.4f, input recovery (rel L2) %.3f"
              % (name, ERR[truth, 2], margin, recovery))
        assert margin > 1e-4
    for m in models:
        m.free()


def test_idw_pool_candidates_select_the_truth(ctx):
    n_steps, s, L, n = 90, 10, 5, 8
    pts, vals = candidates.survey_points(seed=0)
    members = candidates.pool(pts, vals, n, 600.0)
    ref = [b for (Mq, b) in members if Mq == (20, 2.0)][0]
    keep, _ = candidates.select_varied(members, ref, 4)
    picks = [members[i][0] for i in keep]
    cfgs = [candidates.candidate_config(pts, vals, M, q, n=n, n_steps=n_steps) for (M, q) in picks]
    truth = 2
    dt = cfgs[0]["dt"]
    pulse = sin2_pulse(dt * np.arange(1, n_steps + 1), 2 * s * dt)
    models, G = _green(ctx, cfgs, pulse, n_steps)
    ref_w = newmark.analysis(dict(cfgs[truth], p=pulse, dir=2), tol=1e-10)["wave"]
    assert np.linalg.norm(G[truth][:, :, 2] - ref_w) <= 1e-6 * np.linalg.norm(ref_w)
    rng = np.random.default_rng(5)
    ERR = np.zeros((len(cfgs), 2))
    for e in range(2):
        obs = misfit.superpose(G[truth], rng.standard_normal((3, L)) * np.hanning(L + 2)[1:-1], s)
        for c, m in enumerate(models):
            ERR[c, e] = m.misfit(obs, s, L, tau=1e-10)[0]
            err_o = misfit.estimate(G[c], obs, s, L, tau=1e-10)[0]
            assert abs(ERR[c, e] - err_o) <= 1e-9 * max(err_o, 1e-3)
    best, hist = misfit.select(ERR)
    assert np.all(best == truth) and np.all(hist == truth)
    assert ERR[truth].max() < 1e-6
    print("IDW members %s: ERR %s" % (picks, np.round(ERR, 5).tolist()))
    for m in models:
        m.free()
