"""The C ABI's analysis-level entry points against the oracle and each other.

* gsw_run with a direction mask: one uploaded model serves its three
  input-direction analyses (shared mesh and element data, own state); each
  matches the oracle and a separately uploaded single-direction model.
* gsw_checkpoint / gsw_restore: a run resumed from a checkpoint continues
  exactly as the uninterrupted run, including the extrapolated guess's
  increment history and the learned guess's network and optimiser state.
* gsw_mlp_train: training on the next steps, then the learned guess applies.
* Failures injected on the host: a non-finite state is rejected at the
  boundary; a network whose output overflows falls back to the predictor.
"""
import numpy as np
import pytest

from oracle import newmark
from synth import configs

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


def _relerr(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _upload(ctx, cfg, n_steps=None):
    m = ctx.upload(cfg["mesh"], cfg["mat"], cfg["rec_xy"])
    m.set_time(cfg["dt"], n_steps or cfg["n_steps"], cfg["band"])
    return m


@pytest.mark.parametrize("prec", [0, 2])
def test_direction_mask_runs_three_analyses_of_one_model(ctx, prec):
    from paper_2404_17754_gb300 import gsw

    cfg = configs.small_box(nx=4, ny=3, n_steps=25, seed=4)
    tol = 1e-12 if prec == 0 else 1e-8
    m = _upload(ctx, cfg)
    m.set_solver(tol=tol, precision=prec, inner_iters=12, guess_order=2)
    with pytest.raises(gsw.GswError) as ei:
        m.run(dirs_mask=7)  # no inputs yet
    assert ei.value.status == gsw.E_STATE
    for j in range(3):
        m.set_input(j, cfg["p"] * (1.0 + 0.5 * j))
    with pytest.raises(gsw.GswError):
        m.waveforms(1)  # not run yet
    m.run(dirs_mask=7)
    for j in range(3):
        w = m.waveforms(j)
        ref = newmark.analysis(dict(cfg, p=cfg["p"] * (1.0 + 0.5 * j), dir=j), tol=tol)["wave"]
        assert _relerr(w, ref) <= (1e-9 if prec == 0 else 1e-6), j
        assert m.stats(j)["steps_done"] == cfg["n_steps"] and m.stats(j)["relres_last"] <= tol
        # the same analysis on a model of its own
        s = _upload(ctx, cfg)
        s.set_input(j, cfg["p"] * (1.0 + 0.5 * j))
        s.set_solver(tol=tol, precision=prec, inner_iters=12, guess_order=2)
        s.run()
        assert _relerr(s.waveforms(), w) <= (1e-11 if prec == 0 else 1e-7)
        s.free()
    # a subset of the directions, again (instances are reused and reset)
    m.run(dirs_mask=2)
    assert _relerr(m.waveforms(1), newmark.analysis(dict(cfg, p=1.5 * cfg["p"], dir=1), tol=tol)["wave"]) <= (
        1e-9 if prec == 0 else 1e-6)
    m.free()


def test_checkpoint_restore_resumes_extrapolated_guess_exactly(ctx):
    cfg = configs.small_box(nx=4, ny=3, n_steps=30, seed=5)
    m = _upload(ctx, cfg)
    m.set_input(cfg["dir"], cfg["p"])
    m.set_solver(tol=1e-12, precision=0, guess_order=4)
    m.step(12)
    ck = m.checkpoint()
    m.step(10)
    w_ref, s_ref = m.waveforms(), m.stats()
    m.reset()  # lose the state and the increment history
    m.step(3)
    m.restore(ck)
    assert m.stats()["steps_done"] == 12
    m.step(10)
    s = m.stats()
    # the quartic guess resumed with its history (the FP64 scatter's atomics may move a step's
    # count by one between otherwise equal runs; a lost history costs many more)
    assert abs(s["cg_iters_total"] - s_ref["cg_iters_total"]) <= 2
    assert _relerr(m.waveforms(), w_ref) <= 1e-11
    # a checkpoint of another set-up is refused and leaves the model as it was
    m2 = _upload(ctx, configs.small_box(nx=3, ny=2, n_steps=30))
    m2.set_input(0, cfg["p"])
    m2.set_solver(tol=1e-12, precision=0, guess_order=4)
    from paper_2404_17754_gb300 import gsw

    with pytest.raises(gsw.GswError) as ei:
        m2.restore(ck)
    assert ei.value.status == gsw.E_INVALID
    m2.free()
    m.free()


def test_checkpoint_restore_keeps_the_learned_guess(ctx):
    cfg = configs.small_box(nx=4, ny=3, n_steps=40, seed=6)
    m = _upload(ctx, cfg)
    m.set_input(cfg["dir"], cfg["p"])
    m.set_solver(tol=1e-8, precision=1, inner_iters=12)
    m.mlp_train(12, batch=512, iters_per_step=3, lr=1e-3, seed=3)
    m.step(4)
    ck = m.checkpoint()
    th = m.mlp_params()
    st = m.mlp_state()
    m.step(8)
    w_ref = m.waveforms()
    m.mlp_train(6, batch=512, iters_per_step=3, lr=1e-3, seed=3)  # changes the network
    assert np.abs(m.mlp_params() - th).max() > 0
    m.restore(ck)
    assert np.array_equal(m.mlp_params(), th)
    st2 = m.mlp_state()
    assert st2["learned_steps"] == st["learned_steps"] and st2["active"] == st["active"]
    m.step(8)
    assert _relerr(m.waveforms(), w_ref) <= 1e-7
    m.free()


def test_mlp_train_then_apply(ctx):
    from paper_2404_17754_gb300 import gsw

    cfg = configs.config1(n_steps=80)
    m = _upload(ctx, cfg)
    m.set_input(cfg["dir"], cfg["p"])
    m.set_solver(tol=1e-8, precision=1, inner_iters=15)
    with pytest.raises(gsw.GswError) as ei:
        m.mlp_train(200)
    assert ei.value.status == gsw.E_INVALID
    m.mlp_train(40, batch=4096, iters_per_step=4, lr=2e-3, seed=5)
    assert m.stats()["steps_done"] == 40 and m.mlp_loss() > 0
    m.step(40)
    assert m.mlp_state()["learned_steps"] >= 5
    assert m.stats()["relres_last"] <= 1e-8
    ref = newmark.analysis(cfg, tol=1e-8)["wave"]
    assert _relerr(m.waveforms(), ref) <= 1e-6
    m.free()


def test_host_injected_failures(ctx):
    from paper_2404_17754_gb300 import gsw

    cfg = configs.small_box(nx=3, ny=2, n_steps=30, seed=8)
    m = _upload(ctx, cfg)
    m.set_input(cfg["dir"], cfg["p"])
    m.set_solver(tol=1e-8, precision=1, inner_iters=12)
    m.step(2)
    u, v, a, k = m.get_state()
    u[3, 1] = np.nan
    with pytest.raises(gsw.GswError) as ei:
        m.set_state(u, v, a, k)
    assert ei.value.status == gsw.E_INVALID
    m.step(2)  # the model is untouched and keeps stepping
    # a network whose output overflows to infinity: every guess falls back to the predictor
    m.reset()
    m.mlp_train(8, batch=256, iters_per_step=1, lr=1e-3, seed=1)
    m.mlp_params(np.full(5443, 1e30))
    m.step(10)
    assert m.stats()["relres_last"] <= 1e-8
    ref = newmark.analysis(cfg, tol=1e-8, n_steps=18)["wave"]
    assert _relerr(m.waveforms()[:, :, :18], ref) <= 1e-6
    m.free()


def test_bounded_wait_runs_out_and_the_context_stays_usable(ctx):
    """The bounded mbarrier wait that guards the warp-specialised inner operator's stages, on a
    barrier that nothing completes: it runs out and reports GSW_E_TIMEOUT (not a hang, not a
    fault); afterwards the same context solves on the warp-specialised variant as before, and
    limits outside 1 .. 2^22 are rejected."""
    from paper_2404_17754_gb300 import gsw

    for limit in (1, 1000):
        assert ctx.wait_probe(limit) == gsw.E_TIMEOUT
    assert ctx.wait_probe(0) == gsw.E_INVALID
    assert ctx.wait_probe((1 << 22) + 1) == gsw.E_INVALID
    cfg = configs.small_box(nx=3, ny=2, n_steps=12, seed=8)
    m = _upload(ctx, cfg)
    m.set_input(cfg["dir"], cfg["p"])
    m.set_solver(tol=1e-8, precision=2, inner_iters=12, inner_variant=3)
    m.step(12)
    assert m.stats()["relres_last"] <= 1e-8
    ref = newmark.analysis(cfg, tol=1e-8)["wave"]
    assert _relerr(m.waveforms(), ref) <= 1e-6
    m.free()


@pytest.mark.parametrize("prec", [1, 2])
def test_direction_analyses_in_lockstep_share_the_operator(ctx, prec):
    """share_dirs = 1: the three direction analyses of one model advance in lockstep and
    apply the inner operator to their three search directions in one pass; each matches
    the same analysis run on its own (both at relative residual 1e-8) and the oracle."""
    cfg = configs.config3_candidate(3, n_steps=30, n_lateral=6)
    scales = (1.0, -0.7, 1.3)
    out = {}
    for share in (0, 1):
        m = _upload(ctx, cfg)
        m.set_solver(tol=1e-8, precision=prec, inner_iters=12, guess_order=2, share_dirs=share)
        for j in range(3):
            m.set_input(j, scales[j] * cfg["p"])
        m.run(dirs_mask=7)
        out[share] = [m.waveforms(j) for j in range(3)]
        for j in range(3):
            st = m.stats(j)
            assert st["steps_done"] == cfg["n_steps"] and st["relres_last"] <= 1e-8
        m.free()
    for j in range(3):
        ref = newmark.analysis(dict(cfg, p=scales[j] * cfg["p"], dir=j), tol=1e-8)["wave"]
        assert _relerr(out[1][j], ref) <= 1e-6, j
        assert _relerr(out[1][j], out[0][j]) <= 1e-7, j


@pytest.mark.parametrize("prec", [0, 2])
def test_projection_guess_converges_to_the_oracle_on_every_path(ctx, prec):
    """proj_dim = 6: the initial guess is the Galerkin projection onto the last six
    increments.  Host-driven steps, batched steps and direction analyses in lockstep all
    reach the oracle's solution (1e-9 at tolerance 1e-12 in FP64, 1e-6 at 1e-8 mixed)."""
    cfg = configs.small_box(nx=4, ny=3, n_steps=30, seed=9)
    tol = 1e-12 if prec == 0 else 1e-8
    bar = 1e-9 if prec == 0 else 1e-6
    ref = newmark.analysis(cfg, tol=tol)["wave"]
    m = _upload(ctx, cfg)
    m.set_input(cfg["dir"], cfg["p"])
    m.set_solver(tol=tol, precision=prec, inner_iters=12, proj_dim=6)
    m.step(cfg["n_steps"])
    assert m.stats()["relres_last"] <= tol
    assert _relerr(m.waveforms(), ref) <= bar
    m.run()  # batched (device-driven) steps
    assert _relerr(m.waveforms(), ref) <= bar
    if prec != 0:
        m.set_solver(tol=tol, precision=prec, inner_iters=12, proj_dim=6, share_dirs=1)
        for j in range(3):
            m.set_input(j, cfg["p"])
        m.run(dirs_mask=7)
        assert _relerr(m.waveforms(cfg["dir"]), ref) <= bar
        for j in range(3):
            assert _relerr(m.waveforms(j), newmark.analysis(dict(cfg, dir=j), tol=tol)["wave"]) <= bar
    m.free()


def test_projection_hands_over_to_the_extrapolation(ctx):
    """proj_relres: the projection guess acts until a step starts from an initial relative
    residual below the threshold, then the quartic extrapolation takes over for good (its ring
    is filled all along).  A threshold that the first projected step already meets gives the
    quartic run; the handover survives a checkpoint; host-driven and device-driven mixed steps
    with a mid-run handover reach the oracle; inconsistent options are rejected."""
    from paper_2404_17754_gb300 import gsw

    cfg = configs.small_box(nx=4, ny=3, n_steps=40, seed=5)
    runs = {}
    for name, kw in (("quartic", dict(guess_order=4)),
                     ("handover", dict(guess_order=4, proj_dim=6, proj_relres=0.999))):
        m = _upload(ctx, cfg)
        m.set_input(cfg["dir"], cfg["p"])
        m.set_solver(tol=1e-12, precision=0, **kw)
        m.step(2)  # step 1 differs: the projection onto one increment against the predictor
        it2 = m.stats()["cg_iters_total"]
        m.step(cfg["n_steps"] - 2)
        runs[name] = (m.waveforms(), m.stats()["cg_iters_total"] - it2)
        if name == "handover":
            # checkpoint after the handover, resume after a reset: same iterations and waveforms
            m.reset()
            m.step(20)
            ck = m.checkpoint()
            m.step(10)
            w_ref, it_ref = m.waveforms(), m.stats()["cg_iters_total"]
            m.reset()
            m.step(3)
            m.restore(ck)
            m.step(10)
            assert abs(m.stats()["cg_iters_total"] - it_ref) <= 2
            assert _relerr(m.waveforms(), w_ref) <= 1e-11
        m.free()
    assert _relerr(runs["handover"][0], runs["quartic"][0]) <= 1e-9
    # after the handover both runs use the same guesses (solutions equal to ~1e-12, so a
    # step's count may differ by one now and then)
    assert abs(runs["handover"][1] - runs["quartic"][1]) <= 3
    # a handover in the middle of the run, mixed precision, host- and device-driven
    cfg = configs.config1(n_steps=60)
    ref = newmark.analysis(cfg, tol=1e-8)["wave"]
    m = _upload(ctx, cfg)
    m.set_input(cfg["dir"], cfg["p"])
    m.set_solver(tol=1e-8, precision=2, inner_iters=20, guess_order=4, proj_dim=8, proj_relres=1e-3)
    m.step(60)
    assert m.stats()["relres_last"] <= 1e-8
    assert _relerr(m.waveforms(), ref) <= 1e-6
    m.run()
    assert _relerr(m.waveforms(), ref) <= 1e-6
    for bad in (dict(proj_dim=0, guess_order=4, proj_relres=1e-3), dict(proj_dim=8, guess_order=0, proj_relres=1e-3),
                dict(proj_dim=8, guess_order=4, proj_relres=1.0)):
        with pytest.raises(gsw.GswError) as ei:
            m.set_solver(tol=1e-8, precision=2, inner_iters=20, **bad)
        assert ei.value.status == gsw.E_INVALID
    m.free()


def test_projection_guess_checkpoint_and_quality(ctx):
    from paper_2404_17754_gb300 import gsw

    cfg = configs.small_box(nx=4, ny=3, n_steps=40, seed=5)
    m = _upload(ctx, cfg)
    m.set_input(cfg["dir"], cfg["p"])
    m.set_solver(tol=1e-12, precision=0, proj_dim=6)
    m.step(15)
    ck = m.checkpoint()
    m.step(10)
    w_ref, s_ref = m.waveforms(), m.stats()
    m.reset()
    m.step(2)
    m.restore(ck)
    m.step(10)
    # the projection history resumed (a lost history costs tens of iterations; the FP64
    # scatter's atomics make a step's count vary by one between otherwise equal runs)
    assert abs(m.stats()["cg_iters_total"] - s_ref["cg_iters_total"]) <= 2
    assert _relerr(m.waveforms(), w_ref) <= 1e-11
    with pytest.raises(gsw.GswError) as ei:
        m.set_learning(True, train_steps=10, batch=256)
    assert ei.value.status == gsw.E_STATE
    m.free()
    # its initial residual against the quartic extrapolation's (host-driven mixed steps)
    cfg = configs.config1(n_steps=80)
    r0 = {}
    for name, kw in (("quartic", dict(guess_order=4)), ("projection", dict(proj_dim=8))):
        m = _upload(ctx, cfg)
        m.set_input(cfg["dir"], cfg["p"])
        m.set_solver(tol=1e-8, precision=2, inner_iters=20, **kw)
        m.step(20)
        a = m.stats()["init_relres_sum"]
        m.step(60)
        r0[name] = (m.stats()["init_relres_sum"] - a) / 60
        assert _relerr(m.waveforms(), newmark.analysis(cfg, tol=1e-8)["wave"]) <= 1e-6
        m.free()
    print("mean initial relative residual, steps 21-80: quartic %.3e, projection onto 8 increments %.3e"
          % (r0["quartic"], r0["projection"]))
    assert r0["projection"] <= 1.1 * r0["quartic"]


def test_json_run_configuration_end_to_end(ctx, tmp_path):
    """A per-run JSON configuration (two input directions of the small box, FP64 at 1e-12) runs
    through the C ABI, matches the oracle per direction, and its outputs carry the resolved
    configuration."""
    import json

    from paper_2404_17754_gb300 import runconfig

    path = tmp_path / "run.json"
    path.write_text(json.dumps({
        "workload": {"kind": "small-box", "directions": [0, 2]},
        "time": {"n_steps": 15},
        "solver": {"tol": 1e-12, "precision": "fp64", "guess_order": 0},
        "output": {"waveforms": str(tmp_path / "w.npy"), "summary": str(tmp_path / "s.json")}}))
    waves, summary = runconfig.run(str(path), ctx=ctx)
    cfg = configs.small_box(n_steps=15)
    for d in (0, 2):
        ref = newmark.analysis(dict(cfg, dir=d), tol=1e-12)["wave"]
        assert _relerr(waves[d], ref) <= 1e-9, d
        assert summary["stats"][str(d)]["relres_last"] <= 1e-12
    saved = json.loads((tmp_path / "s.json").read_text())
    assert saved["config"]["workload"]["directions"] == [0, 2] and saved["config"]["solver"]["tol"] == 1e-12
    assert np.load(tmp_path / "w.npy").shape == (2,) + waves[0].shape
