"""Batched, graph-captured stepping of uneven models (mixed precision).

Each model in a batch must produce what it produces alone (host-driven
stepping of the same algorithm), the FP64 oracle must agree, and a model
that fails must stop without disturbing the others.
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


def _cfgs(n_steps=30):
    return [configs.small_box(nx=3, ny=2, n_steps=n_steps, direction=0, seed=1),
            configs.small_box(nx=5, ny=4, counts=(3, 2), n_steps=n_steps, direction=2, seed=2),
            configs.config3_candidate(7, n_steps=n_steps, direction=1, n_lateral=6)]


def _upload(ctx, cfg, prec=1, **kw):
    m = ctx.upload(cfg["mesh"], cfg["mat"], cfg["rec_xy"])
    m.set_time(cfg["dt"], cfg["n_steps"], cfg["band"])
    m.set_input(cfg["dir"], cfg["p"])
    m.set_solver(tol=1e-8, precision=prec, inner_iters=12, **kw)
    return m


@pytest.mark.parametrize("prec", [1, 2])
def test_batch_matches_single_model_stepping_and_oracle(ctx, prec):
    cfgs = _cfgs()
    alone = []
    for cfg in cfgs:
        m = _upload(ctx, cfg, prec)
        m.step(cfg["n_steps"])
        alone.append(m.waveforms())
        m.free()
    models = [_upload(ctx, cfg, prec) for cfg in cfgs]
    b = ctx.batch(models)
    b.step(10)
    b.step(25)  # runs past the end: models stop at n_steps
    assert b.launches_per_step() > 0
    for cfg, m, w_alone in zip(cfgs, models, alone):
        st = m.stats()
        assert st["steps_done"] == cfg["n_steps"]
        assert st["relres_last"] <= 1e-8
        w = m.waveforms()
        # both runs converge every step to relative residual 1e-8; the atomic
        # accumulation order of the inner solve differs run to run
        assert _relerr(w, w_alone) <= 1e-7
        ref = newmark.analysis(cfg, tol=1e-8)["wave"]
        assert _relerr(w, ref) <= 1e-6
    b.close()
    for m in models:
        m.free()


def test_batch_failure_is_isolated(ctx):
    from paper_2404_17754_gb300 import gsw

    cfgs = _cfgs(n_steps=12)
    models = [_upload(ctx, cfg) for cfg in cfgs]
    # the second model cannot reach 1e-15 at all: its host-driven completion of
    # the first step hits the outer-iteration cap
    models[1].set_solver(tol=1e-15, precision=1, inner_iters=2, batch_outer=1, max_iter=5)
    b = ctx.batch(models)
    with pytest.raises(gsw.GswError) as e:
        b.step(12)
    assert e.value.status == gsw.E_NOCONV
    assert models[1].stats()["steps_done"] == 0
    for i in (0, 2):
        assert models[i].stats()["steps_done"] == 12
    b.close()
    for m in models:
        m.free()


def test_batch_budget_overflow_is_completed_on_host(ctx):
    """A one-iteration outer budget forces the host-driven completion of most steps."""
    cfgs = _cfgs(n_steps=10)
    alone = []
    for cfg in cfgs:
        m = _upload(ctx, cfg)
        m.step(cfg["n_steps"])
        alone.append(m.waveforms())
        m.free()
    models = [_upload(ctx, cfg, batch_outer=1) for cfg in cfgs]
    b = ctx.batch(models)
    b.step(10)
    for cfg, m, w in zip(cfgs, models, alone):
        assert m.stats()["steps_done"] == cfg["n_steps"]
        assert _relerr(m.waveforms(), w) <= 1e-7
    b.close()
    for m in models:
        m.free()


def test_run_uses_batched_path_for_mixed_models(ctx):
    from paper_2404_17754_gb300 import gsw

    cfgs = _cfgs(n_steps=15)
    models = [_upload(ctx, cfg, 2) for cfg in cfgs]
    ids = np.array([m.id for m in models], dtype=np.int32)
    ctx._check(ctx.lib.gsw_run(ctx.h, ids.ctypes.data_as(gsw._ip), len(ids), 0))
    for cfg, m in zip(cfgs, models):
        ref = newmark.analysis(cfg, tol=1e-8)["wave"]
        assert _relerr(m.waveforms(), ref) <= 1e-6
        m.free()


def test_batch_adaptive_budget(ctx):
    """batch_outer = 0 (outer iterations run in a device-side loop, or, where that
    cannot be built, in a captured budget that follows the steps): every model still
    matches its host-driven run and the oracle."""
    cfgs = _cfgs(n_steps=40)
    alone = []
    for cfg in cfgs:
        m = _upload(ctx, cfg)
        m.step(cfg["n_steps"])
        alone.append((m.waveforms(), m.stats()["cg_iters_max"]))
        m.free()
    models = [_upload(ctx, cfg, batch_outer=0) for cfg in cfgs]
    b = ctx.batch(models)
    b.step(8)
    b.step(32)
    for cfg, m, (w_alone, _) in zip(cfgs, models, alone):
        st = m.stats()
        assert st["steps_done"] == cfg["n_steps"]
        assert st["relres_last"] <= 1e-8
        assert _relerr(m.waveforms(), w_alone) <= 1e-7
        assert _relerr(m.waveforms(), newmark.analysis(cfg, tol=1e-8)["wave"]) <= 1e-6
    assert b.launches_per_step() > 0
    b.close()
    for m in models:
        m.free()


def test_batch_extrapolated_guess(ctx):
    """The increment history of the extrapolated initial guess is kept on the device, so
    batched steps (which only push a step's increment once it commits) match the same
    models stepped alone."""
    cfgs = _cfgs(n_steps=30)
    alone = []
    for cfg in cfgs:
        m = _upload(ctx, cfg, guess_order=3)
        m.step(cfg["n_steps"])
        alone.append(m.waveforms())
        m.free()
    models = [_upload(ctx, cfg, guess_order=3) for cfg in cfgs]
    b = ctx.batch(models)
    b.step(30)
    for cfg, m, w_alone in zip(cfgs, models, alone):
        assert m.stats()["steps_done"] == cfg["n_steps"]
        assert _relerr(m.waveforms(), w_alone) <= 1e-7
        assert _relerr(m.waveforms(), newmark.analysis(cfg, tol=1e-8)["wave"]) <= 1e-6
    b.close()
    for m in models:
        m.free()


def test_batch_with_fp64_outer_operator(ctx):
    """The batched graph with the outer operator in hardware FP64 (search direction and
    shifted state stored as doubles) matches the same models stepped alone and the oracle."""
    from paper_2404_17754_gb300 import gsw

    cfgs = _cfgs(n_steps=20)
    alone = []
    for cfg in cfgs:
        m = _upload(ctx, cfg, outer_op=gsw.OUTER_FP64, guess_order=2)
        m.step(cfg["n_steps"])
        alone.append(m.waveforms())
        m.free()
    models = [_upload(ctx, cfg, outer_op=gsw.OUTER_FP64, guess_order=2) for cfg in cfgs]
    b = ctx.batch(models)
    b.step(20)
    for cfg, m, w_alone in zip(cfgs, models, alone):
        assert m.stats()["steps_done"] == cfg["n_steps"]
        assert _relerr(m.waveforms(), w_alone) <= 1e-7
        assert _relerr(m.waveforms(), newmark.analysis(cfg, tol=1e-8)["wave"]) <= 1e-6
    b.close()
    for m in models:
        m.free()


@pytest.mark.parametrize("guess_order", [0, 3])
def test_fp64_batch_matches_oracle_and_host_driven_steps(ctx, guess_order):
    """Plain FP64 members (block-Jacobi PCG with every iteration in the step graph's
    device-side loop) batched with uneven sizes, together with a mixed member: the
    FP64 members agree with the oracle to 1e-9 at tolerance 1e-12 on both sides, with
    the same PCG iteration count as host-driven steps (+-1 per step)."""
    cfgs = _cfgs(n_steps=20)
    alone = []
    for cfg in cfgs:
        m = _upload(ctx, cfg, 0, guess_order=guess_order)
        m.set_solver(tol=1e-12, precision=0, guess_order=guess_order)
        m.step(cfg["n_steps"])
        alone.append((m.waveforms(), m.stats()["cg_iters_total"]))
        m.free()
    models = []
    for cfg in cfgs:
        m = _upload(ctx, cfg, 0)
        m.set_solver(tol=1e-12, precision=0, guess_order=guess_order)
        models.append(m)
    mixed = _upload(ctx, cfgs[0], 2, guess_order=guess_order)
    b = ctx.batch(models + [mixed])
    b.step(7)
    b.step(20)
    for cfg, m, (w_alone, it_alone) in zip(cfgs, models, alone):
        st = m.stats()
        assert st["steps_done"] == cfg["n_steps"] and st["relres_last"] <= 1e-12
        assert abs(st["cg_iters_total"] - it_alone) <= cfg["n_steps"]
        w = m.waveforms()
        assert _relerr(w, w_alone) <= 1e-10
        assert _relerr(w, newmark.analysis(cfg, tol=1e-12)["wave"]) <= 1e-9
    assert mixed.stats()["steps_done"] == cfgs[0]["n_steps"]
    assert _relerr(mixed.waveforms(), newmark.analysis(cfgs[0], tol=1e-8)["wave"]) <= 1e-6
    b.close()
    for m in models + [mixed]:
        m.free()


def test_fp64_batch_budget_overflow_finishes_on_the_host(ctx):
    """A device-side loop budget smaller than the PCG needs: every step is handed to the
    host-driven solver and the result is unchanged."""
    cfg = _cfgs(n_steps=8)[1]
    m = _upload(ctx, cfg, 0)
    m.set_solver(tol=1e-12, precision=0, batch_outer=3)
    b = ctx.batch([m])
    b.step(cfg["n_steps"])
    assert m.stats()["steps_done"] == cfg["n_steps"]
    assert _relerr(m.waveforms(), newmark.analysis(cfg, tol=1e-12)["wave"]) <= 1e-9
    b.close()
    m.free()
