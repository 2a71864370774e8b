"""Two-level inner preconditioner (first-order vertex coarse level) on the GPU vs the oracle.

* the coarse correction P D_c^-1 P^T x (restriction gather, coarse blocks of
  P^T A P, prolongation) against ``oracle.twolevel`` on meshes of one and of
  many CTAs with a ragged node count;
* mixed solves with the two-level preconditioner reach the oracle's
  waveforms (host-driven steps, the device-driven run, and the three input
  directions in lockstep) and at tight tolerance the oracle's states;
* on the realistic model's lateral crop it needs fewer inner iterations than
  the block-Jacobi inner preconditioner, with the same waveforms.
"""
import numpy as np
import pytest

from oracle import fem, newmark, twolevel
from synth import configs

pytestmark = pytest.mark.gpu

PREC = {"fp32": 1, "fp16": 2}


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


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
@pytest.mark.parametrize("nx,ny", [(3, 2), (14, 9)])
def test_coarse_correction_matches_oracle(ctx, prec, nx, ny):
    import torch

    cfg = configs.small_box(nx=nx, ny=ny, counts=(3, 2), distort=True)
    mesh = cfg["mesh"]
    ops = fem.assemble(mesh, cfg["mat"], cfg["band"])
    dt = cfg["dt"]
    A = (ops["K"] + (2 / dt) * (ops["CR"] + ops["Cabs"]) + (4 / dt ** 2) * ops["M"]).tocsr()
    P, verts = twolevel.prolongation(mesh["conn"], mesh["xyz"].shape[0])
    Dc_inv = twolevel.coarse_inverse_blocks(A, P)
    m = ctx.upload(mesh, cfg["mat"], cfg["rec_xy"])
    m.set_time(dt, 4, cfg["band"])
    m.set_solver(tol=1e-8, precision=PREC[prec], inner_iters=4, coarse_weight=0.7)
    assert m.n_nodes % 4 != 0  # a ragged last node quad
    x = np.random.default_rng(3).standard_normal(3 * m.n_nodes)
    y = m.apply(6, torch.tensor(x, device="cuda")).cpu().numpy()
    ref = twolevel.coarse_correction(P, Dc_inv, x)
    assert _relerr(y, ref) <= 2e-6
    m.free()


def test_coarse_correction_needs_the_option(ctx):
    import torch

    from paper_2404_17754_gb300 import gsw

    cfg = configs.small_box()
    m = ctx.upload(cfg["mesh"], cfg["mat"], cfg["rec_xy"])
    m.set_time(cfg["dt"], 4, cfg["band"])
    m.set_solver(tol=1e-8, precision=1, inner_iters=4)
    x = torch.zeros(3 * m.n_nodes, dtype=torch.float64, device="cuda")
    with pytest.raises(gsw.GswError):
        m.apply(6, x)
    with pytest.raises(gsw.GswError):
        m.set_solver(tol=1e-8, precision=1, inner_iters=4, coarse_weight=-0.5)
    with pytest.raises(gsw.GswError):
        m.set_solver(tol=1e-8, precision=1, inner_iters=4, coarse_weight=float("nan"))
    m.free()


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
@pytest.mark.parametrize("drive", ["step", "run"])
def test_two_level_mixed_matches_oracle(ctx, prec, drive):
    cfg = configs.config1(n_steps=40)
    ref = newmark.analysis(cfg, tol=1e-8)
    m = ctx.upload(cfg["mesh"], cfg["mat"], cfg["rec_xy"])
    m.set_time(cfg["dt"], 40, cfg["band"])
    m.set_input(cfg["dir"], cfg["p"])
    m.set_solver(tol=1e-8, precision=PREC[prec], inner_iters=30, inner_rtol=1e-2, coarse_weight=0.7)
    if drive == "step":
        m.step(40)
    else:
        m.run()
    st = m.stats()
    assert _relerr(m.waveforms(), ref["wave"]) <= 1e-6
    assert st["relres_last"] <= 1e-8
    m.free()


@pytest.mark.parametrize("drive", ["step", "run"])
def test_two_level_switches_off_below_the_threshold(ctx, drive):
    """coarse_relres = 1e-4: the inner solves of the first steps from rest (large outer
    residuals) apply the coarse correction, later ones run on the fine level alone (the
    restriction kernel only passes the scalars on); the run matches the oracle throughout."""
    cfg = configs.config1(n_steps=60)
    ref = newmark.analysis(cfg, tol=1e-8)
    m = ctx.upload(cfg["mesh"], cfg["mat"], cfg["rec_xy"])
    m.set_time(cfg["dt"], 60, cfg["band"])
    m.set_input(cfg["dir"], cfg["p"])
    m.set_solver(tol=1e-8, precision=2, inner_iters=30, inner_rtol=1e-2, guess_order=4, coarse_weight=0.7,
                 coarse_relres=1e-4)
    if drive == "step":
        m.step(60)
    else:
        m.run()
    assert _relerr(m.waveforms(), ref["wave"]) <= 1e-6
    assert m.stats()["relres_last"] <= 1e-8
    m.free()


def test_two_level_tight_tolerance_ragged_box(ctx):
    """tol 1e-12 on a box whose node count is not a multiple of four: the states match the
    oracle to 1e-9 (the recurrence's ragged tail and the coarse level's edges included)."""
    from paper_2404_17754_gb300 import gsw

    cfg = configs.small_box(nx=4, ny=3, n_steps=25, direction=1)
    ref = newmark.analysis(cfg, tol=1e-12)
    wave, stats, m = gsw.analysis(ctx, cfg, tol=1e-12, precision=1, inner_iters=10, batch_outer=40,
                                  coarse_weight=0.7)
    assert m.n_nodes % 4 != 0
    assert _relerr(wave, ref["wave"]) <= 1e-9
    m.free()


def test_two_level_directions_in_lockstep(ctx):
    """The three input directions of one model advance in lockstep (shared inner-operator
    passes), each with its own coarse correction: every direction matches its oracle run."""
    cfg = configs.config1(n_steps=24)
    m = ctx.upload(cfg["mesh"], cfg["mat"], cfg["rec_xy"])
    m.set_time(cfg["dt"], 24, cfg["band"])
    for d in range(3):
        m.set_input(d, cfg["p"])
    m.set_solver(tol=1e-8, precision=2, inner_iters=30, inner_rtol=1e-2, share_dirs=1, coarse_weight=0.7)
    m.run(dirs_mask=7)
    for d in range(3):
        ref = newmark.analysis(dict(cfg, dir=d), tol=1e-8)
        assert _relerr(m.waveforms(d), ref["wave"]) <= 1e-6, d
    m.free()


def test_two_level_cuts_inner_iterations_on_the_realistic_crop(ctx):
    """The realistic model's layers and input on its 120 x 120 m lateral crop (106,875 DOF),
    60 steps from rest with the bench's inner schedule (stop at an 80-fold drop, at most 45
    iterations): the two-level preconditioner reaches the oracle's waveforms, like the block-
    Jacobi inner preconditioner, with fewer inner iterations.

    Tolerance: the mixed paths' bar, surface-velocity relative L2 <= 1e-4 against the FP64
    oracle (each step stops at relative residual 1e-8, so an increment carries a relative error
    up to about kappa * 1e-8, kappa ~ 100 at this dt, and over the first 60 steps from rest the
    small early arrivals dominate the relative L2); the two-level run may not be further from
    the oracle than the block-Jacobi run by more than half."""
    cfg = configs.config2(n_steps=60, crop=12)
    ref = newmark.analysis(cfg, tol=1e-8)["wave"]
    out = {}
    for w in (0.0, 0.7):
        m = ctx.upload(cfg["mesh"], cfg["mat"], cfg["rec_xy"])
        m.set_time(cfg["dt"], cfg["n_steps"], cfg["band"])
        m.set_input(cfg["dir"], cfg["p"])
        m.set_solver(tol=1e-8, precision=2, inner_iters=45, inner_rtol=0.0125, guess_order=4, coarse_weight=w)
        m.step(60)
        st = m.stats()
        out[w] = dict(wave=m.waveforms(), inner=st["inner_iters_total"], outer=st["cg_iters_total"],
                      relres=st["relres_last"])
        m.free()
    e0, e1 = _relerr(out[0.0]["wave"], ref), _relerr(out[0.7]["wave"], ref)
    print("inner iterations block Jacobi %d, two-level %d; outer %d, %d; waveform error vs oracle %.2e, %.2e" % (
        out[0.0]["inner"], out[0.7]["inner"], out[0.0]["outer"], out[0.7]["outer"], e0, e1))
    assert out[0.7]["relres"] <= 1e-8
    assert e0 <= 1e-4 and e1 <= 1e-4 and e1 <= 1.5 * e0
    assert out[0.7]["inner"] < 0.9 * out[0.0]["inner"]


def test_two_level_in_a_batch_of_models(ctx):
    """Three different models advance as one batch (one captured graph per step, the coarse
    level switched per member by its own outer residual): each matches its oracle run."""
    cfgs = [configs.small_box(nx=4, ny=3, n_steps=30, seed=s, direction=s % 3) for s in (3, 4, 5)]
    ms = []
    for cfg in cfgs:
        m = ctx.upload(cfg["mesh"], cfg["mat"], cfg["rec_xy"])
        m.set_time(cfg["dt"], cfg["n_steps"], cfg["band"])
        m.set_input(cfg["dir"], cfg["p"])
        m.set_solver(tol=1e-8, precision=2, inner_iters=20, inner_rtol=1e-2, guess_order=4, coarse_weight=1.0,
                     coarse_relres=1e-5)
        ms.append(m)
    ctx.run(ms)
    for cfg, m in zip(cfgs, ms):
        ref = newmark.analysis(cfg, tol=1e-8)["wave"]
        assert _relerr(m.waveforms(), ref) <= 1e-6
        assert m.stats()["relres_last"] <= 1e-8
        m.free()
