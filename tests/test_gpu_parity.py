"""GPU parity tests through the C ABI against the FP64 CPU oracle.

Tolerances: FP64 path at CG tolerance 1e-12 on both sides must agree to
surface-velocity relative L2 <= 1e-9; production runs at 1e-8 on both sides
to <= 1e-6 (two solutions each within 1e-8 of the exact step solution).
Operator-level checks (EBE vs assembled CSR) are exact up to rounding:
<= 1e-13 relative.
"""
import numpy as np
import pytest

from oracle import fem, misfit, newmark
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


def _upload(ctx, cfg, n_steps=None):
    m = ctx.upload(cfg["mesh"], cfg["mat"], cfg["rec_xy"])
    m.set_time(cfg["dt"], cfg["n_steps"] if n_steps is None else n_steps, cfg["band"])
    return m


def _relerr(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("distort,nx,ny", [(True, 3, 2), (True, 5, 4), (False, 4, 4)])
def test_operators_match_assembled_csr(ctx, distort, nx, ny):
    import torch

    cfg = configs.small_box(nx=nx, ny=ny, distort=distort)
    ops = fem.assemble(cfg["mesh"], cfg["mat"], cfg["band"])
    m = _upload(ctx, cfg)
    dt = cfg["dt"]
    C = ops["CR"] + ops["Cabs"]
    A = ops["K"] + (2 / dt) * C + (4 / dt ** 2) * ops["M"]
    rng = np.random.default_rng(11)
    for which, Mx in ((0, A), (1, ops["K"]), (2, ops["M"]), (3, C)):
        x = rng.standard_normal((m.n_nodes, 3))
        y = m.apply(which, torch.tensor(x, device="cuda")).cpu().numpy().ravel()
        ref = Mx @ x.ravel()
        assert _relerr(y, ref) < 1e-13, which
    # symmetry of the EBE operator
    x1 = torch.tensor(rng.standard_normal((m.n_nodes, 3)), device="cuda")
    x2 = torch.tensor(rng.standard_normal((m.n_nodes, 3)), device="cuda")
    a = float((x2 * m.apply(0, x1)).sum())
    b = float((x1 * m.apply(0, x2)).sum())
    assert abs(a - b) <= 1e-13 * abs(a)
    m.free()


def test_preconditioner_and_receivers_match(ctx):
    cfg = configs.small_box(nx=4, ny=3, distort=True)
    ops = fem.assemble(cfg["mesh"], cfg["mat"], cfg["band"])
    m = _upload(ctx, cfg)
    dt = cfg["dt"]
    A = (ops["K"] + (2 / dt) * (ops["CR"] + ops["Cabs"]) + (4 / dt ** 2) * ops["M"]).tocsr()
    Dinv = newmark.block_jacobi_inverse(A)
    d = m.preconditioner()
    full = np.stack([d[:, [0, 3, 4]], d[:, [3, 1, 5]], d[:, [4, 5, 2]]], axis=1)
    assert _relerr(full, Dinv) < 1e-12
    nodes, w = m.receivers()
    rn, rw = fem.receiver_weights(cfg["mesh"], cfg["rec_xy"])
    field = np.random.default_rng(2).standard_normal(m.n_nodes)
    np.testing.assert_allclose((w * field[nodes]).sum(1), (rw * field[rn]).sum(1), rtol=1e-12, atol=1e-12)
    m.free()


@pytest.mark.parametrize("direction", [0, 1, 2])
def test_small_box_time_stepping_fp64(ctx, direction):
    cfg = configs.small_box(nx=4, ny=3, n_steps=30, direction=direction)
    ref = newmark.analysis(cfg, tol=1e-12)
    from paper_2404_17754_gb300 import gsw

    wave, stats, m = gsw.analysis(ctx, cfg, tol=1e-12)
    assert _relerr(wave, ref["wave"]) <= 1e-9
    assert abs(stats["cg_iters_total"] - ref["iters"].sum()) <= cfg["n_steps"]
    u, v, a, step = m.get_state()
    assert step == cfg["n_steps"]
    assert _relerr(v.ravel(), ref["v"]) <= 1e-9
    m.free()


def test_config1_fp64_parity_tight(ctx):
    """Two-layer 24,375-DOF model, 40 steps at CG tolerance 1e-12."""
    from paper_2404_17754_gb300 import gsw

    cfg = configs.config1(n_steps=40)
    ref = newmark.analysis(cfg, tol=1e-12)
    wave, stats, m = gsw.analysis(ctx, cfg, tol=1e-12)
    assert _relerr(wave, ref["wave"]) <= 1e-9
    m.free()


def test_config1_production_tolerance(ctx):
    """Production relative residual 1e-8 on both sides: agreement <= 1e-6."""
    from paper_2404_17754_gb300 import gsw

    cfg = configs.config1(n_steps=60)
    ref = newmark.analysis(cfg, tol=1e-8)
    wave, stats, m = gsw.analysis(ctx, cfg, tol=1e-8)
    assert _relerr(wave, ref["wave"]) <= 1e-6
    assert stats["relres_last"] <= 1e-8
    # same iteration counts up to rounding at the stopping threshold
    assert abs(stats["cg_iters_total"] - ref["iters"].sum()) <= 60
    m.free()


def test_checkpoint_restore_continues_identically(ctx):
    from paper_2404_17754_gb300 import gsw

    cfg = configs.small_box(nx=3, ny=3, n_steps=24)
    m = _upload(ctx, cfg)
    m.set_input(cfg["dir"], cfg["p"])
    m.set_solver(tol=1e-12)
    m.step(12)
    u, v, a, step = m.get_state()
    m.step(12)
    w_full = m.waveforms()
    m.reset()
    m.set_state(u, v, a, step)
    m.step(12)
    w_resumed = m.waveforms()
    # atomic scatter order differs run to run: equal up to rounding
    np.testing.assert_allclose(w_resumed[:, :, 12:], w_full[:, :, 12:], rtol=0, atol=1e-10 * np.abs(w_full).max())
    m.free()


def test_error_paths(ctx):
    from paper_2404_17754_gb300 import gsw

    cfg = configs.small_box(nx=3, ny=2, n_steps=10)
    mesh = dict(cfg["mesh"])
    bad = mesh["conn"].copy()
    bad[3, 4] = mesh["xyz"].shape[0] + 5
    with pytest.raises(gsw.GswError) as e:
        ctx.upload(dict(mesh, conn=bad), cfg["mat"], cfg["rec_xy"])
    assert e.value.status == gsw.E_INVALID
    flipped = mesh["conn"].copy()
    flipped[0, [1, 2]] = flipped[0, [2, 1]]
    flipped[0, 4:] = mesh["conn"][0, [4 + 2, 4 + 1, 4 + 0, 4 + 3, 4 + 5, 4 + 4]]
    with pytest.raises(gsw.GswError) as e:
        ctx.upload(dict(mesh, conn=flipped), cfg["mat"], cfg["rec_xy"])
    assert e.value.status == gsw.E_INVALID and "volume" in str(e.value)
    with pytest.raises(gsw.GswError):
        ctx.upload(mesh, cfg["mat"], np.array([[1e4, 1e4]]))
    m = _upload(ctx, cfg)
    with pytest.raises(gsw.GswError) as e:
        m.set_input(0, np.full(cfg["n_steps"], np.nan))
    assert e.value.status == gsw.E_INVALID
    m.set_input(0, cfg["p"])
    m.set_solver(tol=1e-14, max_iter=2)
    with pytest.raises(gsw.GswError) as e:
        m.step(3)
    assert e.value.status == gsw.E_NOCONV
    with pytest.raises(gsw.GswError) as e:
        m.step(1)
    assert e.value.status == gsw.E_STATE
    m.reset()
    m.set_solver(tol=1e-8)
    m.step(cfg["n_steps"])
    m.free()


def test_misfit_matches_oracle_and_inverse_crime(ctx):
    rng = np.random.default_rng(3)
    n_rec, n_t, s, L = 5, 200, 8, 10
    t = np.arange(n_t)
    G = np.zeros((n_rec, 3, 3, n_t))
    for k in range(n_rec):
        for i in range(3):
            for j in range(3):
                G[k, i, j] = rng.standard_normal() * np.sin(2 * np.pi * rng.uniform(0.01, 0.08) * t) * np.exp(-t / 90)
    obs = rng.standard_normal((n_rec, 3, n_t))
    obs[2, 1] = 0.0  # dropped pair
    e_gpu, c_gpu = ctx.misfit_green(G, obs, s, L, tau=1e-10)
    e_ref, c_ref = misfit.estimate(G, obs, s, L, tau=1e-10)
    assert abs(e_gpu - e_ref) <= 1e-9 * e_ref
    assert np.abs(c_gpu - c_ref).max() <= 1e-8 * np.abs(c_ref).max()
    c_true = rng.standard_normal((3, L))
    obs2 = misfit.superpose(G, c_true, s)
    e2, c2 = ctx.misfit_green(G, obs2, s, L, tau=1e-12)
    assert e2 < 1e-8
    np.testing.assert_allclose(c2, c_true, atol=1e-7)


def _sampled_rows(mesh, mat, band, nodes):
    """Oracle operator rows at `nodes` from the elements and faces touching them only."""
    conn = mesh["conn"]
    el = np.nonzero(np.isin(conn, nodes).any(axis=1))[0]
    fc = np.nonzero(np.isin(mesh["faces"], nodes).any(axis=1))[0]
    sub = dict(mesh, conn=conn[el], elem_mat=mesh["elem_mat"][el], faces=mesh["faces"][fc],
               face_elem=np.searchsorted(el, mesh["face_elem"][fc]), face_tag=mesh["face_tag"][fc])
    assert np.all(el[sub["face_elem"]] == mesh["face_elem"][fc])
    return fem.assemble(sub, mat, band)


def test_realistic_model_full_size_sampled_rows_and_true_residual(ctx):
    """Full 9.93 M DOF three-layer model: sampled operator rows vs the oracle,
    and the true Newmark residual of GPU steps at relative residual 1e-8."""
    import torch

    cfg = configs.config2(n_steps=4)
    mesh = cfg["mesh"]
    m = _upload(ctx, cfg)
    dt = cfg["dt"]
    rng = np.random.default_rng(5)
    nodes = rng.choice(m.n_nodes, 24, replace=False)
    ops = _sampled_rows(mesh, cfg["mat"], cfg["band"], nodes)
    x = rng.standard_normal((m.n_nodes, 3))
    xt = torch.tensor(x, device="cuda")
    rows = (3 * nodes[:, None] + np.arange(3)).ravel()
    C = ops["CR"] + ops["Cabs"]
    A = ops["K"] + (2 / dt) * C + (4 / dt ** 2) * ops["M"]
    for which, Mx in ((0, A), (1, ops["K"]), (2, ops["M"]), (3, C)):
        y = m.apply(which, xt).cpu().numpy().ravel()[rows]
        ref = (Mx @ x.ravel())[rows]
        assert _relerr(y, ref) < 1e-12, which
    # steps at production tolerance; check the equation of motion at t_{n+1}
    m.set_input(cfg["dir"], cfg["p"])
    m.set_solver(tol=1e-8)
    m.step(2)
    u0, v0, a0, _ = m.get_state()
    m.step(1)
    u1, v1, a1, _ = m.get_state()
    st = m.stats()
    assert st["relres_last"] <= 1e-8
    base = fem.assemble(dict(mesh, conn=mesh["conn"][:1], elem_mat=mesh["elem_mat"][:1],
                             faces=mesh["faces"][mesh["face_tag"] == 1],
                             face_elem=np.zeros(int((mesh["face_tag"] == 1).sum()), dtype=np.int32),
                             face_tag=mesh["face_tag"][mesh["face_tag"] == 1]),
                        np.repeat(cfg["mat"][-1:], cfg["mat"].shape[0], axis=0), cfg["band"])
    f = 2.0 * cfg["p"][2] * base["w"][cfg["dir"]]
    tt = lambda a: torch.tensor(a, device="cuda")
    lhs = (m.apply(2, tt(a1)) + m.apply(3, tt(v1)) + m.apply(1, tt(u1))).cpu().numpy().ravel()
    res = f - lhs
    Adu = m.apply(0, tt(u1 - u0)).cpu().numpy().ravel()
    b = Adu + res
    assert np.linalg.norm(res) / np.linalg.norm(b) <= 2e-8
    m.free()
