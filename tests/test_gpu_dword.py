"""Double-word (paired FP32) outer operator against the FP64 oracle.

A double-word value carries about 48 significant bits and each operation is
an error-free transformation, so A x agrees with the FP64 assembled operator
to a few units of 2^-46 times the cancellation of the element sums: <= 1e-12
relative for random vectors (no cancellation beyond the operator's own), and
<= 1e-10 for a smooth displacement field (wavelength about ten elements,
where K x cancels by about (wavelength / element size)^2).  Solves with the
double-word operator converge to the same tolerance, so they agree with the
FP64-operator solve and with the oracle like two FP64 solves do.
"""
import numpy as np
import pytest

from oracle import fem, newmark
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


def _upload(ctx, cfg):
    m = ctx.upload(cfg["mesh"], cfg["mat"], cfg["rec_xy"])
    m.set_time(cfg["dt"], cfg["n_steps"], cfg["band"])
    return m


@pytest.mark.parametrize("distort,nx,ny", [(True, 3, 2), (True, 5, 4), (False, 4, 4)])
def test_dword_operator_matches_assembled_csr(ctx, distort, nx, ny):
    import torch

    cfg = configs.small_box(nx=nx, ny=ny, distort=distort)
    ops = fem.assemble(cfg["mesh"], cfg["mat"], cfg["band"])
    dt = cfg["dt"]
    A = ops["K"] + (2 / dt) * (ops["CR"] + ops["Cabs"]) + (4 / dt ** 2) * ops["M"]
    m = _upload(ctx, cfg)
    rng = np.random.default_rng(21)
    x = rng.standard_normal((m.n_nodes, 3))
    ref = A @ x.ravel()
    for scale in (1.0, 1e-12, 1e12):
        y = m.apply(5, torch.tensor(scale * x, device="cuda")).cpu().numpy().ravel()
        assert _relerr(y, scale * ref) < 1e-12, scale
    # a smooth field: the stiffness sums cancel, the mass does not
    xyz = cfg["mesh"]["xyz"]
    L = np.ptp(xyz, axis=0).max()
    k = 2 * np.pi / (L / 2)
    xs = np.stack([np.sin(k * xyz[:, 0] + 0.3), np.cos(k * xyz[:, 1]), np.sin(k * (xyz[:, 2] + xyz[:, 0]))], axis=1)
    y = m.apply(5, torch.tensor(xs, device="cuda")).cpu().numpy().ravel()
    assert _relerr(y, A @ xs.ravel()) < 1e-10
    yk = m.apply(5, torch.tensor(xs, device="cuda")).cpu().numpy().ravel()
    assert np.linalg.norm(yk - y) / np.linalg.norm(y) < 1e-13  # atomics: only the summation order varies
    m.free()


def test_dword_operator_full_size_sampled_rows(ctx):
    """Full 9.93 M DOF three-layer model: sampled rows of the double-word A x vs the oracle."""
    import torch
    from test_gpu_parity import _sampled_rows

    cfg = configs.config2(n_steps=4)
    m = _upload(ctx, cfg)
    dt = cfg["dt"]
    rng = np.random.default_rng(6)  # sampled nodes may or may not touch dashpot faces
    nodes = rng.choice(m.n_nodes, 24, replace=False)
    ops = _sampled_rows(cfg["mesh"], cfg["mat"], cfg["band"], nodes)
    A = ops["K"] + (2 / dt) * (ops["CR"] + ops["Cabs"]) + (4 / dt ** 2) * ops["M"]
    x = rng.standard_normal((m.n_nodes, 3))
    xt = torch.tensor(x, device="cuda")
    rows = (3 * nodes[:, None] + np.arange(3)).ravel()
    y5 = m.apply(5, xt).cpu().numpy().ravel()
    y0 = m.apply(0, xt).cpu().numpy().ravel()
    assert _relerr(y5[rows], (A @ x.ravel())[rows]) < 1e-12
    assert _relerr(y5, y0) < 1e-12
    m.free()


@pytest.mark.parametrize("prec", [1, 2])
def test_mixed_solve_dword_matches_fp64_outer(ctx, prec):
    from paper_2404_17754_gb300 import gsw

    cfg = configs.config3_candidate(7, n_steps=30, direction=1, n_lateral=6)
    out = {}
    for op in (gsw.OUTER_FP64, gsw.OUTER_AUTO):
        m = _upload(ctx, cfg)
        m.set_input(cfg["dir"], cfg["p"])
        m.set_solver(tol=1e-8, precision=prec, inner_iters=12, outer_op=op, guess_order=2)
        m.step(cfg["n_steps"])
        st = m.stats()
        assert st["relres_last"] <= 1e-8
        out[op] = (m.waveforms(), st["cg_iters_total"])
        m.free()
    (w64, it64), (wdw, itdw) = out[gsw.OUTER_FP64], out[gsw.OUTER_AUTO]
    assert _relerr(wdw, w64) <= 1e-7
    assert abs(itdw - it64) <= max(2, 0.05 * it64)
    assert _relerr(wdw, newmark.analysis(cfg, tol=1e-8)["wave"]) <= 1e-6


def test_fp64_mode_with_dword_operator(ctx):
    from paper_2404_17754_gb300 import gsw

    cfg = configs.small_box(nx=4, ny=3, n_steps=25, direction=2, seed=3)
    m = _upload(ctx, cfg)
    m.set_input(cfg["dir"], cfg["p"])
    m.set_solver(tol=1e-10, outer_op=gsw.OUTER_DWORD)
    m.step(cfg["n_steps"])
    assert m.stats()["relres_last"] <= 1e-10
    assert _relerr(m.waveforms(), newmark.analysis(cfg, tol=1e-10)["wave"]) <= 1e-8
    with pytest.raises(gsw.GswError) as e:
        m.set_solver(tol=1e-8, outer_op=3)
    assert e.value.status == gsw.E_INVALID
    m.free()
