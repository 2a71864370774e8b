"""Pins of the oracle's solver and Newmark time stepping (CPU only).

* PCG against a dense direct solve, with its stop rule;
* the discrete Newmark average-acceleration frequency of a single mode,
  (2/dt) atan(w dt / 2), on a generalised eigenvector of (K, M);
* exact energy conservation with damping, dashpots and force off, and
  monotone decay with Rayleigh damping on;
* the closed-form 1D transfer function of vertically incident S and P waves
  through horizontal layers over the absorbing base (homogeneous column:
  surface velocity = 2 v_in(t - D/V)), with O(dt^2) and fast h convergence;
* linearity and time invariance: a direct run with a superposed input equals
  the superposition of shifted single-pulse responses.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import fem, misfit, newmark, transfer1d
from synth import configs
from synth.configs import MAT_TWO_LAYER
from synth.mesh import layered_box
from synth.waves import ricker, sin2_pulse


def _tiny():
    cfg = configs.small_box(nx=2, ny=2, counts=(1, 1), depth=20.0, L=(20.0, 20.0), distort=True)
    ops = fem.assemble(cfg["mesh"], cfg["mat"], cfg["band"])
    return cfg, ops


def test_pcg_matches_dense_solve_and_stop_rule():
    cfg, ops = _tiny()
    dt = 0.01
    A = (ops["K"] + (2 / dt) * (ops["CR"] + ops["Cabs"]) + (4 / dt ** 2) * ops["M"]).tocsr()
    rng = np.random.default_rng(0)
    b = rng.standard_normal(A.shape[0])
    Dinv = newmark.block_jacobi_inverse(A)
    # D^-1 really inverts the 3x3 nodal diagonal blocks
    Ad = A.toarray()
    for n in (0, 5, A.shape[0] // 3 - 1):
        np.testing.assert_allclose(Dinv[n] @ Ad[3 * n:3 * n + 3, 3 * n:3 * n + 3], np.eye(3), atol=1e-12)
    for tol in (1e-6, 1e-10):
        x, it, rel = newmark.pcg(A, b, np.zeros_like(b), Dinv, tol, 5000)
        true = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
        assert rel <= tol and true <= 2 * tol
        xd = np.linalg.solve(Ad, b)
        cond = np.linalg.cond(Ad)
        assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 2 * tol * cond
    # zero right-hand side gives zero, in zero iterations
    x, it, _ = newmark.pcg(A, np.zeros_like(b), b, Dinv, 1e-8, 10)
    assert it == 0 and not x.any()
    with pytest.raises(newmark.NoConvergence):
        newmark.pcg(A, b, np.zeros_like(b), Dinv, 1e-14, 2)


def test_newmark_modal_frequency():
    cfg, ops = _tiny()
    K, M = ops["K"], ops["M"]
    w2, V = sla.eigh(K.toarray(), M.toarray())
    idx = np.argmin(np.abs(w2 - np.median(w2[w2 > 1e-6 * w2.max()])))
    w, phi = np.sqrt(w2[idx]), V[:, idx]
    dt = 0.4 / w
    n_steps = 40
    zero = 0.0 * K
    seen = np.zeros(n_steps)
    newmark.newmark_run(K, M, zero, lambda n: np.zeros(K.shape[0]), dt, n_steps, u0=phi,
                        v0=np.zeros_like(phi), a0=-w2[idx] * phi, tol=1e-13,
                        observe=lambda n, u, v, a: seen.__setitem__(n, (u @ (M @ phi)) / (phi @ (M @ phi))))
    wbar = (2.0 / dt) * np.arctan(w * dt / 2.0)
    ref = np.cos(wbar * dt * np.arange(1, n_steps + 1))
    np.testing.assert_allclose(seen, ref, atol=1e-9)
    # and it is not the exact frequency
    assert np.abs(seen - np.cos(w * dt * np.arange(1, n_steps + 1))).max() > 1e-4


def test_energy_conservation_and_damped_decay():
    cfg, ops = _tiny()
    K, M = ops["K"], ops["M"]
    rng = np.random.default_rng(1)
    v0 = rng.standard_normal(K.shape[0]) * 1e-3
    energies = []

    def obs(n, u, v, a):
        energies.append(0.5 * v @ (M @ v) + 0.5 * u @ (K @ u))

    newmark.newmark_run(K, M, 0.0 * K, lambda n: np.zeros(K.shape[0]), 0.01, 200, v0=v0, tol=1e-13, observe=obs)
    E0 = 0.5 * v0 @ (M @ v0)
    assert np.abs(np.array(energies) / E0 - 1.0).max() < 1e-10
    energies.clear()
    newmark.newmark_run(K, M, ops["CR"], lambda n: np.zeros(K.shape[0]), 0.01, 200, v0=v0, tol=1e-13, observe=obs)
    e = np.array(energies)
    assert np.all(np.diff(e) <= 1e-12 * E0) and e[-1] < 0.5 * E0


def _column(direction, counts=(4, 2), dt=0.01, n_steps=300, mat=MAT_TWO_LAYER):
    mesh = layered_box(3, 3, 15.0, 15.0, list(counts), [20.0], 50.0, periodic=True)
    t = dt * np.arange(1, n_steps + 1)
    cfg = dict(mesh=mesh, mat=mat, dt=dt, n_steps=n_steps, band=(0.5, 5.0), p=ricker(t, 2.0, 0.75, 0.01),
               dir=direction, rec_xy=np.array([[2.5, 2.5], [11.0, 7.0]]))
    ops = fem.assemble(mesh, mat, cfg["band"])
    out = newmark.analysis(cfg, tol=1e-10, ops=ops)
    lam, mu, rho = fem.lame(mat)
    G = mu if direction < 2 else lam + 2 * mu
    V = mat[:, 1] if direction < 2 else mat[:, 0]
    ab = ops["rayleigh"]
    layers = [(20.0, rho[0], G[0], ab[0, 0], ab[0, 1]), (30.0, rho[1], G[1], ab[1, 0], ab[1, 1])]
    ref = transfer1d.surface_response(cfg["p"], dt, layers, rho[1] * V[1])
    return out["wave"], ref


def test_transfer_function_homogeneous_closed_form():
    f = np.linspace(0.0, 5.0, 51)
    D, V, rho = 50.0, 500.0, 1900.0
    H = transfer1d.transfer(f, [(D, rho, rho * V * V, 0.0, 0.0)], rho * V)
    np.testing.assert_allclose(H, 2.0 * np.exp(-2j * np.pi * f * D / V), atol=1e-12)
    # layer over half-space: resonance at V1 / (4 H) with amplification 2 Z2 / Z1
    H1, V1, r1, V2, r2 = 20.0, 150.0, 1700.0, 500.0, 1900.0
    f0 = V1 / (4 * H1)
    Hf = transfer1d.transfer([f0], [(H1, r1, r1 * V1 ** 2, 0.0, 0.0), (1e-9, r2, r2 * V2 ** 2, 0.0, 0.0)], r2 * V2)
    np.testing.assert_allclose(abs(Hf[0]), 2.0 * r2 * V2 / (r1 * V1), rtol=1e-9)


def test_homogeneous_column_doubles_and_delays():
    mat = np.array([[1800.0, 500.0, 1900.0, 0.0], [1800.0, 500.0, 1900.0, 0.0]])
    wave, _ = _column(0, dt=0.005, n_steps=400, mat=mat)
    t = 0.005 * np.arange(1, 401)
    ref = 2.0 * ricker(t - 50.0 / 500.0, 2.0, 0.75, 0.01)
    assert np.linalg.norm(wave[0, 0] - ref) / np.linalg.norm(ref) < 5e-3
    # laterally uniform: every receiver sees the same motion, other components vanish
    assert np.abs(wave[0] - wave[1]).max() < 1e-6 * np.abs(wave).max()
    assert np.abs(wave[:, 1:]).max() < 1e-6 * np.abs(wave).max()


@pytest.mark.parametrize("direction", [0, 2])
def test_layered_column_transfer_function_and_dt_order(direction):
    w1, r1 = _column(direction, dt=0.01, n_steps=300)
    w2, r2 = _column(direction, dt=0.005, n_steps=600)
    e1 = np.linalg.norm(w1[0, direction] - r1) / np.linalg.norm(r1)
    e2 = np.linalg.norm(w2[0, direction] - r2) / np.linalg.norm(r2)
    assert e1 < 1e-2, "config-1 resolution must be within 1 % of the 1D closed form"
    assert 3.0 < e1 / e2 < 5.0, "error must fall as dt^2"


def test_layered_column_h_convergence():
    errs = []
    for counts in ((1, 1), (2, 1)):
        w, r = _column(0, counts=counts, dt=0.0025, n_steps=1200)
        errs.append(np.linalg.norm(w[0, 0] - r) / np.linalg.norm(r))
    assert errs[0] / errs[1] > 8.0, "quadratic elements: at least O(h^3) in the surface velocity"


def test_linearity_and_shift_invariance():
    cfg = configs.small_box(nx=2, ny=2, counts=(1, 1), depth=20.0, L=(20.0, 20.0), n_steps=60, dt=0.01)
    ops = fem.assemble(cfg["mesh"], cfg["mat"], cfg["band"])
    s, L = 5, 4
    t = cfg["dt"] * np.arange(1, cfg["n_steps"] + 1)
    pulse = sin2_pulse(t, 2 * s * cfg["dt"])
    G = np.zeros((cfg["rec_xy"].shape[0], 3, 3, cfg["n_steps"]))
    for j in range(3):
        G[:, :, j] = newmark.analysis(dict(cfg, p=pulse, dir=j), ops=ops)["wave"]
    c = np.random.default_rng(4).standard_normal((3, L))
    U = misfit.superpose(G, c, s)
    direct = np.zeros_like(U)
    for j in range(3):
        f = sum(c[j, l] * sin2_pulse(t - l * s * cfg["dt"], 2 * s * cfg["dt"]) for l in range(L))
        direct += newmark.analysis(dict(cfg, p=f, dir=j), ops=ops)["wave"]
    assert np.abs(U - direct).max() <= 1e-8 * np.abs(direct).max()
