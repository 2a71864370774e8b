"""Seeded synthetic workloads.

Each function returns a plain dict of numpy arrays and scalars:

* ``mesh``: output of :func:`synth.mesh.layered_box`;
* ``mat``: float64 [n_mat, 4] rows (Vp, Vs, rho, h) -- P/S velocity (m/s),
  density (kg/m^3) and damping ratio h of each layer (top layer first);
* ``dt``, ``n_steps``: time increment (s) and number of steps;
* ``band``: (f1, f2) Hz band of the Rayleigh-damping fit;
* ``p``: float64 [n_steps] input velocity at t_{n+1} = (n+1) dt;
* ``dir``: input direction (0 = x1, 1 = x2, 2 = x3);
* ``rec_xy``: float64 [n_rec, 2] receiver positions on the free surface.

The paper's own data (borehole records, the survey-point depths, the
reference model's layer map) are not available; these workloads stand in
for them with the sizes and structure of the paper's analyses.
"""
import numpy as np

from .fields import grf2d
from .mesh import layered_box
from .waves import random_phase, ricker, sin2_pulse

MAT_TWO_LAYER = np.array([[1500.0, 150.0, 1700.0, 0.03],
                          [1800.0, 500.0, 1900.0, 0.01]])
MAT_THREE_LAYER = np.array([[1500.0, 150.0, 1700.0, 0.03],
                            [1800.0, 400.0, 1850.0, 0.02],
                            [2500.0, 1000.0, 2100.0, 0.01]])


def grid_receivers(x0, step, n):
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    return np.stack([x0 + step * i.ravel(), x0 + step * j.ravel()], axis=1).astype(np.float64)


def config1(n_steps=500, direction=0):
    """Plain FP64 single model: 100 x 100 x 50 m, soft 0-20 m over hard rock.

    12 x 12 lateral cells, 4 soft cells of 5 m and 2 hard cells of 15 m
    (8,125 nodes, 24,375 DOF, 5,184 tetrahedra); 2 Hz Ricker SV input,
    dt = 0.01 s, 25 receivers at (10 + 20 i, 10 + 20 j).
    """
    mesh = layered_box(12, 12, 100.0, 100.0, [4, 2], [20.0], 50.0)
    dt = 0.01
    t = dt * np.arange(1, n_steps + 1)
    return dict(mesh=mesh, mat=MAT_TWO_LAYER.copy(), dt=dt, n_steps=n_steps, band=(0.5, 5.0),
                p=ricker(t, 2.0, 0.75, 0.01), dir=direction, rec_xy=grid_receivers(10.0, 20.0, 5),
                name="two-layer 100x100x50 m, 24,375 DOF")


def _three_layer_interfaces(nx, h, ell, rng, crop=None):
    n = nx + 1
    g1 = grf2d(n, n, h, ell, rng)
    g2 = grf2d(n, n, h, ell, rng)
    soft = np.clip(35.0 + 10.0 * g1, 10.0, 60.0)
    mid = np.clip(150.0 + 25.0 * g2, 100.0, 200.0)
    if crop is not None:
        soft, mid = soft[:crop + 1, :crop + 1], mid[:crop + 1, :crop + 1]
    return [soft, mid]


def config2(n_steps=4000, seed=2, crop=None, direction=0):
    """Realistic single model: 1.2 x 1.2 x 0.3 km, three layers, ~9.93 M DOF.

    120 x 120 lateral cells of 10 m; 4 soft + 10 intermediate + 14 bedrock
    cell levels (241 x 241 x 57 = 3,310,617 nodes, 2,419,200 tetrahedra).
    Soft-layer depth clip(35 + 10 g, 10, 60) m and intermediate/bedrock depth
    clip(150 + 25 g', 100, 200) m with g, g' unit Gaussian random fields of
    correlation length 200 m.  Band-limited 0.1-2.5 Hz random-phase input,
    dt = 0.005 s, 100 receivers at (60 + 120 i, 60 + 120 j).

    ``crop`` (lateral cells) keeps the first ``crop`` x ``crop`` cells of the
    same interface realisation and cell size: a bounded sample of the same
    workload for CPU timing.
    """
    rng = np.random.default_rng(seed)
    nx = 120
    itf = _three_layer_interfaces(nx, 10.0, 200.0, rng, crop)
    n = nx if crop is None else crop
    L = 10.0 * n
    mesh = layered_box(n, n, L, L, [4, 10, 14], itf, 300.0)
    dt = 0.005
    p = random_phase(n_steps, dt, np.random.default_rng(seed + 100))
    rec = grid_receivers(60.0, 120.0, 10)
    rec = rec[(rec[:, 0] < L) & (rec[:, 1] < L)]
    return dict(mesh=mesh, mat=MAT_THREE_LAYER.copy(), dt=dt, n_steps=n_steps, band=(0.1, 2.5),
                p=p, dir=direction, rec_xy=rec,
                name="three-layer %gx%gx300 m, %d DOF" % (L, L, 3 * mesh["xyz"].shape[0]))


def config3_candidate(l, n_steps=2000, direction=0, n_lateral=None):
    """Batched-ensemble candidate l: config-1 box, seeded soft-layer depth.

    Soft depth clip(20 + 5 g, 10, 30) m, g a unit GRF of correlation length
    40 m (seed 1000 + l); lateral cells n ~ U{35..62} (seeded), n_z =
    ceil(n / 2) levels split 40 % soft / 60 % hard; sin^2 basis pulse with
    T_p = 0.4 s; dt = 0.01 s.  ``l = -1`` is the hidden truth model (seed
    999, n = 48).
    """
    if l < 0:
        rng = np.random.default_rng(999)
        n = 48
    else:
        rng = np.random.default_rng(1000 + l)
        n = int(rng.integers(35, 63))
    if n_lateral is not None:
        n = n_lateral
    nz = int(np.ceil(n / 2))
    ns = max(1, int(round(0.4 * nz)))
    soft = np.clip(20.0 + 5.0 * grf2d(n + 1, n + 1, 100.0 / n, 40.0, rng), 10.0, 30.0)
    mesh = layered_box(n, n, 100.0, 100.0, [ns, nz - ns], [soft], 50.0)
    dt = 0.01
    t = dt * np.arange(1, n_steps + 1)
    return dict(mesh=mesh, mat=MAT_TWO_LAYER.copy(), dt=dt, n_steps=n_steps, band=(0.5, 5.0),
                p=sin2_pulse(t, 0.4), dir=direction, rec_xy=grid_receivers(10.0, 20.0, 5),
                name="candidate %d (%d lateral cells)" % (l, n))


def config4_candidate(l, n_steps=2000, direction=0):
    """Mixed-precision-ensemble candidate l: 120 x 120 x 300 m, ~287 k DOF.

    20 x 20 lateral cells of 6 m, 4 + 10 + 14 levels (41 x 41 x 57 =
    95,817 nodes), three-layer statistics of the realistic model with
    correlation length 20 m (seed 5000 + l); sin^2 basis pulse T_p = 0.4 s;
    dt = 0.005 s; 25 receivers at (12 + 24 i, 12 + 24 j).
    """
    rng = np.random.default_rng(5000 + l)
    itf = _three_layer_interfaces(20, 6.0, 20.0, rng)
    mesh = layered_box(20, 20, 120.0, 120.0, [4, 10, 14], itf, 300.0)
    dt = 0.005
    t = dt * np.arange(1, n_steps + 1)
    return dict(mesh=mesh, mat=MAT_THREE_LAYER.copy(), dt=dt, n_steps=n_steps, band=(0.1, 2.5),
                p=sin2_pulse(t, 0.4), dir=direction, rec_xy=grid_receivers(12.0, 24.0, 5),
                name="candidate %d (120x120x300 m)" % l)


def small_box(nx=3, ny=2, counts=(2, 1), depth=30.0, L=(30.0, 20.0), n_steps=20, seed=7,
              distort=True, direction=0, dt=0.01):
    """Tiny two-layer box for unit and parity tests (a few hundred nodes).

    With ``distort`` the interface is a seeded random surface, so elements
    are genuinely irregular.
    """
    rng = np.random.default_rng(seed)
    itf = 12.0 + (3.0 * rng.uniform(-1, 1, size=(nx + 1, ny + 1)) if distort else 0.0)
    mesh = layered_box(nx, ny, L[0], L[1], list(counts), [itf], depth)
    t = dt * np.arange(1, n_steps + 1)
    rec = np.array([[0.31 * L[0], 0.47 * L[1]], [0.77 * L[0], 0.2 * L[1]], [0.5 * L[0], 0.5 * L[1]]])
    return dict(mesh=mesh, mat=MAT_TWO_LAYER.copy(), dt=dt, n_steps=n_steps, band=(0.5, 5.0),
                p=ricker(t, 4.0, 0.1, 0.01), dir=direction, rec_xy=rec, name="small box")
