"""Candidate ground-model pool from survey points (Section 3, candidate models).

The paper builds its pool from the first/second-layer boundary depth known at
120 survey points: the boundary depth at any lateral position is the inverse
distance weighted (IDW) mean of the M nearest survey values with weights
1/d^q (Section 3, the IDW equation), for M = 1..50 and q = 0.1, 0.2, ..., 4.0
(2000 models); the boundary is then Laplace-smoothed five times, and the
models that differ most from the one built with the common choice M = 20,
q = 2.0 are kept.  The survey data are not available, so the survey points
and their depths are seeded synthetic stand-ins (a Gaussian random field
sampled at random positions).

Readings where the paper is silent (each listed in the design notes):

* a survey point at distance 0 from the evaluation point returns its own
  depth (the IDW limit d -> 0);
* ties in distance are broken by survey-point index (stable sort);
* one Laplace smoothing pass replaces every lattice value by the mean of its
  4-neighbours that lie inside the lattice (the boundary keeps its
  available neighbours);
* "substantial variation" ranks the pool by the RMS difference of the
  smoothed boundary from the reference (M = 20, q = 2.0) boundary and keeps
  the n largest (ties by pool index).

Everything here is input generation (no part of the analysis arithmetic).
"""
import numpy as np

from .fields import grf2d
from .mesh import layered_box

M_VALUES = tuple(range(1, 51))
Q_VALUES = tuple(round(0.1 * i, 1) for i in range(1, 41))


def survey_points(n=120, L=600.0, mean=20.0, amp=5.0, ell=100.0, lo=10.0, hi=30.0, seed=0):
    """Seeded survey points: positions uniform in [0, L]^2 and boundary depths
    sampled from a Gaussian random field clip(mean + amp g, lo, hi)."""
    rng = np.random.default_rng(seed)
    xy = rng.uniform(0.0, L, size=(n, 2))
    nf = 65
    g = grf2d(nf, nf, L / (nf - 1), ell, rng)
    # bilinear sample of the field at the survey positions
    s = xy / (L / (nf - 1))
    i0 = np.minimum(np.floor(s).astype(int), nf - 2)
    f = s - i0
    z = ((1 - f[:, 0]) * (1 - f[:, 1]) * g[i0[:, 0], i0[:, 1]] + f[:, 0] * (1 - f[:, 1]) * g[i0[:, 0] + 1, i0[:, 1]]
         + (1 - f[:, 0]) * f[:, 1] * g[i0[:, 0], i0[:, 1] + 1] + f[:, 0] * f[:, 1] * g[i0[:, 0] + 1, i0[:, 1] + 1])
    return xy, np.clip(mean + amp * z, lo, hi)


def idw(points, values, x, y, M, q):
    """IDW estimate at the positions (x, y) (arrays of one shape) from the M
    nearest points with weights d^-q (Section 3, the IDW equation)."""
    P = np.asarray(points, dtype=np.float64)
    z = np.asarray(values, dtype=np.float64)
    X = np.stack([np.ravel(x), np.ravel(y)], axis=1)
    d = np.sqrt(((X[:, None, :] - P[None, :, :]) ** 2).sum(axis=2))
    M = min(int(M), P.shape[0])
    order = np.argsort(d, axis=1, kind="stable")[:, :M]
    dn = np.take_along_axis(d, order, axis=1)
    zn = z[order]
    out = np.empty(X.shape[0])
    exact = dn[:, 0] == 0.0
    out[exact] = zn[exact, 0]
    # weights d^-q scaled by the nearest distance (same ratios, no underflow)
    dd = dn[~exact]
    w = (dd[:, :1] / dd) ** float(q)
    out[~exact] = (w * zn[~exact]).sum(axis=1) / w.sum(axis=1)
    return out.reshape(np.shape(x))


def laplace_smooth(z, times=5):
    """``times`` passes of 4-neighbour averaging on a 2D lattice (boundary
    values average the neighbours that exist)."""
    z = np.asarray(z, dtype=np.float64).copy()
    n1, n2 = z.shape
    cnt = np.zeros((n1, n2))
    cnt[1:, :] += 1
    cnt[:-1, :] += 1
    cnt[:, 1:] += 1
    cnt[:, :-1] += 1
    for _ in range(times):
        s = np.zeros_like(z)
        s[1:, :] += z[:-1, :]
        s[:-1, :] += z[1:, :]
        s[:, 1:] += z[:, :-1]
        s[:, :-1] += z[:, 1:]
        z = s / cnt
    return z


def boundary(points, values, n, L, M, q, smooth=5):
    """Boundary depth on the (n+1) x (n+1) lateral vertex lattice of an
    L x L domain for the pool member (M, q)."""
    c = np.linspace(0.0, L, n + 1)
    X, Y = np.meshgrid(c, c, indexing="ij")
    return laplace_smooth(idw(points, values, X, Y, M, q), smooth)


def pool(points, values, n, L, smooth=5):
    """The 2000-member pool: list of ((M, q), boundary) for M in M_VALUES, q in Q_VALUES."""
    return [((M, q), boundary(points, values, n, L, M, q, smooth)) for M in M_VALUES for q in Q_VALUES]


def select_varied(members, reference, n_keep):
    """Indices of the ``n_keep`` members whose boundary differs most (RMS)
    from ``reference``, in decreasing order of that difference."""
    rms = np.array([np.sqrt(np.mean((b - reference) ** 2)) for _, b in members])
    order = np.lexsort((np.arange(rms.size), -rms))
    return order[:n_keep], rms


def candidate_config(points, values, M, q, n=24, L=600.0, depth=50.0, n_soft=4, n_hard=4, n_steps=2000,
                     direction=0):
    """A two-layer workload (the paper's first/second layers, config-1
    materials) whose interface is the pool member (M, q); lateral n x n cells
    over L x L, n_soft + n_hard levels down to ``depth``; sin^2 basis pulse
    (T_p = 0.4 s), dt = 0.01 s; 25 receivers on a 5 x 5 grid."""
    from .configs import MAT_TWO_LAYER, grid_receivers
    from .waves import sin2_pulse

    itf = boundary(points, values, n, L, M, q)
    mesh = layered_box(n, n, L, L, [n_soft, n_hard], [itf], depth)
    dt = 0.01
    t = dt * np.arange(1, n_steps + 1)
    step = L / 5.0
    return dict(mesh=mesh, mat=MAT_TWO_LAYER.copy(), dt=dt, n_steps=n_steps, band=(0.5, 5.0),
                p=sin2_pulse(t, 0.4), dir=direction, rec_xy=grid_receivers(step / 2, step, 5),
                name="IDW candidate M=%d q=%.1f (%dx%d cells)" % (M, q, n, n))
