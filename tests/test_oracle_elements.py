"""Pins of the oracle's element, face and assembled operators (CPU only).

Each check compares the oracle against something other than itself: the
closed-form quadratic-tetrahedron and -triangle mass patterns, the rigid-body
null space of elasticity, patch tests (exact reproduction of linear and
quadratic displacement fields), closed-form Rayleigh-fit integrals and
closed-form boundary integrals.
"""
import numpy as np
import pytest

from oracle import fem
from synth import configs
from synth.mesh import layered_box

EDGES = fem.TET_EDGES


def closed_form_tet_mass_pattern():
    """420/(rho V) * M_e for the quadratic tetrahedron (textbook pattern)."""
    P = np.zeros((10, 10))
    for a in range(4):
        for b in range(4):
            P[a, b] = 6.0 if a == b else 1.0
        for m, e in enumerate(EDGES):
            P[a, 4 + m] = P[4 + m, a] = -4.0 if a in e else -6.0
    for m, e in enumerate(EDGES):
        for n, f in enumerate(EDGES):
            if m == n:
                P[4 + m, 4 + n] = 32.0
            elif set(e) & set(f):
                P[4 + m, 4 + n] = 16.0
            else:
                P[4 + m, 4 + n] = 8.0
    return P


def test_tet_mass_closed_form():
    Mref = fem.reference_mass_tet()
    np.testing.assert_allclose(420.0 * Mref, closed_form_tet_mass_pattern(), atol=1e-12)
    rs = Mref.sum(axis=1)
    np.testing.assert_allclose(rs[:4], -1.0 / 20.0, atol=1e-15)
    np.testing.assert_allclose(rs[4:], 1.0 / 5.0, atol=1e-15)
    assert abs(Mref.sum() - 1.0) < 1e-14


def test_tri_mass_and_load_closed_form():
    P = np.zeros((6, 6))
    tri_edges = fem.TRI_EDGES
    for a in range(3):
        for b in range(3):
            P[a, b] = 6.0 if a == b else -1.0
        for m, e in enumerate(tri_edges):
            P[a, 3 + m] = P[3 + m, a] = 0.0 if a in e else -4.0
    for m in range(3):
        for n in range(3):
            P[3 + m, 3 + n] = 32.0 if m == n else 16.0
    np.testing.assert_allclose(180.0 * fem.reference_mass_tri(), P, atol=1e-12)
    np.testing.assert_allclose(fem.reference_load_tri(), [0, 0, 0, 1 / 3, 1 / 3, 1 / 3], atol=1e-15)


def _random_tets(n, seed=0):
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1, 1, size=(n, 4, 3)) * np.array([10.0, 7.0, 5.0])
    J = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], axis=2)
    neg = np.linalg.det(J) < 0
    X[neg] = X[neg][:, [0, 2, 1, 3]]
    xyz = np.zeros((n * 10, 3))
    conn = np.arange(n * 10).reshape(n, 10)
    xyz[conn[:, :4].ravel()] = X.reshape(-1, 3)
    for m, (a, b) in enumerate(EDGES):
        xyz[conn[:, 4 + m]] = 0.5 * (X[:, a] + X[:, b])
    return xyz, conn


def test_stiffness_symmetry_rank_and_rigid_modes():
    xyz, conn = _random_tets(5)
    g, V = fem.tet_geometry(xyz, conn)
    assert np.all(V > 0)
    lam = np.full(5, 2.0e9)
    mu = np.full(5, 7.0e8)
    K = fem.element_stiffness(g, V, lam, mu)
    for e in range(5):
        Ke = K[e]
        scale = np.abs(Ke).max()
        assert np.abs(Ke - Ke.T).max() < 1e-13 * scale
        ev = np.linalg.eigvalsh(Ke)
        assert np.sum(ev < 1e-10 * ev.max()) == 6, "rigid-body null space must be exactly 6-dimensional"
        assert ev.min() > -1e-10 * ev.max()
        X = xyz[conn[e]]
        modes = []
        for d in range(3):
            t = np.zeros((10, 3))
            t[:, d] = 1.0
            modes.append(t)
        for axis in np.eye(3):
            modes.append(np.cross(axis, X))
        for u in modes:
            assert np.abs(Ke @ u.ravel()).max() < 1e-11 * scale * np.abs(u).max()


def _interior_nodes(mesh):
    boundary = np.unique(mesh["faces"].ravel())
    return np.setdiff1d(np.arange(mesh["xyz"].shape[0]), boundary)


def test_patch_linear_field():
    """K u = 0 at interior nodes for any linear displacement on a distorted mesh."""
    cfg = configs.small_box(nx=4, ny=3, counts=(2, 2), distort=True)
    mesh = cfg["mesh"]
    mat = np.repeat(cfg["mat"][1:], 2, axis=0)  # one material, distorted layer geometry
    ops = fem.assemble(mesh, mat, cfg["band"])
    rng = np.random.default_rng(3)
    B = rng.standard_normal((3, 3)) * 1e-3
    u = (mesh["xyz"] @ B.T + rng.standard_normal(3)).ravel()
    f = (ops["K"] @ u).reshape(-1, 3)
    inner = _interior_nodes(mesh)
    scale = np.abs(ops["K"]).max() * np.abs(u).max()
    assert inner.size > 10
    assert np.abs(f[inner]).max() < 1e-12 * scale


def test_patch_quadratic_field_single_material():
    """Quadratic u: interior rows of K u equal the consistent load of -div(sigma).

    For u_i = x^T Q_i x (Q_i symmetric) the stress is linear, so
    b = -div(sigma) is constant and int N_a b dV = b * sum_e V_e * s_a with
    s_a = -1/20 (vertex) or 1/5 (edge), the row sums of the mass pattern.
    """
    mesh = layered_box(4, 3, 30.0, 20.0, [3], [], 18.0)
    mat = np.array([[1800.0, 500.0, 1900.0, 0.01]])
    ops = fem.assemble(mesh, mat, (0.5, 5.0))
    lam, mu, _ = fem.lame(mat)
    rng = np.random.default_rng(5)
    Q = rng.standard_normal((3, 3, 3))
    Q = 0.5 * (Q + Q.transpose(0, 2, 1)) * 1e-4
    x = mesh["xyz"]
    u = np.einsum("nj,ijk,nk->ni", x, Q, x).ravel()
    # grad u_i = 2 Q_i x ; d_j d_k u_i = 2 Q_i[j,k]
    H = 2.0 * Q  # second derivatives H[i, j, k]
    div_grad = np.einsum("ijj->i", H)           # d_j d_j u_i
    grad_div = np.einsum("jji->i", H)           # d_i d_j u_j
    body = -((lam[0] + mu[0]) * grad_div + mu[0] * div_grad)  # -div sigma
    # consistent load int N_a b dV = b * sum_e V_e s_a
    g, V = fem.tet_geometry(x, mesh["conn"])
    s = np.array([-1.0 / 20] * 4 + [1.0 / 5] * 6)
    weight = np.zeros(x.shape[0])
    np.add.at(weight, mesh["conn"].ravel(), (V[:, None] * s[None, :]).ravel())
    f = (ops["K"] @ u).reshape(-1, 3)
    inner = _interior_nodes(mesh)
    ref = weight[inner, None] * body[None, :]
    assert inner.size > 10
    np.testing.assert_allclose(f[inner], ref, atol=1e-9 * np.abs(ref).max())


def test_rayleigh_fit_closed_form_integrals():
    for h, f1, f2 in ((0.03, 0.5, 5.0), (0.01, 0.1, 2.5), (0.2, 1.0, 3.0)):
        a, b = fem.rayleigh_fit(h, f1, f2)
        pi = np.pi
        G = np.array([[(1 / f1 - 1 / f2) / (16 * pi ** 2), (f2 - f1) / 4.0],
                      [(f2 - f1) / 4.0, pi ** 2 * (f2 ** 3 - f1 ** 3) / 3.0]])
        r = np.array([np.log(f2 / f1) / (4 * pi), pi * (f2 ** 2 - f1 ** 2) / 2.0])
        ref = np.linalg.solve(G, h * r)
        np.testing.assert_allclose([a, b], ref, rtol=1e-10)


def test_dashpot_totals_and_base_load():
    cfg = configs.config1(n_steps=1)
    mesh, mat = cfg["mesh"], cfg["mat"]
    ops = fem.assemble(mesh, mat, cfg["band"])
    area = 100.0 * 100.0
    rho, Vp, Vs = mat[1, 2], mat[1, 0], mat[1, 1]
    w = ops["w"]
    np.testing.assert_allclose(w[0].sum(), rho * Vs * area, rtol=1e-13)
    np.testing.assert_allclose(w[1].sum(), rho * Vs * area, rtol=1e-13)
    np.testing.assert_allclose(w[2].sum(), rho * Vp * area, rtol=1e-13)
    # force acts only along the input direction
    assert np.abs(w[0][1::3]).max() == 0 and np.abs(w[0][2::3]).max() == 0
    # vertex nodes of base faces get no load (int N_vertex dA = 0)
    verts = np.unique(mesh["faces"][mesh["face_tag"] == 1][:, :3])
    assert np.abs(w[2][3 * verts + 2]).max() < 1e-6
    # absorbing matrix: symmetric, PSD, and the side + base totals for a uniform x-velocity
    C = ops["Cabs"]
    assert abs(C - C.T).max() < 1e-9 * abs(C).max()
    ux = np.zeros(C.shape[0])
    ux[0::3] = 1.0
    tot = ux @ (C @ ux)
    sides_x = 2 * (rho * Vp * 30 * 100 + mat[0, 2] * mat[0, 0] * 20 * 100)   # x-normal faces: P impedance
    sides_y = 2 * (rho * Vs * 30 * 100 + mat[0, 2] * mat[0, 1] * 20 * 100)   # y-normal faces: S impedance
    np.testing.assert_allclose(tot, rho * Vs * area + sides_x + sides_y, rtol=1e-12)


def test_mass_total_and_receiver_interpolation():
    cfg = configs.small_box(nx=4, ny=3, distort=True)
    mesh = cfg["mesh"]
    ops = fem.assemble(mesh, cfg["mat"], cfg["band"])
    g, V = fem.tet_geometry(mesh["xyz"], mesh["conn"])
    rho = cfg["mat"][mesh["elem_mat"], 2]
    ux = np.zeros(ops["M"].shape[0])
    ux[0::3] = 1.0
    np.testing.assert_allclose(ux @ (ops["M"] @ ux), (rho * V).sum(), rtol=1e-13)
    rng = np.random.default_rng(9)
    pts = np.stack([rng.uniform(0, 30, 7), rng.uniform(0, 20, 7)], axis=1)
    nodes, w = fem.receiver_weights(mesh, pts)
    np.testing.assert_allclose(w.sum(axis=1), 1.0, atol=1e-13)
    x = mesh["xyz"]
    fq = lambda X, Y: 1.0 + 0.3 * X - 0.2 * Y + 0.01 * X * X - 0.02 * X * Y + 0.03 * Y * Y
    vals = (w * fq(x[nodes, 0], x[nodes, 1])).sum(axis=1)
    np.testing.assert_allclose(vals, fq(pts[:, 0], pts[:, 1]), rtol=1e-12)


def test_assemble_without_absorbing_faces():
    """A mesh whose only boundary faces are free surface (tag 0): no dashpots, no
    base load, and K, M, C_R identical to those of the same mesh with its
    absorbing faces."""
    cfg = configs.small_box(nx=3, ny=2, distort=True)
    mesh = dict(cfg["mesh"])
    full = fem.assemble(mesh, cfg["mat"], cfg["band"])
    keep = mesh["face_tag"] == 0
    for key in ("faces", "face_elem", "face_tag"):
        mesh[key] = mesh[key][keep]
    assert mesh["faces"].shape[0] > 0 and (mesh["face_tag"] == 0).all()
    ops = fem.assemble(mesh, cfg["mat"], cfg["band"])
    n = 3 * mesh["xyz"].shape[0]
    for key in ("Cabs", "Cbase"):
        assert ops[key].shape == (n, n) and ops[key].nnz == 0
    assert np.abs(ops["w"]).max() == 0.0
    for key in ("K", "M", "CR"):
        assert abs(ops[key] - full[key]).max() == 0.0
    # and with no boundary faces at all
    for key in ("faces", "face_elem", "face_tag"):
        mesh[key] = mesh[key][:0]
    ops0 = fem.assemble(mesh, cfg["mat"], cfg["band"])
    assert ops0["Cabs"].nnz == 0 and abs(ops0["K"] - full["K"]).max() == 0.0
