"""Pins of the oracle's two-level inner preconditioner (CPU only).

The prolongation must reproduce affine displacement fields exactly (the
quadratic interpolant of a linear field); the coarse operator P^T A P of a
single straight-sided tetrahedron must be the textbook constant-strain
(4-node) tetrahedron: stiffness V B^T D B, consistent mass rho V / 20
(1 + delta_ab), and on an absorbing face the linear-triangle dashpot
(area / 12) (1 + delta_ab) T.  The combined preconditioner is symmetric
positive definite, and the PCG it drives reaches the direct solution.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spl

from oracle import fem, newmark, twolevel
from synth import configs

LAM, MU, RHO = 2.0e9, 1.2e9, 1900.0


def _vertex_gradients(X):
    """Gradients [4, 3] of the linear barycentric coordinates of a tetrahedron, and its volume."""
    T = np.hstack([np.ones((4, 1)), X])
    C = np.linalg.inv(T)  # L_a(x) = C[0, a] + C[1:, a] . x
    return C[1:, :].T, abs(np.linalg.det(T)) / 6.0


def _one_tet(face_tag=None, seed=0):
    rng = np.random.default_rng(seed)
    X = np.array([[0.0, 0.0, 0.0], [10.0, 0.0, 0.0], [0.0, 8.0, 0.0], [0.0, 0.0, 7.0]])  # positively oriented
    X = X + rng.uniform(-1.5, 1.5, size=X.shape)
    mids = [0.5 * (X[a] + X[b]) for a, b in fem.TET_EDGES]
    xyz = np.vstack([X, mids])
    conn = np.arange(10, dtype=np.int32)[None, :]
    if face_tag is None:
        faces = np.zeros((0, 6), dtype=np.int32)
        face_elem = np.zeros(0, dtype=np.int32)
        tags = np.zeros(0, dtype=np.int32)
    else:
        # face (0, 1, 2); its mid-edge nodes in the triangle edge order (0,1), (1,2), (2,0)
        faces = np.array([[0, 1, 2, 4, 5, 6]], dtype=np.int32)
        face_elem = np.zeros(1, dtype=np.int32)
        tags = np.array([face_tag], dtype=np.int32)
    mesh = dict(xyz=xyz, conn=conn, elem_mat=np.zeros(1, dtype=np.int32), faces=faces, face_elem=face_elem,
                face_tag=tags, period=np.zeros(2))
    Vs = np.sqrt(MU / RHO)
    Vp = np.sqrt((LAM + 2.0 * MU) / RHO)
    mat = np.array([[Vp, Vs, RHO, 0.0]])
    return mesh, mat, X


def test_prolongation_reproduces_affine_fields():
    mesh = configs.small_box(nx=4, ny=3)["mesh"]
    xyz = mesh["xyz"]
    P, verts = twolevel.prolongation(mesh["conn"], xyz.shape[0])
    rng = np.random.default_rng(1)
    B, c = rng.standard_normal((3, 3)), rng.standard_normal(3)
    u = xyz @ B.T + c  # an affine displacement field at every node
    np.testing.assert_allclose(P @ u[verts].ravel(), u.ravel(), rtol=0, atol=1e-11 * np.abs(u).max())
    # every quadratic node is covered, every row of P sums to one per component
    np.testing.assert_allclose(np.asarray(P.sum(axis=1)).ravel(), 1.0, atol=1e-15)


def test_coarse_operator_of_one_tet_is_the_linear_tet():
    mesh, mat, X = _one_tet()
    ops = fem.assemble(mesh, mat, (0.5, 5.0))
    P, verts = twolevel.prolongation(mesh["conn"], 10)
    assert list(verts) == [0, 1, 2, 3]
    g, V = _vertex_gradients(X)
    # constant-strain tetrahedron: B maps the 12 vertex DOF to the 6 Voigt strains
    Bm = np.zeros((6, 12))
    for a in range(4):
        gx, gy, gz = g[a]
        Bm[:, 3 * a:3 * a + 3] = [[gx, 0, 0], [0, gy, 0], [0, 0, gz], [gy, gx, 0], [0, gz, gy], [gz, 0, gx]]
    D = np.zeros((6, 6))
    D[:3, :3] = LAM
    D[range(3), range(3)] += 2.0 * MU
    D[range(3, 6), range(3, 6)] = MU
    K_lin = V * Bm.T @ D @ Bm
    Kc = twolevel.coarse_operator(ops["K"], P).toarray()
    np.testing.assert_allclose(Kc, K_lin, rtol=0, atol=1e-9 * np.abs(K_lin).max())
    M_lin = np.kron(RHO * V / 20.0 * (np.ones((4, 4)) + np.eye(4)), np.eye(3))
    Mc = twolevel.coarse_operator(ops["M"], P).toarray()
    np.testing.assert_allclose(Mc, M_lin, rtol=0, atol=1e-9 * np.abs(M_lin).max())


@pytest.mark.parametrize("tag", [1, 2])
def test_coarse_dashpot_of_one_face_is_the_linear_triangle(tag):
    mesh, mat, X = _one_tet(face_tag=tag, seed=3)
    ops = fem.assemble(mesh, mat, (0.5, 5.0))
    P, _ = twolevel.prolongation(mesh["conn"], 10)
    Cc = twolevel.coarse_operator(ops["Cabs"], P).toarray()
    n = np.cross(X[1] - X[0], X[2] - X[0])
    area = 0.5 * np.linalg.norm(n)
    n = n / np.linalg.norm(n)
    Vp, Vs = mat[0, 0], mat[0, 1]
    T = RHO * Vp * np.outer(n, n) + RHO * Vs * (np.eye(3) - np.outer(n, n))
    W = np.zeros((4, 4))
    W[:3, :3] = area / 12.0 * (np.ones((3, 3)) + np.eye(3))
    np.testing.assert_allclose(Cc, np.kron(W, T), rtol=0, atol=1e-9 * np.abs(T).max() * area)


@pytest.fixture(scope="module")
def box_system():
    cfg = configs.small_box(nx=4, ny=3)
    ops = fem.assemble(cfg["mesh"], cfg["mat"], cfg["band"])
    dt = cfg["dt"]
    A = (ops["K"] + (2.0 / dt) * (ops["CR"] + ops["Cabs"]) + (4.0 / dt ** 2) * ops["M"]).tocsr()
    P, _ = twolevel.prolongation(cfg["mesh"]["conn"], cfg["mesh"]["xyz"].shape[0])
    return A, P, newmark.block_jacobi_inverse(A), twolevel.coarse_inverse_blocks(A, P)


def test_preconditioner_is_symmetric_positive_definite(box_system):
    A, P, Dinv, Dc_inv = box_system
    rng = np.random.default_rng(2)
    x, y = rng.standard_normal((2, A.shape[0]))
    for omega in (0.0, 0.7):
        zx = twolevel.apply(Dinv, P, Dc_inv, omega, x)
        zy = twolevel.apply(Dinv, P, Dc_inv, omega, y)
        assert abs(y @ zx - x @ zy) <= 1e-12 * np.linalg.norm(zx) * np.linalg.norm(y)
        assert x @ zx > 0.0 and y @ zy > 0.0
    # omega = 0 is the fine block-Jacobi preconditioner alone
    np.testing.assert_allclose(twolevel.apply(Dinv, P, Dc_inv, 0.0, x), twolevel.block_apply(Dinv, x), rtol=1e-15)
    # the coarse blocks invert A_c's diagonal blocks
    Ac = twolevel.coarse_operator(A, P)
    base = 3 * np.arange(Dc_inv.shape[0])
    for v in (0, Dc_inv.shape[0] // 2, Dc_inv.shape[0] - 1):
        blk = Ac[base[v]:base[v] + 3, base[v]:base[v] + 3].toarray()
        np.testing.assert_allclose(Dc_inv[v] @ blk, np.eye(3), atol=1e-10)


def test_two_level_pcg_reaches_the_direct_solution_in_fewer_iterations(box_system):
    A, P, Dinv, Dc_inv = box_system
    b = np.random.default_rng(4).standard_normal(A.shape[0])
    x_ref = spl.spsolve(A.tocsc(), b)
    _, k1, _ = twolevel.pcg(A, b, lambda r: twolevel.block_apply(Dinv, r), 1e-10, 2000)
    x2, k2, rel = twolevel.pcg(A, b, lambda r: twolevel.apply(Dinv, P, Dc_inv, 0.7, r), 1e-10, 2000)
    assert rel <= 1e-10
    np.testing.assert_allclose(x2, x_ref, rtol=0, atol=1e-8 * np.abs(x_ref).max())
    assert k2 < k1
