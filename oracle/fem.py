"""Element, face and assembled operators of the discretised Eq. (1) (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Discretisation (Section 2, Eq. (1); Section 3, computational-cost paragraph):
linear isotropic elasticity, c_ijkl = lambda d_ij d_kl + mu (d_ik d_jl +
d_il d_jk), on straight-sided 10-node tetrahedra with the standard quadratic
Lagrange shape functions in barycentric coordinates L_1..L_4:

    vertex a:        N_a  = L_a (2 L_a - 1)
    edge (a, b):     N_ab = 4 L_a L_b

DOF numbering is node-major: dof = 3 * node + component.

Readings of points the paper leaves open (each applied identically here and
in the GPU library):

* mass matrix: consistent (exactly integrated);
* damping: Rayleigh, C_e = alpha_e M_e + beta_e K_e, with (alpha, beta) the
  least-squares fit of alpha/(4 pi f) + beta pi f to the layer's damping
  ratio h over a frequency band;
* absorbing boundary (Section 2, boundary-condition sentence): Lysmer
  viscous dashpots, traction -(rho Vp v_n n + rho Vs v_t), on base and side
  faces, with the adjacent element's material;
* input (Section 2, external-force sentence): force 2 C_base (v_in e_j) on
  the base, so a homogeneous half-space doubles at the free surface.
"""
from math import factorial

import numpy as np
import scipy.integrate as si
import scipy.sparse as sp

TET_EDGES = ((0, 1), (1, 2), (0, 2), (0, 3), (1, 3), (2, 3))
TRI_EDGES = ((0, 1), (1, 2), (2, 0))

# ----------------------------------------------------------------------------
# Polynomials in barycentric coordinates: dict {exponent tuple: coefficient}
# ----------------------------------------------------------------------------


def _pmul(p, q):
    out = {}
    for ea, ca in p.items():
        for eb, cb in q.items():
            e = tuple(x + y for x, y in zip(ea, eb))
            out[e] = out.get(e, 0.0) + ca * cb
    return out


def _mono(n, idx, power=1):
    e = [0] * n
    e[idx] = power
    return {tuple(e): 1.0}


def _quadratic_shapes(n_vert, edges):
    """Quadratic Lagrange shape functions as homogeneous degree-2 polynomials.

    L_a (2 L_a - 1) is made homogeneous with sum_k L_k = 1:
    L_a (2 L_a - sum_k L_k).
    """
    shapes = []
    for a in range(n_vert):
        s = {}
        for k in range(n_vert):
            term = _pmul(_mono(n_vert, a), _mono(n_vert, k))
            for e, c in term.items():
                s[e] = s.get(e, 0.0) - c
        e2 = [0] * n_vert
        e2[a] = 2
        s[tuple(e2)] = s.get(tuple(e2), 0.0) + 2.0
        shapes.append(s)
    for (a, b) in edges:
        shapes.append({k: 4.0 * v for k, v in _pmul(_mono(n_vert, a), _mono(n_vert, b)).items()})
    return shapes


def _integrate_simplex(poly, dim):
    """Integral over a simplex of unit measure of a barycentric polynomial.

    Exact formula: int L_1^a1 ... L_n^an d(measure) =
    measure * dim! * a1! ... an! / (a1 + ... + an + dim)!.
    """
    tot = 0.0
    for e, c in poly.items():
        num = factorial(dim)
        for x in e:
            num *= factorial(x)
        tot += c * num / factorial(sum(e) + dim)
    return tot


def reference_mass_tet():
    """10x10 matrix int N_a N_b dV / V for the quadratic tetrahedron."""
    N = _quadratic_shapes(4, TET_EDGES)
    return np.array([[_integrate_simplex(_pmul(N[a], N[b]), 3) for b in range(10)] for a in range(10)])


def reference_mass_tri():
    """6x6 matrix int N_a N_b dA / A for the quadratic triangle."""
    N = _quadratic_shapes(3, TRI_EDGES)
    return np.array([[_integrate_simplex(_pmul(N[a], N[b]), 2) for b in range(6)] for a in range(6)])


def reference_load_tri():
    """6-vector int N_a dA / A for the quadratic triangle."""
    N = _quadratic_shapes(3, TRI_EDGES)
    return np.array([_integrate_simplex(N[a], 2) for a in range(6)])


# ----------------------------------------------------------------------------
# Geometry
# ----------------------------------------------------------------------------


def _unwrap(X, period):
    """Shift vertex coordinates by whole periods to the image nearest vertex 0."""
    X = X.copy()
    for d in range(2):
        P = period[d]
        if P > 0:
            dx = X[:, :, d] - X[:, :1, d]
            X[:, :, d] -= P * np.round(dx / P)
    return X


def tet_geometry(xyz, conn, period=(0.0, 0.0)):
    """Barycentric gradients [E,4,3] and volumes [E] of affine tetrahedra.

    With J = [x1 - x0, x2 - x0, x3 - x0] (columns), L_1..L_3 = J^{-1}(x - x0),
    so grad L_k (k = 1..3) are the rows of J^{-1} and grad L_0 = -sum.
    """
    X = _unwrap(xyz[conn[:, :4]], period)
    J = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], axis=2)
    V = np.linalg.det(J) / 6.0
    Jinv = np.linalg.inv(J)
    g = np.zeros((conn.shape[0], 4, 3))
    g[:, 1:] = Jinv
    g[:, 0] = -Jinv.sum(axis=1)
    return g, V


def lame(mat):
    """(lambda, mu, rho) from rows (Vp, Vs, rho, h)."""
    Vp, Vs, rho = mat[:, 0], mat[:, 1], mat[:, 2]
    mu = rho * Vs ** 2
    lam = rho * Vp ** 2 - 2.0 * mu
    return lam, mu, rho


# ----------------------------------------------------------------------------
# Element matrices
# ----------------------------------------------------------------------------

_GAUSS_A = (5.0 + 3.0 * np.sqrt(5.0)) / 20.0
_GAUSS_B = (5.0 - np.sqrt(5.0)) / 20.0
GAUSS4 = np.array([[_GAUSS_A if i == q else _GAUSS_B for i in range(4)] for q in range(4)])


def shape_gradients(L, g):
    """Gradients [E,10,3] of the 10 quadratic shape functions at barycentric L.

    grad N_a = (4 L_a - 1) grad L_a;  grad N_ab = 4 (L_a grad L_b + L_b grad L_a).
    """
    E = g.shape[0]
    dN = np.zeros((E, 10, 3))
    for a in range(4):
        dN[:, a] = (4.0 * L[a] - 1.0) * g[:, a]
    for m, (a, b) in enumerate(TET_EDGES):
        dN[:, 4 + m] = 4.0 * (L[a] * g[:, b] + L[b] * g[:, a])
    return dN


def strain_matrix(dN):
    """Voigt B [E,6,30] (strains xx, yy, zz, 2yz, 2xz, 2xy)."""
    E = dN.shape[0]
    B = np.zeros((E, 6, 30))
    gx, gy, gz = dN[..., 0], dN[..., 1], dN[..., 2]
    B[:, 0, 0::3] = gx
    B[:, 1, 1::3] = gy
    B[:, 2, 2::3] = gz
    B[:, 3, 1::3] = gz
    B[:, 3, 2::3] = gy
    B[:, 4, 0::3] = gz
    B[:, 4, 2::3] = gx
    B[:, 5, 0::3] = gy
    B[:, 5, 1::3] = gx
    return B


def elasticity_voigt(lam, mu):
    """Isotropic D [E,6,6] in Voigt notation with engineering shear strains."""
    E = lam.shape[0]
    D = np.zeros((E, 6, 6))
    D[:, :3, :3] = lam[:, None, None]
    for i in range(3):
        D[:, i, i] += 2.0 * mu
        D[:, 3 + i, 3 + i] = mu
    return D


def element_stiffness(g, V, lam, mu):
    """K_e [E,30,30] = int B^T D B dV by the 4-point degree-2 Gauss rule.

    The integrand is quadratic for affine quadratic tetrahedra, so the rule
    is exact.
    """
    D = elasticity_voigt(lam, mu)
    K = np.zeros((g.shape[0], 30, 30))
    for q in range(4):
        B = strain_matrix(shape_gradients(GAUSS4[q], g))
        K += np.einsum("eji,ejk,ekl->eil", B, D, B) * (V / 4.0)[:, None, None]
    return K


def element_mass(V, rho):
    """M_e [E,30,30] = rho int N_a N_b dV (x) I_3, exactly integrated."""
    Mref = np.kron(reference_mass_tet(), np.eye(3))
    return (rho * V)[:, None, None] * Mref[None]


# ----------------------------------------------------------------------------
# Rayleigh damping fit
# ----------------------------------------------------------------------------


def rayleigh_fit(h, f1, f2):
    """Least-squares (alpha, beta) of zeta(f) = alpha/(4 pi f) + beta pi f ~ h on [f1, f2].

    Normal equations of min int (alpha phi1 + beta phi2 - h)^2 df with
    phi1 = 1/(4 pi f), phi2 = pi f, integrals by adaptive quadrature.
    """
    phi = [lambda f: 1.0 / (4.0 * np.pi * f), lambda f: np.pi * f]
    G = np.array([[si.quad(lambda f: phi[i](f) * phi[j](f), f1, f2, epsabs=0, epsrel=1e-13)[0]
                   for j in range(2)] for i in range(2)])
    r = np.array([si.quad(phi[i], f1, f2, epsabs=0, epsrel=1e-13)[0] for i in range(2)])
    return np.linalg.solve(G, h * r)


# ----------------------------------------------------------------------------
# Boundary faces
# ----------------------------------------------------------------------------


def face_geometry(xyz, faces, period=(0.0, 0.0)):
    """Areas [F] and unit normals [F,3] (orientation irrelevant) of flat 6-node faces."""
    X = _unwrap(xyz[faces[:, :3]], period)
    cr = np.cross(X[:, 1] - X[:, 0], X[:, 2] - X[:, 0])
    nrm = np.linalg.norm(cr, axis=1)
    return 0.5 * nrm, cr / nrm[:, None]


def dashpot_faces(xyz, faces, face_elem, elem_mat, mat, period=(0.0, 0.0)):
    """Per-face 18x18 Lysmer dashpot matrices.

    C_face[3a+c, 3b+d] = int N_a N_b dA * T[c, d] with
    T = rho Vp n n^T + rho Vs (I - n n^T) of the adjacent element's layer.
    """
    A, n = face_geometry(xyz, faces, period)
    m = elem_mat[face_elem]
    rho, Vp, Vs = mat[m, 2], mat[m, 0], mat[m, 1]
    nn = n[:, :, None] * n[:, None, :]
    T = (rho * Vp)[:, None, None] * nn + (rho * Vs)[:, None, None] * (np.eye(3)[None] - nn)
    Mtri = reference_mass_tri()
    return A[:, None, None, None, None] * Mtri[None, :, None, :, None] * T[:, None, :, None, :]


# ----------------------------------------------------------------------------
# Assembly
# ----------------------------------------------------------------------------


def _assemble(blocks, nodes, n_dof):
    """Sum element blocks [E, n*3, n*3] into a CSR matrix over node lists [E, n].

    An empty block list (E = 0, e.g. a mesh with no absorbing faces) sums to
    the zero matrix."""
    if nodes.shape[0] == 0:
        return sp.csr_matrix((n_dof, n_dof))
    dofs = (3 * nodes[:, :, None] + np.arange(3)[None, None, :]).reshape(nodes.shape[0], -1)
    k = dofs.shape[1]
    rows = np.repeat(dofs, k, axis=1).ravel()
    cols = np.tile(dofs, (1, k)).ravel()
    return sp.coo_matrix((blocks.reshape(-1), (rows, cols)), shape=(n_dof, n_dof)).tocsr()


def assemble(model, mat, band, chunk=20000):
    """Assembled CSR operators of one model.

    ``model``: mesh dict (xyz, conn, elem_mat, faces, face_elem, face_tag,
    period).  ``mat``: [n_mat, 4] rows (Vp, Vs, rho, h).  ``band``: (f1, f2)
    of the Rayleigh fit.

    Returns a dict with K, M, CR (Rayleigh), Cabs (base + side dashpots),
    Cbase (base dashpots only), w (float64 [3, n_dof]: w[j] = Cbase applied
    to the uniform unit velocity field in direction j) and the fitted
    (alpha, beta) per material.
    """
    xyz, conn, em = model["xyz"], model["conn"].astype(np.int64), model["elem_mat"]
    period = model.get("period", (0.0, 0.0))
    n_dof = 3 * xyz.shape[0]
    lam_m, mu_m, rho_m = lame(mat)
    ab = np.array([rayleigh_fit(h, band[0], band[1]) for h in mat[:, 3]])
    K = sp.csr_matrix((n_dof, n_dof))
    M = sp.csr_matrix((n_dof, n_dof))
    CR = sp.csr_matrix((n_dof, n_dof))
    for s in range(0, conn.shape[0], chunk):
        c = conn[s:s + chunk]
        e_m = em[s:s + chunk]
        g, V = tet_geometry(xyz, c, period)
        Ke = element_stiffness(g, V, lam_m[e_m], mu_m[e_m])
        Me = element_mass(V, rho_m[e_m])
        K = K + _assemble(Ke, c, n_dof)
        M = M + _assemble(Me, c, n_dof)
        CR = CR + _assemble(ab[e_m, 0][:, None, None] * Me + ab[e_m, 1][:, None, None] * Ke, c, n_dof)
    faces = model["faces"].astype(np.int64)
    tag = model["face_tag"]
    absorb = tag != 0
    Cf = dashpot_faces(xyz, faces[absorb], model["face_elem"][absorb], em, mat, period)
    Cabs = _assemble(Cf.reshape(-1, 18, 18), faces[absorb], n_dof)
    isbase = tag[absorb] == 1
    Cbase = _assemble(Cf[isbase].reshape(-1, 18, 18), faces[absorb][isbase], n_dof)
    w = np.zeros((3, n_dof))
    for j in range(3):
        unit = np.zeros(n_dof)
        unit[j::3] = 1.0
        w[j] = Cbase @ unit
    return dict(K=K, M=M, CR=CR, Cabs=Cabs, Cbase=Cbase, w=w, rayleigh=ab)


# ----------------------------------------------------------------------------
# Receivers
# ----------------------------------------------------------------------------


def receiver_weights(model, rec_xy):
    """Nodes [R,6] and weights [R,6] interpolating the free surface at (x1, x2).

    The containing top-surface triangle is found by brute force (barycentric
    coordinates of the horizontal projection all >= -1e-10); the weights are
    the 6-node triangle's quadratic shape functions there.
    """
    xyz = model["xyz"]
    top = model["faces"][model["face_tag"] == 0].astype(np.int64)
    period = model.get("period", (0.0, 0.0))
    X = _unwrap(xyz[top[:, :3]], period)[:, :, :2]
    nodes = np.zeros((rec_xy.shape[0], 6), dtype=np.int64)
    wts = np.zeros((rec_xy.shape[0], 6))
    for r, pt in enumerate(rec_xy):
        found = False
        for f in range(top.shape[0]):
            T = np.stack([X[f, 1] - X[f, 0], X[f, 2] - X[f, 0]], axis=1)
            l12 = np.linalg.solve(T, pt - X[f, 0])
            L = np.array([1.0 - l12.sum(), l12[0], l12[1]])
            if np.all(L >= -1e-10):
                N = [L[a] * (2 * L[a] - 1) for a in range(3)] + [4 * L[a] * L[b] for (a, b) in TRI_EDGES]
                nodes[r] = top[f]
                wts[r] = N
                found = True
                break
        if not found:
            raise ValueError("receiver %d at %s is not on the free surface" % (r, pt))
    return nodes, wts
