"""Two-level (first-order coarse level) preconditioner of the inner solve (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Section 3 (computational-cost paragraph) says the CG solver follows the
authors' earlier GPU solver, a variable preconditioner whose inner solves
run partly on a coarser, first-order mesh.  The coarse level here is the
4-node (linear) tetrahedral mesh on the same vertices:

* prolongation P from vertex values to the quadratic nodes: a vertex node
  takes its vertex's value, a mid-edge node the mean of its edge's two
  vertices (the quadratic interpolant of the piecewise-linear field, exact
  for straight-sided elements);
* coarse operator A_c = P^T A P (on straight-sided elements this is the
  linear-element operator: the linear hat function of a vertex equals
  N_a + 1/2 sum of N_ab over its edges);
* coarse smoother: the inverted 3x3 nodal diagonal blocks D_c of A_c;
* additive combination with the fine block-Jacobi D:

      z = D^-1 r + omega P D_c^-1 P^T r

  a fixed symmetric positive-definite operator (so the inner PCG stays a
  standard PCG).

The choice of the additive form, one coarse block-Jacobi sweep and the
weight omega are readings of the paper's one-sentence description; the
paper gives no formula.
"""
import numpy as np
import scipy.sparse as sp

from . import fem, newmark


def vertices(conn):
    """Sorted fine node ids of the vertices (first four nodes of each element)."""
    return np.unique(np.asarray(conn)[:, :4])


def prolongation(conn, n_nodes):
    """P [3 n_nodes, 3 n_vert] (CSR) and the vertex node ids.

    Column block j is vertex verts[j]; a vertex node's row is the identity of
    its own column block, a mid-edge node's row 1/2 on each endpoint's block."""
    conn = np.asarray(conn, dtype=np.int64)
    verts = vertices(conn)
    vid = -np.ones(n_nodes, dtype=np.int64)
    vid[verts] = np.arange(verts.size)
    parent = {}
    for e in range(conn.shape[0]):
        for k, (a, b) in enumerate(fem.TET_EDGES):
            parent.setdefault(int(conn[e, 4 + k]), (int(conn[e, a]), int(conn[e, b])))
    rows, cols, vals = [], [], []
    for v in verts:
        for c in range(3):
            rows.append(3 * v + c)
            cols.append(3 * vid[v] + c)
            vals.append(1.0)
    for m, (a, b) in parent.items():
        if vid[m] >= 0:
            continue  # a node that is both a vertex and a mid-edge node: not a valid mesh
        for c in range(3):
            for e in (a, b):
                rows.append(3 * m + c)
                cols.append(3 * vid[e] + c)
                vals.append(0.5)
    P = sp.csr_matrix((vals, (rows, cols)), shape=(3 * n_nodes, 3 * verts.size))
    return P, verts


def coarse_operator(A, P):
    """A_c = P^T A P (CSR)."""
    return (P.T @ A @ P).tocsr()


def coarse_inverse_blocks(A, P):
    """Inverses [n_vert, 3, 3] of A_c's 3x3 nodal diagonal blocks."""
    return newmark.block_jacobi_inverse(coarse_operator(A, P))


def block_apply(Dinv, r):
    """Apply inverted nodal 3x3 blocks [n, 3, 3] to a node-major vector."""
    return np.einsum("nij,nj->ni", Dinv, r.reshape(-1, 3)).ravel()


def coarse_correction(P, Dc_inv, r):
    """P D_c^-1 P^T r."""
    return P @ block_apply(Dc_inv, P.T @ r)


def apply(Dinv, P, Dc_inv, omega, r):
    """z = D^-1 r + omega P D_c^-1 P^T r."""
    return block_apply(Dinv, r) + omega * coarse_correction(P, Dc_inv, r)


def pcg(A, b, precond, tol, max_iter):
    """Textbook PCG from x = 0 with a fixed preconditioner callable.

    Returns (x, iterations, final ||r|| / ||b||)."""
    bn = np.linalg.norm(b)
    x = np.zeros_like(b)
    if bn == 0.0:
        return x, 0, 0.0
    r = b.copy()
    z = precond(r)
    p = z.copy()
    rz = r @ z
    for k in range(1, max_iter + 1):
        q = A @ p
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        rel = np.linalg.norm(r) / bn
        if rel <= tol:
            return x, k, rel
        z = precond(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, max_iter, np.linalg.norm(r) / bn
