"""Newmark time stepping and block-Jacobi PCG (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Time integration (Section 3, computational-cost paragraph: Newmark-beta,
implicit): the average-acceleration member, beta = 1/4, gamma = 1/2 (the
paper does not give the constants).  With A = K + (2/dt) C + (4/dt^2) M and
C = C_R + C_abs, each step solves

    A du = f_{n+1} - K u_n + C v_n + M (a_n + (4/dt) v_n)

and updates u_{n+1} = u_n + du, v_{n+1} = (2/dt) du - v_n,
a_{n+1} = (4/dt^2) du - (4/dt) v_n - a_n.

Linear solve (same paragraph: conjugate gradients with a preconditioner):
block-Jacobi PCG, the preconditioner being the inverted 3x3 nodal diagonal
blocks of A, started from the predictor du_0 = dt v_n + (dt^2 / 2) a_n and
stopped when the recursively updated residual satisfies
||r||_2 / ||b||_2 <= tol.  The GPU library runs the same algorithm.
"""
import numpy as np

from . import fem


class NoConvergence(RuntimeError):
    pass


def block_jacobi_inverse(A):
    """Inverses [N,3,3] of the 3x3 nodal diagonal blocks of a CSR matrix."""
    n = A.shape[0] // 3
    D = np.zeros((n, 3, 3))
    base = 3 * np.arange(n)
    for c1 in range(3):
        for c2 in range(3):
            D[:, c1, c2] = np.asarray(A[base + c1, base + c2]).ravel()
    return np.linalg.inv(D)


def pcg(A, b, x0, Dinv, tol, max_iter):
    """Block-Jacobi preconditioned CG.  Returns (x, iterations, final ||r||/||b||)."""
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return np.zeros_like(b), 0, 0.0
    x = x0.copy()
    r = b - A @ x
    rel = np.linalg.norm(r) / bn
    if rel <= tol:
        return x, 0, rel
    z = np.einsum("nij,nj->ni", Dinv, r.reshape(-1, 3)).ravel()
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
        z = np.einsum("nij,nj->ni", Dinv, r.reshape(-1, 3)).ravel()
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    raise NoConvergence("PCG did not reach %g in %d iterations (at %g)" % (tol, max_iter, rel))


def newmark_run(K, M, C, force, dt, n_steps, u0=None, v0=None, a0=None, tol=1e-12,
                max_iter=10000, observe=None):
    """Newmark average-acceleration run of M a + C v + K u = f(t).

    ``force(n)`` returns f_{n+1} (the load at t_{n+1}); ``observe(n, u, v, a)``
    is called after each step with the state at t_{n+1}.  Returns the final
    state and the per-step iteration counts.
    """
    n_dof = K.shape[0]
    u = np.zeros(n_dof) if u0 is None else u0.copy()
    v = np.zeros(n_dof) if v0 is None else v0.copy()
    a = np.zeros(n_dof) if a0 is None else a0.copy()
    A = (K + (2.0 / dt) * C + (4.0 / dt ** 2) * M).tocsr()
    Dinv = block_jacobi_inverse(A)
    iters = np.zeros(n_steps, dtype=np.int64)
    for n in range(n_steps):
        b = force(n) - K @ u + C @ v + M @ (a + (4.0 / dt) * v)
        x0 = dt * v + 0.5 * dt * dt * a
        du, iters[n], _ = pcg(A, b, x0, Dinv, tol, max_iter)
        u = u + du
        v_new = (2.0 / dt) * du - v
        a = (4.0 / dt ** 2) * du - (4.0 / dt) * v - a
        v = v_new
        if observe is not None:
            observe(n, u, v, a)
    return u, v, a, iters


def analysis(cfg, tol=1e-12, max_iter=10000, n_steps=None, ops=None):
    """One directional wave-propagation analysis of a synthetic workload.

    ``cfg``: dict from ``synth.configs`` (mesh, mat, dt, band, p, dir,
    rec_xy).  The base force of step n is 2 p[n] w_dir (w from
    :func:`oracle.fem.assemble`).  Returns a dict with ``wave``
    (float64 [n_rec, 3, n_steps], receiver velocity at t_{n+1}), ``iters``
    (CG iterations per step) and the final state.
    """
    mesh = cfg["mesh"]
    n_steps = cfg["n_steps"] if n_steps is None else n_steps
    dt = cfg["dt"]
    if ops is None:
        ops = fem.assemble(mesh, cfg["mat"], cfg["band"])
    rn, rw = fem.receiver_weights(mesh, cfg["rec_xy"])
    C = (ops["CR"] + ops["Cabs"]).tocsr()
    w = ops["w"][cfg["dir"]]
    p = cfg["p"]
    wave = np.zeros((rn.shape[0], 3, n_steps))

    def observe(n, u, v, a):
        vv = v.reshape(-1, 3)
        wave[:, :, n] = np.einsum("rk,rkc->rc", rw, vv[rn])

    u, v, a, iters = newmark_run(ops["K"], ops["M"], C, lambda n: 2.0 * p[n] * w, dt, n_steps,
                                 tol=tol, max_iter=max_iter, observe=observe)
    return dict(wave=wave, iters=iters, u=u, v=v, a=a)
