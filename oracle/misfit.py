"""Input-wave estimation, misfit ERR and model selection (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Section 2: the input velocity is f_j(t) = sum_l c_jl p(t - (l-1) Dt_p); by
linearity and time invariance the response at observation point k in
direction i is U^k_i(t) = sum_j sum_l G^k_ij(t - (l-1) Dt_p) c_jl, with
G^k_ij the response to p(t) input in direction j.  With Dt_p = s dt (s
whole time steps) and the system at rest before t = 0, a shift by l strides
is a shift of the sampled record by l s samples (zero before the start).

Readings (the paper states ERR, Eq. (2), and that c follows from A c = b
solved with a truncated SVD pseudo-inverse):

* A, b are the normal equations of the weighted least-squares problem
  min_c sum_{k,i} w_ki sum_n (U^k_i[n] - obs^k_i[n])^2,
  w_ki = 1 / sum_n obs^k_i[n]^2 (the denominators of Eq. (2), squared);
* pairs (k, i) with sum obs^2 < 1e-12 * max_(k,i) sum obs^2 are dropped and
  n_obs counts the kept pairs (Eq. (2) divides by their energy);
* A is symmetric positive semi-definite, so its SVD is its eigen
  decomposition; eigenvalues below tau * lambda_max are discarded;
* the time integrals of Eq. (2) are sums over the recorded samples (dt
  cancels in the ratio).
"""
import numpy as np


def design(G, s, L):
    """Shifted design matrices Phi [n_rec, 3(i), n_t, 3 L] from G [n_rec, 3(i), 3(j), n_t].

    Phi[k, i, n, j L + l] = G[k, i, j, n - l s] (0 where n - l s < 0).
    """
    n_rec, _, _, n_t = G.shape
    Phi = np.zeros((n_rec, 3, n_t, 3 * L))
    for j in range(3):
        for l in range(L):
            sh = l * s
            if sh < n_t:
                Phi[:, :, sh:, j * L + l] = G[:, :, j, :n_t - sh]
    return Phi


def kept_pairs(obs, drop=1e-12):
    energy = (obs ** 2).sum(axis=-1)
    return energy >= drop * energy.max(), energy


def normal_equations(G, obs, s, L, drop=1e-12):
    """A [3L, 3L] and b [3L] of the weighted least-squares input estimate."""
    Phi = design(G, s, L)
    keep, energy = kept_pairs(obs, drop)
    A = np.zeros((3 * L, 3 * L))
    b = np.zeros(3 * L)
    for k in range(G.shape[0]):
        for i in range(3):
            if keep[k, i]:
                w = 1.0 / energy[k, i]
                A += w * Phi[k, i].T @ Phi[k, i]
                b += w * Phi[k, i].T @ obs[k, i]
    return A, b


def pinv_sym(A, tau):
    """Truncated pseudo-inverse of a symmetric PSD matrix via its eigenvectors."""
    lam, V = np.linalg.eigh(A)
    lmax = lam.max()
    inv = np.where(lam >= tau * lmax, 1.0 / np.where(lam > 0, lam, 1.0), 0.0) if lmax > 0 else np.zeros_like(lam)
    return (V * inv[None, :]) @ V.T


def superpose(G, c, s):
    """U [n_rec, 3, n_t] = sum_j sum_l G[:, :, j, n - l s] c[j, l]."""
    L = c.shape[1]
    n_t = G.shape[-1]
    U = np.zeros((G.shape[0], 3, n_t))
    for j in range(3):
        for l in range(L):
            sh = l * s
            if sh < n_t:
                U[:, :, sh:] += c[j, l] * G[:, :, j, :n_t - sh]
    return U


def err(U, obs, drop=1e-12):
    """Eq. (2): mean over kept (k, i) of sqrt(sum (U - obs)^2) / sqrt(sum obs^2)."""
    keep, energy = kept_pairs(obs, drop)
    num = np.sqrt(((U - obs) ** 2).sum(axis=-1))
    return float((num[keep] / np.sqrt(energy[keep])).mean())


def estimate(G, obs, s, L, tau=1e-10, drop=1e-12):
    """(ERR, c [3, L]) for one candidate's Green's functions and one event."""
    A, b = normal_equations(G, obs, s, L, drop)
    c = (pinv_sym(A, tau) @ b).reshape(3, L)
    return err(superpose(G, c, s), obs, drop), c


def select(ERR):
    """Model selection from ERR [n_models, n_events].

    Returns (best per event, best by historical maximum after each event):
    argmin_l ERR[l, e] and argmin_l max_{e' <= e} ERR[l, e'], ties to the
    lowest model index.
    """
    ERR = np.asarray(ERR)
    per_event = np.argmin(ERR, axis=0)
    hist = np.maximum.accumulate(ERR, axis=1)
    return per_event, np.argmin(hist, axis=0)
