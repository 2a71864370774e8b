"""Closed-form 1D layered transfer function (oracle pin for vertical incidence).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

A plane wave at vertical incidence through horizontal layers over the
absorbing base is one-dimensional: with z pointing down from the free
surface and time dependence exp(i w t), each layer with Rayleigh damping
(alpha M + beta K) has complex modulus G* = G (1 + i w beta), complex
density rho* = rho (1 - i alpha / w) and wavenumber k = w sqrt(rho*/G*)
(G = mu for S waves, lambda + 2 mu for P waves).  Starting from unit
displacement and zero stress at the surface, the layer transfer matrix
propagates (U, tau) to the base:

    U'   =  U cos kH + tau sin kH / (G* k)
    tau' = -U G* k sin kH + tau cos kH.

The base dashpot with impedance Z = rho_b V_b driven by 2 Z v_in gives
tau_D = i w Z (2 U_in - U_D), hence surface/incident
H(w) = 2 / (U_D + tau_D / (i w Z)).  For a homogeneous column of depth D,
H = 2 exp(-i w D / V): the incident wave delayed by D / V and doubled.
"""
import numpy as np


def transfer(freqs, layers, Z_base):
    """H(f) for ``layers`` = [(H, rho, G, alpha, beta), ...] top to bottom."""
    w = 2.0 * np.pi * np.asarray(freqs, dtype=np.float64)
    out = np.zeros(w.shape, dtype=np.complex128)
    for n, om in enumerate(w):
        if om == 0.0:
            out[n] = 2.0
            continue
        U, tau = 1.0 + 0j, 0.0 + 0j
        for (H, rho, G, alpha, beta) in layers:
            Gs = G * (1.0 + 1j * om * beta)
            rs = rho * (1.0 - 1j * alpha / om)
            k = om * np.sqrt(rs / Gs)
            c, s = np.cos(k * H), np.sin(k * H)
            U, tau = U * c + tau * s / (Gs * k), -U * Gs * k * s + tau * c
        out[n] = 2.0 / (U + tau / (1j * om * Z_base))
    return out


def surface_response(v_in, dt, layers, Z_base, pad=8):
    """Surface velocity for input velocity samples ``v_in`` (zero-padded FFT)."""
    n = len(v_in)
    nf = pad * n
    V = np.fft.rfft(v_in, n=nf)
    f = np.fft.rfftfreq(nf, d=dt)
    return np.fft.irfft(V * transfer(f, layers, Z_base), n=nf)[:n]
