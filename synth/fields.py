"""Seeded 2D Gaussian random fields for layer-interface depths.

Spectral synthesis on a regular lattice: white noise is filtered in the
Fourier domain by the square root of the spectral density of the Gaussian
covariance exp(-r^2 / ell^2), on a zero-padded periodic grid so the result
is not itself periodic, then cropped and normalised to zero mean and unit
sample variance.
"""
import numpy as np


def grf2d(n1, n2, h, ell, rng):
    """Unit Gaussian random field on an ``n1`` x ``n2`` lattice of spacing ``h``.

    ``ell`` is the correlation length (metres) of the covariance
    exp(-r^2/ell^2); ``rng`` is a ``numpy.random.Generator``.
    """
    pad = int(np.ceil(3.0 * ell / h))
    m1 = int(2 ** np.ceil(np.log2(n1 + pad)))
    m2 = int(2 ** np.ceil(np.log2(n2 + pad)))
    w = rng.standard_normal((m1, m2))
    k1 = 2 * np.pi * np.fft.fftfreq(m1, d=h)
    k2 = 2 * np.pi * np.fft.fftfreq(m2, d=h)
    K2 = k1[:, None] ** 2 + k2[None, :] ** 2
    filt = np.exp(-K2 * ell * ell / 8.0)  # sqrt of exp(-k^2 ell^2 / 4)
    g = np.real(np.fft.ifft2(np.fft.fft2(w) * filt))[:n1, :n2]
    g = g - g.mean()
    s = g.std()
    return g / s if s > 0 else g
