"""Input velocity wavelets (seeded where random).

All functions return velocity samples in m/s.  The input of time step n
(0-based) is the wavelet evaluated at t_{n+1} = (n+1) dt.
"""
import numpy as np


def ricker(t, f, t0, amp):
    """Ricker wavelet amp (1 - 2 pi^2 f^2 tau^2) exp(-pi^2 f^2 tau^2), tau = t - t0."""
    a = (np.pi * f * (np.asarray(t, dtype=np.float64) - t0)) ** 2
    return amp * (1.0 - 2.0 * a) * np.exp(-a)


def sin2_pulse(t, Tp):
    """Unit pulse sin^2(pi t / Tp) on [0, Tp], zero elsewhere."""
    t = np.asarray(t, dtype=np.float64)
    return np.where((t >= 0) & (t <= Tp), np.sin(np.pi * t / Tp) ** 2, 0.0)


def random_phase(n_steps, dt, rng, f_lo=0.1, f_pass_lo=0.2, f_pass_hi=2.3, f_hi=2.5,
                 n_fft=4096, t_window=10.0, peak=0.01):
    """Band-limited random-phase wavelet sampled at t_{n+1} = (n+1) dt.

    Amplitude spectrum 1 on [f_pass_lo, f_pass_hi] with cosine tapers to 0 at
    f_lo and f_hi; phases uniform on [0, 2 pi); inverse real FFT on ``n_fft``
    samples; Tukey (cosine-taper, 10 %) window over [0, t_window]; scaled to
    the given peak absolute value.
    """
    nfft = max(n_fft, n_steps + 1)
    f = np.fft.rfftfreq(nfft, d=dt)
    amp = np.zeros_like(f)
    band = (f >= f_pass_lo) & (f <= f_pass_hi)
    amp[band] = 1.0
    lo = (f >= f_lo) & (f < f_pass_lo)
    amp[lo] = 0.5 * (1 - np.cos(np.pi * (f[lo] - f_lo) / (f_pass_lo - f_lo)))
    hi = (f > f_pass_hi) & (f <= f_hi)
    amp[hi] = 0.5 * (1 + np.cos(np.pi * (f[hi] - f_pass_hi) / (f_hi - f_pass_hi)))
    ph = rng.uniform(0.0, 2 * np.pi, size=f.size)
    x = np.fft.irfft(amp * np.exp(1j * ph), n=nfft)
    t = np.arange(nfft) * dt
    win = np.zeros(nfft)
    inside = t <= t_window
    r = 0.1
    u = t[inside] / t_window
    w = np.ones_like(u)
    e1 = u < r / 2
    w[e1] = 0.5 * (1 + np.cos(2 * np.pi / r * (u[e1] - r / 2)))
    e2 = u > 1 - r / 2
    w[e2] = 0.5 * (1 + np.cos(2 * np.pi / r * (u[e2] - 1 + r / 2)))
    win[inside] = w
    x = x * win
    x = x * (peak / np.max(np.abs(x)))
    return x[1:n_steps + 1].copy()
