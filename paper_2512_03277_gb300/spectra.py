"""Linear spectra from trajectories (host-side analysis of cavmd_observables output).

The paper's molecular spectrum is I_m(w) ~ w^2 int_0^inf dt cos(w t) S[<mu_x(t) mu_x(0)>] and its
angle-resolved photonic spectrum uses the photon coordinate q_k in place of mu_x (Results); S is
a smoothing of the correlation function. Here S is a Hann window over the correlation time.
"""
from __future__ import annotations

import numpy as np

EV = 0.0367493   # Hartree per electron-volt


def autocorrelation(x: np.ndarray, max_lag: int | None = None) -> np.ndarray:
    """<x(t) x(0)> of a mean-removed series (unbiased over the available pairs), by FFT."""
    x = np.asarray(x, float)
    x = x - x.mean(axis=0)
    n = len(x)
    max_lag = n // 2 if max_lag is None else max_lag
    f = np.fft.rfft(x, 2 * n, axis=0)
    ac = np.fft.irfft(f * np.conj(f), axis=0)[:max_lag]
    counts = (n - np.arange(max_lag)).reshape((-1,) + (1,) * (x.ndim - 1))
    return ac / counts


def spectrum(x: np.ndarray, dt: float, max_lag: int | None = None, pad: int = 8):
    """(omega [Hartree], I(omega)) of a series sampled every dt (atomic units of time)."""
    return spectrum_from_acf(autocorrelation(x, max_lag), dt, pad)


def spectrum_from_acf(c: np.ndarray, dt: float, pad: int = 8):
    """(omega, I(omega)) from correlation functions c[lag, ...] sampled every dt, e.g. the
    device-accumulated ones of cavmd_autocorrelation (transposed to lag-major)."""
    c = np.asarray(c, float)
    n = len(c)
    w = 0.5 * (1.0 + np.cos(np.pi * np.arange(n) / n))          # Hann half-window
    c = c * w.reshape((-1,) + (1,) * (c.ndim - 1))
    m = pad * n
    omega = 2.0 * np.pi * np.fft.rfftfreq(2 * m, dt)
    # cosine transform of the even extension
    ext = np.concatenate([c, np.zeros((2 * m - 2 * n + 1,) + c.shape[1:]), c[:0:-1]], axis=0)
    I = np.fft.rfft(ext, axis=0).real
    return omega, (omega ** 2).reshape((-1,) + (1,) * (I.ndim - 1)) * I


def peaks(omega: np.ndarray, I: np.ndarray, lo: float, hi: float, n: int = 3) -> np.ndarray:
    """The n highest local maxima of I(omega) with lo < omega < hi, in increasing omega."""
    sel = np.where((omega > lo) & (omega < hi))[0]
    idx = [i for i in sel[1:-1] if I[i] > I[i - 1] and I[i] >= I[i + 1]]
    idx = sorted(idx, key=lambda i: -I[i])[:n]
    return np.sort(omega[idx])
