"""Host spectra tool: the autocorrelation equals the direct pair average, and the w^2-weighted
cosine transform puts its peaks at the frequencies of a sum of sinusoids."""
import numpy as np

from paper_2512_03277_gb300 import spectra as S


def test_autocorrelation_matches_direct_average():
    rng = np.random.default_rng(0)
    x = rng.normal(size=300)
    c = S.autocorrelation(x, 50)
    y = x - x.mean()
    direct = np.array([np.mean(y[:len(y) - k] * y[k:]) for k in range(50)])
    np.testing.assert_allclose(c, direct, rtol=1e-12, atol=1e-12)


def test_peaks_of_a_sum_of_sinusoids():
    dt = 20.0
    t = np.arange(20000) * dt
    w = np.array([0.0096, 0.0149, 0.0157])
    x = np.cos(w[0] * t) + 0.7 * np.sin(w[1] * t + 0.3) + 0.5 * np.cos(w[2] * t + 1.0)
    om, I = S.spectrum(x, dt)
    pk = S.peaks(om, I, 0.005, 0.02, n=3)
    res = 2 * np.pi / (len(t) * dt)
    np.testing.assert_allclose(pk, w, atol=res)
