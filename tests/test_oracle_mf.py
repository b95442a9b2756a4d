"""Pins of the oracle's template method (no GPU)."""
import numpy as np
import pytest

from oracle import mf, waveform as W
from paper_2110_13115_gb300 import inputs


def _band_limited(rng, n):
    x = rng.standard_normal(n)
    X = np.fft.rfft(x)
    X[0] = 0
    X[-1] = 0
    return np.fft.irfft(X, n=n)


@pytest.mark.parametrize("n", [64, 256, 1024])
def test_brute_force_circular_correlation(n):
    """Flat PSD: Re z[m] = (2 dt/S) sum_n s[n+m] h[n]; Im z uses the quadrature template."""
    rng = np.random.default_rng(n)
    fs = 128.0
    dt = 1 / fs
    s = _band_limited(rng, n)
    h = _band_limited(rng, n)
    hq = np.fft.irfft(1j * np.fft.rfft(h), n=n)
    S = 3.7
    psd = np.full(n // 2 + 1, S)
    s_fd = mf.strain_fd(s, fs)
    h_fd = np.fft.rfft(h) * dt
    z, sig = mf.snr_series(s_fd, h_fd, psd, n, fs)
    re = np.array([np.sum(np.roll(s, -m) * h) for m in range(n)]) * 2 * dt / S
    im = np.array([np.sum(np.roll(s, -m) * hq) for m in range(n)]) * 2 * dt / S
    np.testing.assert_allclose(z.real, re, atol=1e-12 * np.abs(re).max())
    np.testing.assert_allclose(z.imag, im, atol=1e-12 * np.abs(im).max())
    # Parseval: sigma^2 = (2 dt / S) sum h[n]^2
    np.testing.assert_allclose(sig ** 2, 2 * dt / S * np.sum(h * h), rtol=1e-12)


def _tiny_grid():
    return inputs.Grid(fs=512.0, n=4096, f_low=30.0)


def test_optimal_snr_noiseless_injection():
    """A template injected at an integer sample with amplitude A peaks there at rho = A sigma."""
    g = _tiny_grid()
    psd = inputs.analytic_psd(g)
    bank = inputs.draw_bank(inputs.BankSpec(6, 8.0, 20.0, 0.0, 2))
    hs = W.bank_templates(bank, g.fs, g.n, g.f_low, 2)
    t0, m0, amp = 2, 3000, 0.37
    f = g.freqs
    s_fd = amp * hs[t0] * np.exp(-2j * np.pi * f * m0 / g.fs)
    strain = np.fft.irfft(s_fd, n=g.n) * g.fs
    sd = mf.strain_fd(strain, g.fs)
    z, sig = mf.snr_series(sd, hs[t0], psd, g.n, g.fs)
    rho = np.abs(z) / sig
    assert int(np.argmax(rho)) == m0
    np.testing.assert_allclose(rho[m0], amp * sig, rtol=1e-12)
    np.testing.assert_allclose(np.angle(z[m0]), 0.0, atol=1e-12)
    for t in range(len(bank)):
        z2, s2 = mf.snr_series(sd, hs[t], psd, g.n, g.fs)
        assert np.max(np.abs(z2)) / s2 <= amp * sig * (1 + 1e-12)  # Cauchy-Schwarz


def test_psd_scale_invariance():
    g = _tiny_grid()
    psd = inputs.analytic_psd(g)
    strain = inputs.coloured_noise(g, psd, 7)
    h = W.template((14.0, 9.0, 0, 0), g.fs, g.n, g.f_low, 2)
    sd = mf.strain_fd(strain, g.fs)
    z1, s1 = mf.snr_series(sd, h, psd, g.n, g.fs)
    # the noise level A scales the data by sqrt(A) and the PSD by A: SNR unchanged
    z2, s2 = mf.snr_series(sd * np.sqrt(1e3), h, psd * 1e3, g.n, g.fs)
    np.testing.assert_allclose(np.abs(z1) / s1, np.abs(z2) / s2, rtol=1e-12)


def test_noise_statistics():
    """Pure coloured noise: E[rho^2] = 2 and P(rho > x) = exp(-x^2/2)."""
    g = inputs.Grid(fs=1024.0, n=1 << 16, f_low=30.0)
    psd = inputs.analytic_psd(g)
    strain = inputs.coloured_noise(g, psd, inputs.noise_seed(3, 1))
    sd = mf.strain_fd(strain, g.fs)
    vals = []
    for p in [(12.0, 10.0, 0, 0), (25.0, 14.0, 0, 0), (18.0, 17.0, 0, 0)]:
        h = W.template(p, g.fs, g.n, g.f_low, 2)
        z, sig = mf.snr_series(sd, h, psd, g.n, g.fs)
        vals.append((np.abs(z) / sig) ** 2)
    r2 = np.concatenate(vals)
    neff = r2.size / 8  # neighbouring samples are correlated
    assert abs(r2.mean() - 2.0) < 5 * 2.0 / np.sqrt(neff)
    frac = np.mean(r2 > 2.5 ** 2)
    p = np.exp(-2.5 ** 2 / 2)
    assert abs(frac - p) < 5 * np.sqrt(p / neff)


def test_window_triggers_ties_and_alignment():
    n, w = 32, 4
    rho = np.zeros(n)
    rho[16:20] = [1.0, 6.0, 6.0, 2.0]  # tie: first index wins
    rho[20:24] = [5.0, 4.9, 0.0, 0.0]  # exactly at threshold: kept
    rho[28:32] = [0.0, 0.0, 0.0, 4.99]  # below
    z = rho * np.exp(0.3j)
    out = mf.window_triggers(7, rho, z, n, w, 5.0)
    assert out["sample"].tolist() == [17, 20]
    assert out["template"].tolist() == [7, 7]
    np.testing.assert_allclose(out["phase"], 0.3)
    rho[0] = 100.0  # invalid half is ignored
    assert len(mf.window_triggers(0, rho, z, n, w, 5.0)) == 2
