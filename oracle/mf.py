"""The template method, FP64, one template at a time (test infrastructure only).

Follows Sec. II of arXiv:2110.13115:

* Eq. (1): <s|h> = 4 int s(f) h*(f) / S_n(f) df, discretised on the block's
  frequency grid f_j = j df, one-sided (0 <= j < n/2, Nyquist excluded).
* Eq. (3)-(4): the coalescence time enters as exp(2 pi i f t_0), so the whole
  SNR time series is one unnormalised inverse DFT of length n:
      z[m] = sum_{j<n/2} 4 df s(f_j) h*(f_j)/S_j exp(+2 pi i j m / n).
* Eq. (2) with the phase maximised over (Sec. II, after Eq. 3): rho[m] = |z[m]| / sigma,
  sigma^2 = <h|h> = 4 df sum_j |h(f_j)|^2 / S_j.
* Sec. III.F: blocks of n samples overlap by n/2; only m in [n/2, n) is kept.
* Triggers: one per template and per aligned window of w valid samples (the
  bins of Sec. III.C), at the window's arg-max (ties to the smaller index),
  kept when rho >= rho_II.

Pinned by: brute-force circular time-domain correlation (real and quadrature
parts), Parseval for sigma^2, the closed-form optimal SNR of a noiseless
injection, Cauchy-Schwarz across templates, PSD-scale invariance and the
chi^2(2 dof) statistics of pure noise (tests/test_oracle_mf.py).
"""
from __future__ import annotations

import numpy as np

from . import waveform

TRIGGER_DTYPE = np.dtype([("template", np.int64), ("sample", np.int64), ("snr", np.float64), ("phase", np.float64)])


def strain_fd(strain, fs):
    """s(f_j) = dt * sum_n s[n] exp(-2 pi i j n / n_samples), j in [0, n/2]."""
    x = np.asarray(strain, dtype=np.float64)
    return np.fft.rfft(x) / fs


def inner_weights(psd, n, fs):
    """4 df / S_j on 0 <= j < n/2 (zero at DC and Nyquist)."""
    nf = n // 2 + 1
    wgt = np.zeros(nf)
    j = np.arange(1, n // 2)
    wgt[j] = 4.0 * (fs / n) / np.asarray(psd, dtype=np.float64)[j]
    return wgt


def sigma2(h, psd, n, fs):
    """<h|h> = 4 df sum_j |h_j|^2 / S_j (Eq. 2 denominator)."""
    return float(np.sum(inner_weights(psd, n, fs) * np.abs(h) ** 2))


def snr_series(s_fd, h, psd, n, fs):
    """Complex z[m], m in [0, n), of Eq. (4) as an unnormalised inverse DFT, and sigma."""
    q = np.zeros(n, dtype=np.complex128)
    wgt = inner_weights(psd, n, fs)
    q[: n // 2] = (wgt * s_fd * np.conj(h))[: n // 2]
    z = np.fft.ifft(q) * n
    return z, np.sqrt(sigma2(h, psd, n, fs))


def window_triggers(template_id, rho, z, n, w, rho_th):
    """Per aligned window of w valid samples: arg-max (first on ties); keep rho >= rho_th."""
    lo = n // 2
    r = rho[lo:].reshape(-1, w)
    am = np.argmax(r, axis=1)  # numpy returns the first maximum
    best = r[np.arange(r.shape[0]), am]
    keep = np.nonzero(best >= rho_th)[0]
    out = np.zeros(len(keep), dtype=TRIGGER_DTYPE)
    m = lo + keep * w + am[keep]
    out["template"] = template_id
    out["sample"] = m
    out["snr"] = best[keep]
    out["phase"] = np.angle(z[m])
    return out


def flat_triggers(bank, strain, psd, fs, n, f_low, pn_order, w, rho_ii, templates=None, which=None):
    """Template-method triggers of a whole bank (or the rows ``which``).

    ``templates`` may pass precomputed h(f) rows; otherwise they are generated.
    Returns a TRIGGER_DTYPE array sorted by (template, sample).
    """
    s_fd = strain_fd(strain, fs)
    idx = range(len(bank)) if which is None else which
    parts = []
    for t in idx:
        h = templates[t] if templates is not None else waveform.template(bank[t], fs, n, f_low, pn_order)
        z, sig = snr_series(s_fd, h, psd, n, fs)
        parts.append(window_triggers(t, np.abs(z) / sig, z, n, w, rho_ii))
    out = np.concatenate(parts) if parts else np.zeros(0, TRIGGER_DTYPE)
    return np.sort(out, order=["template", "sample"])


def snr_matrix(bank, strain, psd, fs, n, f_low, pn_order, templates=None):
    """rho[t, m] and complex z[t, m] over the valid half for every template (small cases)."""
    s_fd = strain_fd(strain, fs)
    rows_r, rows_z = [], []
    for t in range(len(bank)):
        h = templates[t] if templates is not None else waveform.template(bank[t], fs, n, f_low, pn_order)
        z, sig = snr_series(s_fd, h, psd, n, fs)
        rows_r.append(np.abs(z[n // 2:]) / sig)
        rows_z.append(z[n // 2:] / sig)
    return np.array(rows_r), np.array(rows_z)
