"""Reduced-basis filtering and the two-stage hierarchy, FP64 (test infrastructure only).

Follows arXiv:2110.13115:

* Sec. III.B / Eq. (5b): the bank's whitened templates, normalised to unit
  norm and stored row-wise (no mean subtraction), are decomposed by an SVD;
  the leading right singular vectors are the basis, ranked by singular value.
  (The paper reaches the same subspace through an eigen-decomposition of the
  covariance, Eq. 5a; any exact route gives the same projector.)
* Eq. (6)-(7): with h = sum_k c_k p_k, the SNR series is
  z(t) = sum_k c_k^* beta_k(t), beta_k = IFFT(<s|p_k>).  Coefficients are
  stored divided by sigma_t so that |sum_k a_k^* beta_k| is the SNR directly.
* Eq. (8): the mean fractional SNR loss of truncating to k vectors,
  1 - sum_{i<k} s_i^2 / sum_i s_i^2.
* Sec. III.C, Eq. (9): beta^avg_k[i] = (1/w) sum_{j<w} beta_k[i w + j] over
  non-overlapping bins aligned to sample 0; stage one keeps (template, bin)
  pairs with |sum_k a_k^* beta^avg_k[i]| >= rho_I; stage two reconstructs
  every sample of those bins at full resolution and keeps the bin's arg-max
  when it is >= rho_II.
* Sec. III.D, Eqs. (10)-(12): the bin average of z equals a length-n/w inverse
  DFT of the folded spectrum Omega(f') = (1/w) sum_l Q[l n/w + f'] G(l n/w + f'),
  G(f) = sum_{r<w} exp(2 pi i f r / n), with the unnormalised inverse DFT of Eq. 6 (Eqs. 10-12 mix
  normalisation conventions; this one makes the folded series equal the bin mean exactly).
* Sec. III.G: the low-pass alternative to that first stage: the SNR series band-limited to the
  lowest n/w frequency bins (|f| < fs / (2 w) of the series' one-sided spectrum Q) and decimated by w,
  z_lp[b] = sum_{j < n/w} Q[j] exp(2 pi i j b w / n), b in [0, n/w).

The basis lives in whitened coordinates g_t[j] = sqrt(4 df / S_j) h_t[j] on
0 <= j < n/2, in which <a|b> of Eq. (1) is the Euclidean product.

Pinned by: full-rank reconstruction equal to the template method, the exact
truncation identity for noiseless self-injections and its bank average
against Eq. (8), the Eckart-Young residual, binning linearity, the
folded-first-stage identity, and the low-pass series against a brick-wall
filter of the full-rate series followed by decimation (tests/test_oracle_rb.py).
"""
from __future__ import annotations

import numpy as np

from .mf import TRIGGER_DTYPE

CAND_DTYPE = np.dtype([("template", np.int64), ("bin", np.int64), ("snr_avg", np.float64)])


def whitened_rows(templates, psd, n, fs):
    """Unit-normalised whitened rows g_t / sigma_t on j in [0, n/2) and sigma_t (FP64)."""
    df = fs / n
    half = n // 2
    scale = np.zeros(half)
    scale[1:] = np.sqrt(4.0 * df / np.asarray(psd, dtype=np.float64)[1:half])
    g = np.asarray(templates)[:, :half] * scale[None, :]
    sigma = np.sqrt(np.sum(np.abs(g) ** 2, axis=1))
    return g / sigma[:, None], sigma


def svd_basis(g_hat, k):
    """Leading-k right singular vectors (rows, [k, n/2]), all singular values, and the
    normalised coefficients a[t, k] = <g_hat_t, p_k> ([T, k])."""
    u, s, vh = np.linalg.svd(g_hat, full_matrices=False)
    basis = vh[:k]
    a = g_hat @ np.conj(basis).T
    return basis, s, a


def truncation_loss(s, k):
    """Eq. (8): mean SNR loss from keeping k of the singular values s."""
    s2 = np.asarray(s, dtype=np.float64) ** 2
    return 1.0 - float(np.sum(s2[:k]) / np.sum(s2))


def whitened_data(s_fd, psd, n, fs):
    """sqrt(4 df / S_j) s(f_j) on j in [0, n/2), zero at DC."""
    df = fs / n
    half = n // 2
    out = np.zeros(half, dtype=np.complex128)
    j = np.arange(1, half)
    out[j] = np.sqrt(4.0 * df / np.asarray(psd, dtype=np.float64)[j]) * s_fd[j]
    return out


def basis_series(s_fd, psd, basis, n, fs):
    """beta_k[m] = sum_{j<n/2} s_hat_j p_k[j]^* exp(2 pi i j m / n), m in [0, n) (Eq. 7)."""
    sh = whitened_data(s_fd, psd, n, fs)
    q = np.zeros((basis.shape[0], n), dtype=np.complex128)
    q[:, : n // 2] = sh[None, :] * np.conj(basis)
    return np.fft.ifft(q, axis=1) * n


def bin_average(beta, w):
    """Eq. (9): mean over non-overlapping bins of w samples aligned to sample 0."""
    k, n = beta.shape
    return beta.reshape(k, n // w, w).mean(axis=2)


def reconstruct(a, beta):
    """Eq. (7): z[t, m] = sum_k a[t, k]^* beta[k, m] (in SNR units)."""
    return np.conj(a) @ beta


def stage1(a, beta_avg, n, w, rho_i):
    """First-stage candidates: valid bins i in [n/(2w), n/w) with |sum a^* beta^avg| >= rho_I."""
    lo = n // (2 * w)
    r = np.abs(reconstruct(a, beta_avg[:, lo:]))
    t, i = np.nonzero(r >= rho_i)
    out = np.zeros(len(t), dtype=CAND_DTYPE)
    out["template"] = t
    out["bin"] = i + lo
    out["snr_avg"] = r[t, i]
    return out, r


def stage2(a, beta, cands, w, rho_ii):
    """Second stage: full-resolution reconstruction inside each candidate bin."""
    rows = []
    for c in cands:
        t, b = int(c["template"]), int(c["bin"])
        z = np.conj(a[t]) @ beta[:, b * w:(b + 1) * w]
        r = np.abs(z)
        j = int(np.argmax(r))
        if r[j] >= rho_ii:
            rows.append((t, b * w + j, r[j], np.angle(z[j])))
    out = np.array(rows, dtype=TRIGGER_DTYPE) if rows else np.zeros(0, TRIGGER_DTYPE)
    return np.sort(out, order=["template", "sample"])


def hierarchical_triggers(a, s_fd, psd, basis, n, fs, w, rho_i, rho_ii):
    """The whole hierarchy for one block; returns (triggers, candidates, beta)."""
    beta = basis_series(s_fd, psd, basis, n, fs)
    cands, _ = stage1(a, bin_average(beta, w), n, w, rho_i)
    return stage2(a, beta, cands, w, rho_ii), cands, beta


def folded_first_stage(s_fd, h, psd, n, fs, w):
    """Sec. III.D: bin-averaged z of one template from a length-n/w inverse DFT.

    Q[j] = 4 df s_j h_j^* / S_j (j < n/2, else 0); Omega(f') = (1/w) sum_{l<w}
    Q[l n/w + f'] G(l n/w + f') with G(f) = sum_{r<w} exp(2 pi i f r / n); then
    <z>_b = sum_{f'<n/w} Omega(f') exp(2 pi i f' b / (n/w)) for b in [0, n/w).
    """
    df = fs / n
    q = np.zeros(n, dtype=np.complex128)
    j = np.arange(1, n // 2)
    q[j] = 4.0 * df * s_fd[j] * np.conj(h[j]) / np.asarray(psd, dtype=np.float64)[j]
    f = np.arange(n)
    r = np.arange(w)
    g = np.exp(2j * np.pi * np.outer(f, r) / n).sum(axis=1)
    m = n // w
    omega = (q * g).reshape(w, m).sum(axis=0) / w
    return np.fft.ifft(omega) * m


def lowpass_first_stage(s_fd, h, psd, n, fs, w):
    """Sec. III.G: the low-pass and decimation first stage of one template.

    Q[j] = 4 df s_j h_j^* / S_j (0 < j < n/2); z_lp[b] = sum_{j < n/w} Q[j] exp(2 pi i j b / (n/w)) for
    b in [0, n/w): the full-rate series of Eq. 4 with every frequency bin j >= n/w removed, read at
    samples b w.
    """
    df = fs / n
    m = n // w
    q = np.zeros(m, dtype=np.complex128)
    j = np.arange(1, min(m, n // 2))
    q[j] = 4.0 * df * s_fd[j] * np.conj(h[j]) / np.asarray(psd, dtype=np.float64)[j]
    return np.fft.ifft(q) * m
