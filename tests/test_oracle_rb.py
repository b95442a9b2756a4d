"""Pins of the oracle's reduced basis and hierarchy (no GPU)."""
import numpy as np
import pytest

from oracle import mf, rb, waveform as W
from paper_2110_13115_gb300 import inputs


@pytest.fixture(scope="module")
def small():
    g = inputs.Grid(fs=512.0, n=4096, f_low=30.0)
    psd = inputs.analytic_psd(g)
    bank = inputs.draw_bank(inputs.BankSpec(24, 8.0, 20.0, 0.0, 2))
    hs = W.bank_templates(bank, g.fs, g.n, g.f_low, 2)
    ghat, sigma = rb.whitened_rows(hs, psd, g.n, g.fs)
    return g, psd, bank, hs, ghat, sigma


def test_sigma_matches_template_method(small):
    g, psd, bank, hs, ghat, sigma = small
    for t in range(3):
        np.testing.assert_allclose(sigma[t] ** 2, mf.sigma2(hs[t], psd, g.n, g.fs), rtol=1e-12)
    np.testing.assert_allclose(np.linalg.norm(ghat, axis=1), 1.0, rtol=1e-12)


def test_full_rank_basis_reproduces_template_method(small):
    """With every basis vector kept, Eq. (7) reproduces Eq. (4) exactly."""
    g, psd, bank, hs, ghat, sigma = small
    T = len(bank)
    basis, s, a = rb.svd_basis(ghat, T)
    strain = inputs.coloured_noise(g, psd, 11)
    sd = mf.strain_fd(strain, g.fs)
    beta = rb.basis_series(sd, psd, basis, g.n, g.fs)
    zr = rb.reconstruct(a, beta)
    for t in range(T):
        z, sig = mf.snr_series(sd, hs[t], psd, g.n, g.fs)
        np.testing.assert_allclose(zr[t], z / sig, atol=1e-10 * np.abs(z / sig).max())


def test_svd_against_gram_eigenvalues_and_eckart_young(small):
    g, psd, bank, hs, ghat, sigma = small
    k = 10
    basis, s, a = rb.svd_basis(ghat, k)
    ev = np.linalg.eigvalsh(ghat @ ghat.conj().T)[::-1]
    np.testing.assert_allclose(s ** 2, ev, rtol=1e-9, atol=1e-12 * ev[0])
    np.testing.assert_allclose(basis @ basis.conj().T, np.eye(k), atol=1e-12)
    resid = ghat - a @ basis
    np.testing.assert_allclose(np.sum(np.abs(resid) ** 2), np.sum(s[k:] ** 2), rtol=1e-9)


def test_truncation_identity_and_eq8(small):
    """Noiseless self-injection: rho_k / rho = 1 - r_t^2; the bank mean of r_t^2 is Eq. (8)."""
    g, psd, bank, hs, ghat, sigma = small
    k = 6
    basis, s, a = rb.svd_basis(ghat, k)
    r2 = 1.0 - np.sum(np.abs(a) ** 2, axis=1)
    np.testing.assert_allclose(np.mean(r2), rb.truncation_loss(s, k), rtol=1e-10)
    m0 = 3100
    f = g.freqs
    for t in [0, 5, 17]:
        s_fd = hs[t] * np.exp(-2j * np.pi * f * m0 / g.fs)
        beta = rb.basis_series(s_fd, psd, basis, g.n, g.fs)
        zr = rb.reconstruct(a[t:t + 1], beta)[0]
        z, sig = mf.snr_series(s_fd, hs[t], psd, g.n, g.fs)
        ratio = np.abs(zr[m0]) / (np.abs(z[m0]) / sig)
        np.testing.assert_allclose(ratio, 1.0 - r2[t], rtol=1e-10)


def test_binning_linearity_and_stages(small):
    g, psd, bank, hs, ghat, sigma = small
    T = len(bank)
    basis, s, a = rb.svd_basis(ghat, T)
    strain = inputs.coloured_noise(g, psd, 5)
    sd = mf.strain_fd(strain, g.fs)
    beta = rb.basis_series(sd, psd, basis, g.n, g.fs)
    w = 8
    zavg = rb.reconstruct(a, rb.bin_average(beta, w))
    zfull = rb.reconstruct(a, beta)
    np.testing.assert_allclose(zavg, zfull.reshape(T, -1, w).mean(axis=2), atol=1e-12)
    # stage 1 by brute force
    rho_i = 1.2
    cands, r = rb.stage1(a, rb.bin_average(beta, w), g.n, w, rho_i)
    lo = g.n // (2 * w)
    brute = [(t, i) for t in range(T) for i in range(lo, g.n // w) if abs(zavg[t, i]) >= rho_i]
    assert sorted(zip(cands["template"].tolist(), cands["bin"].tolist())) == brute
    # rho_I = 0 keeps every bin: the hierarchy equals the flat search (full-rank basis)
    trig, _, _ = rb.hierarchical_triggers(a, sd, psd, basis, g.n, g.fs, w, 0.0, 3.0)
    flat = mf.flat_triggers(bank, strain, psd, g.fs, g.n, g.f_low, 2, w, 3.0, templates=hs)
    assert trig["template"].tolist() == flat["template"].tolist()
    assert trig["sample"].tolist() == flat["sample"].tolist()
    np.testing.assert_allclose(trig["snr"], flat["snr"], rtol=1e-9)


@pytest.mark.parametrize("w", [2, 4, 8, 16])
def test_folded_first_stage_identity(small, w):
    """Sec. III.D: the folded length-n/w IFFT equals the bin mean of the exact series."""
    g, psd, bank, hs, ghat, sigma = small
    strain = inputs.coloured_noise(g, psd, 9)
    sd = mf.strain_fd(strain, g.fs)
    z, sig = mf.snr_series(sd, hs[4], psd, g.n, g.fs)
    zb = rb.folded_first_stage(sd, hs[4], psd, g.n, g.fs, w)
    np.testing.assert_allclose(zb, z.reshape(-1, w).mean(axis=1), atol=1e-11 * np.abs(z).max())


@pytest.mark.parametrize("w", [2, 4, 8, 16])
def test_lowpass_first_stage_is_band_limited_decimated_series(small, w):
    """Sec. III.G: the low-pass first stage equals the template method's full-rate series of a template
    band-limited to the lowest n/w frequency bins, read every w samples."""
    g, psd, bank, hs, ghat, sigma = small
    strain = inputs.coloured_noise(g, psd, 11)
    sd = mf.strain_fd(strain, g.fs)
    h = hs[3].copy()
    h[g.n // w:] = 0.0
    z, _ = mf.snr_series(sd, h, psd, g.n, g.fs)
    zl = rb.lowpass_first_stage(sd, hs[3], psd, g.n, g.fs, w)
    np.testing.assert_allclose(zl, z[::w], atol=1e-11 * np.abs(z).max())
    # and it differs from the bin average, which keeps every frequency (Eq. 11)
    zb = rb.folded_first_stage(sd, hs[3], psd, g.n, g.fs, w)
    assert np.abs(zl - zb).max() > 1e-3 * np.abs(zb).max()
