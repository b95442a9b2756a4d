"""GPU parity of template generation and the reduced basis (step a0), and of the whole
pipeline on synthetic chirp banks, against the FP64 oracle."""
import numpy as np
import pytest

from oracle import mf, rb, waveform as W
from paper_2110_13115_gb300 import inputs

from parity_util import compare_triggers

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_13115_gb300 import api as A, _native as N

    N.load()
    return A


def _bank_case(T, fs, n, mrange, chi, pn, f_low=30.0, seed=0):
    g = inputs.Grid(fs=fs, n=n, f_low=f_low)
    psd = inputs.analytic_psd(g)
    bank = inputs.draw_bank(inputs.BankSpec(T, mrange[0], mrange[1], chi, pn), seed=seed)
    return g, psd, bank


@pytest.mark.parametrize("T,fs,n,mrange,chi,pn", [(16, 1024.0, 1 << 14, (10, 30), 0.0, 2),
                                                  (12, 2048.0, 1 << 15, (3, 50), 0.5, 3),
                                                  (5, 1024.0, 1 << 12, (5, 8), 0.0, 0)])
def test_templates_parity(api, T, fs, n, mrange, chi, pn):
    g, psd, bank = _bank_case(T, fs, n, mrange, chi, pn)
    b = api.Bank(bank, fs, n, g.f_low, pn)
    rows, s2 = api.rb_templates(b, torch.from_numpy(psd).cuda())
    hs = W.bank_templates(bank, fs, n, g.f_low, pn)
    ref, sig = rb.whitened_rows(hs, psd, n, fs)
    np.testing.assert_allclose(s2.cpu().numpy(), sig ** 2, rtol=1e-12)
    got = rows.cpu().numpy()
    assert np.abs(got - ref).max() < 2e-6 * np.abs(ref).max()
    # identical support
    assert np.array_equal(np.abs(got) > 0, np.abs(ref) > 0)


def _projector_error(Pg, Po, seed=0):
    """max over random probes of |x Pg^H Pg - x Po^H Po| / |x|."""
    x = inputs.complex_normal((8, Po.shape[1]), seed)
    a = (x @ Pg.conj().T) @ Pg
    b = (x @ Po.conj().T) @ Po
    return np.abs(a - b).max() / np.abs(x).max()


def test_build_exact_small_bank(api):
    """T <= l: the sketch spans the whole row space, so the basis is the exact truncated SVD."""
    g, psd, bank = _bank_case(64, 1024.0, 1 << 14, (10, 30), 0.0, 2)
    b = api.Bank(bank, g.fs, g.n, g.f_low, 2)
    k = 16
    basis = api.rb_build(b, torch.from_numpy(psd).cuda(), k, oversample=64, power_iters=1)
    hs = W.bank_templates(bank, g.fs, g.n, g.f_low, 2)
    ghat, sig = rb.whitened_rows(hs, psd, g.n, g.fs)
    Po, s, ao = rb.svd_basis(ghat, k)
    np.testing.assert_allclose(basis.singular_values, s[:k], rtol=2e-5)
    np.testing.assert_allclose(basis.sigma2.cpu().numpy(), sig ** 2, rtol=1e-12)
    Pg = basis.vectors.cpu().numpy().astype(np.complex128)
    np.testing.assert_allclose(Pg @ Pg.conj().T, np.eye(k), atol=2e-5)
    assert _projector_error(Pg, Po) < 1e-4
    ag = basis.coeff.cpu().numpy().astype(np.complex128)
    # captured fraction ||a_t||^2 = 1 - r_t^2 (Eq. 8 per template) agrees template by template
    np.testing.assert_allclose(np.sum(np.abs(ag) ** 2, 1), np.sum(np.abs(ao) ** 2, 1), atol=2e-5)
    # coefficients are basis-dependent only through a unitary: compare reconstructions
    np.testing.assert_allclose(ag @ Pg, ao @ Po, atol=2e-4 * np.abs(ao @ Po).max())


def test_build_randomised_large_bank(api):
    """T > l: randomised subspace iteration vs the exact SVD on a 1.5PN spinning bank."""
    g, psd, bank = _bank_case(600, 2048.0, 1 << 15, (3, 50), 0.5, 3)
    b = api.Bank(bank, g.fs, g.n, g.f_low, 3)
    k = 64
    basis = api.rb_build(b, torch.from_numpy(psd).cuda(), k, oversample=64, power_iters=2)
    hs = W.bank_templates(bank, g.fs, g.n, g.f_low, 3)
    ghat, _ = rb.whitened_rows(hs, psd, g.n, g.fs)
    Po, s, ao = rb.svd_basis(ghat, k)
    np.testing.assert_allclose(basis.singular_values[:48], s[:48], rtol=1e-4)
    loss_gpu = 1.0 - np.mean(np.sum(np.abs(basis.coeff.cpu().numpy().astype(np.complex128)) ** 2, 1))
    loss_ref = rb.truncation_loss(s, k)
    assert abs(loss_gpu - loss_ref) <= 0.02 * loss_ref + 1e-6, (loss_gpu, loss_ref)


@pytest.mark.parametrize("k,w,rho_i", [(16, 8, 2.5), (40, 4, 3.0), (64, 16, 2.0)])
def test_pipeline_real_bank_vs_oracle_rb(api, k, w, rho_i):
    """GPU rb_build + rb_filter against the oracle's SVD + hierarchy on the tiny workload."""
    wl = inputs.tiny(w=w, k=k)
    g = wl.grid
    psd_d = torch.from_numpy(wl.psd).cuda()
    b = api.Bank(wl.bank, g.fs, g.n, g.f_low, 2)
    basis = api.rb_build(b, psd_d, k, oversample=64, power_iters=1)
    rho_ii = 5.0
    d = api.make_desc(g.fs, g.n, k, len(wl.bank), w=w, rho_i=rho_i, rho_ii=rho_ii, cand_capacity=1 << 18)
    api.rb_pack_coeff(d, basis)
    buf, nt = api.rb_filter(d, basis, torch.from_numpy(wl.strain).cuda(), psd_d)
    got = api.triggers_numpy(buf, nt)
    hs = W.bank_templates(wl.bank, g.fs, g.n, g.f_low, 2)
    ghat, _ = rb.whitened_rows(hs, wl.psd, g.n, g.fs)
    P, s, a = rb.svd_basis(ghat, k)
    s_fd = mf.strain_fd(wl.strain.astype(np.float64), g.fs)
    ref, cands, beta = rb.hierarchical_triggers(a, s_fd, wl.psd, P, g.n, g.fs, w, rho_i, rho_ii)
    half = g.n // 2
    zfull = np.abs(rb.reconstruct(a, beta[:, half:]))
    ravg = np.abs(rb.reconstruct(a, rb.bin_average(beta, w)[:, g.n // (2 * w):]))
    stats = compare_triggers(got, ref, w, rho_ii, ref_rho=zfull, rho_avg=ravg, rho_i=rho_i)
    assert stats["both"] >= 3, stats


def test_plain_real_bank_vs_oracle_template_method(api):
    """GPU rb_templates + rb_filter_plain against the oracle's per-template FFT matched filter."""
    wl = inputs.tiny(w=8)
    g = wl.grid
    psd_d = torch.from_numpy(wl.psd).cuda()
    b = api.Bank(wl.bank, g.fs, g.n, g.f_low, 2)
    rows, _ = api.rb_templates(b, psd_d)
    rho_ii = 5.0
    d = api.make_desc(g.fs, g.n, 1, len(wl.bank), w=8, rho_ii=rho_ii)
    buf, nt = api.rb_filter_plain(d, rows, torch.from_numpy(wl.strain).cuda(), psd_d)
    got = api.triggers_numpy(buf, nt)
    ref = mf.flat_triggers(wl.bank, wl.strain, wl.psd, g.fs, g.n, g.f_low, 2, 8, rho_ii)
    rho, _ = mf.snr_matrix(wl.bank, wl.strain, wl.psd, g.fs, g.n, g.f_low, 2)
    stats = compare_triggers(got, ref, 8, rho_ii, ref_rho=rho)
    assert stats["both"] >= 5, stats
