"""Sub-banks along lines of equal chirp time, each with its own basis size (Sec. III.B, Table I), on
the GPU: the per-template loss that chooses each basis size, rb_filter_banks against one rb_filter per
sub-bank, and the whole path (rb_build, the basis size for a per-template SNR-loss tolerance,
rb_filter_banks) against the FP64 oracle's template method on noiseless injections."""
import numpy as np
import pytest

from oracle import mf, rb
from paper_2110_13115_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GATE = 1e-3  # relative SNR loss allowed against the template method (per template, not a bank mean)


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_13115_gb300 import api as A, _native as N

    N.load()
    return A


def _parts(api, wl, parts):
    g = wl.grid
    bank = api.Bank(wl.bank, g.fs, g.n, g.f_low, wl.bank_spec.pn_order)
    order, offs = api.rb_bank_split_tau0(api.rb_bank_tau0(bank, g.f_low), parts)
    return [order[offs[p]:offs[p + 1]] for p in range(parts)]


def _sub_bases(api, wl, psd, parts, k_build, tol=None, ks=None):
    g = wl.grid
    out = []
    for p, idx in enumerate(parts):
        b = api.rb_build(api.Bank(np.ascontiguousarray(wl.bank[idx]), g.fs, g.n, g.f_low, wl.bank_spec.pn_order),
                         psd, min(k_build, len(idx)), oversample=64, power_iters=1)
        loss = api.rb_basis_max_loss(b)
        if ks is not None:
            k = ks[p]
        else:
            ok = np.nonzero(loss <= tol)[0]
            assert len(ok), (p, loss[-1])
            k = int(ok[0]) + 1
        out.append((idx, api.truncate(b, k), loss))
    return out


def test_max_loss_matches_coefficients(api):
    k = 24
    wl = inputs.tiny(k=k)
    g = wl.grid
    psd = torch.from_numpy(wl.psd).cuda()
    b = api.rb_build(api.Bank(wl.bank, g.fs, g.n, g.f_low, 2), psd, k, oversample=64, power_iters=1)
    got = api.rb_basis_max_loss(b)
    a = b.coeff.cpu().numpy().astype(np.complex128)
    want = np.maximum(1.0 - np.cumsum(np.abs(a) ** 2, axis=1), 0.0).max(axis=0)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-14)
    assert np.all(np.diff(got) <= 1e-15)  # more vectors never lose more


@pytest.mark.parametrize("prec", ["fp16_split_a", "fp32"])
def test_banks_equal_one_filter_per_sub_bank(api, prec):
    """rb_filter_banks (whitening once, one trigger list, global template rows) gives bit for bit the
    triggers of one rb_filter call per sub-bank with the rows shifted by the sub-banks before it; host
    buffers give the same again."""
    wl = inputs.scaled("sub", 2048.0, 1 << 15, 300, n_inj=2, min_sep=1.0)
    g = wl.grid
    psd = torch.from_numpy(wl.psd).cuda()
    strain = torch.from_numpy(wl.strain).cuda()
    subs = _sub_bases(api, wl, psd, _parts(api, wl, 3), 64, ks=[40, 32, 24])
    descs, bases, ref = [], [], []
    base = 0
    for idx, b, _ in subs:
        d = api.make_desc(g.fs, g.n, b.k, len(idx), w=8, precision=prec, rho_i=2.5, rho_ii=4.0, cand_capacity=1 << 18)
        api.rb_pack_coeff(d, b)
        buf, n = api.rb_filter(d, b, strain, psd, capacity=1 << 18)
        t = api.triggers_numpy(buf, n)
        t["tmpl"] += base
        ref.append(t)
        base += len(idx)
        descs.append(d)
        bases.append(b)
    ref = np.sort(np.concatenate(ref), order=["tmpl", "sample"])
    assert len(ref) > 10
    buf, n = api.rb_filter_banks(descs, bases, strain, psd, capacity=1 << 18)
    assert np.array_equal(api.triggers_numpy(buf, n), ref)
    hbuf, hn = api.rb_filter_banks(descs, bases, np.ascontiguousarray(wl.strain), psd, capacity=1 << 18, host=True)
    assert np.array_equal(np.sort(hbuf[:hn], order=["tmpl", "sample"]), ref)


def test_banks_injections_vs_oracle_template_method(api):
    """Full-size recipe scaled down (1,000 templates, 64 s at 2048 Hz, three noiseless injections), two
    tau0 sub-banks whose basis sizes hold every template's loss within the gate. For each injection
    the best template's hierarchical SNR matches the FP64 oracle's template method within the gate,
    and the GPU matches the oracle's own reduced-basis series of the same basis to FP32 accuracy."""
    wl = inputs.scaled("sub-e2e", 2048.0, 1 << 17, 1000, n_inj=3, snr_range=(8.0, 15.0), min_sep=4.0, noise=False)
    g = wl.grid
    psd = torch.from_numpy(wl.psd).cuda()
    strain = torch.from_numpy(wl.strain).cuda()
    subs = _sub_bases(api, wl, psd, _parts(api, wl, 2), 320, tol=GATE)
    descs, bases, rows = [], [], []
    for idx, b, loss in subs:
        assert loss[b.k - 1] <= GATE
        d = api.make_desc(g.fs, g.n, b.k, len(idx), w=8, precision="fp16_split_a", rho_i=2.0, rho_ii=3.0,
                          cand_capacity=1 << 22)
        api.rb_pack_coeff(d, b)
        descs.append(d)
        bases.append(b)
        rows.append(idx)
    rows = np.concatenate(rows)  # global row -> bank template
    buf, n = api.rb_filter_banks(descs, bases, strain, psd, capacity=1 << 22)
    hier = api.triggers_numpy(buf, n)
    # the best template of each injection from the template method on the GPU (sub-bank row order)
    templates = api.rb_templates(api.Bank(np.ascontiguousarray(wl.bank[rows]), g.fs, g.n, g.f_low,
                                          wl.bank_spec.pn_order), psd)[0]
    dp = api.make_desc(g.fs, g.n, 1, len(rows), w=8, rho_ii=3.0)
    pbuf, pn = api.rb_filter_plain(dp, templates, strain, psd, capacity=1 << 22)
    flat = api.triggers_numpy(pbuf, pn)
    s_fd = mf.strain_fd(wl.strain.astype(np.float64), g.fs)
    hmap = {(int(t["tmpl"]), int(t["sample"]) // 8): t for t in hier}
    from oracle import waveform as W

    worst = 0.0
    betas = {}
    for inj in wl.injections:
        m_c = int(round(inj.tc * g.fs))
        near = flat[np.abs(flat["sample"] - m_c) <= int(0.05 * g.fs)]
        best = near[np.argmax(near["snr"])]
        r, key = int(best["tmpl"]), (int(best["tmpl"]), int(best["sample"]) // 8)
        h = W.template(wl.bank[rows[r]], g.fs, g.n, g.f_low, wl.bank_spec.pn_order)
        z, sig = mf.snr_series(s_fd, h, wl.psd, g.n, g.fs)
        w0 = key[1] * 8
        rho_flat = np.abs(z[w0:w0 + 8]).max() / sig
        assert key in hmap, (inj, key)
        rho_gpu = float(hmap[key]["snr"])
        # the oracle's FP64 reduced-basis SNR of the same basis (FP32 parity of the GPU path)
        sub = np.searchsorted(np.cumsum([len(i) for i, _, _ in subs]), r, side="right")
        idx, b, _ = subs[sub]
        local = r - sum(len(i) for i, _, _ in subs[:sub])
        if sub not in betas:
            betas[sub] = rb.basis_series(s_fd, wl.psd, b.vectors.cpu().numpy().astype(np.complex128), g.n, g.fs)
        a = b.coeff.cpu().numpy().astype(np.complex128)[local:local + 1]
        rho_rb = np.abs(rb.reconstruct(a, betas[sub][:, w0:w0 + 8])).max()
        assert abs(rho_gpu - rho_rb) <= 1e-4 * rho_rb, (inj, rho_gpu, rho_rb)
        rel = abs(rho_gpu - rho_flat) / rho_flat
        worst = max(worst, rel)
        assert rel <= GATE, (inj, rho_gpu, rho_flat, rel)
    print(f"worst injection SNR loss {worst:.2e}; basis sizes {[b.k for _, b, _ in subs]}")
