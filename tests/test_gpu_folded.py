"""The first stage by the template method (Sec. III.D, Eqs. 10-12) and its low-pass alternative
(Sec. III.G) on the GPU against the FP64 oracle: one short inverse transform per template of the
folded (or band-limited) spectrum, thresholded at rho_I."""
import numpy as np
import pytest

from oracle import mf, rb
from paper_2110_13115_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_13115_gb300 import api as A, _native as N

    N.load()
    return A


def _case(n, fs, seed):
    g = inputs.Grid(fs=fs, n=n, f_low=30.0)
    psd = inputs.analytic_psd(g)
    x = inputs.coloured_noise(g, psd, inputs.noise_seed(seed, 0))
    spec = inputs.BankSpec(1, 10.0, 30.0, 0.0, 2)
    for j in inputs.draw_injections(spec, g, 1, 12.0, seed=7 + seed):
        x = x + inputs.injection_series(g, psd, j, 2)
    return g, psd, x.astype(np.float32)


CASES = [(1 << 14, 1024.0, 2), (1 << 14, 1024.0, 4), (1 << 14, 1024.0, 8), (1 << 14, 1024.0, 16),
         (1 << 19, 2048.0, 4), (1 << 19, 2048.0, 8), (1 << 19, 2048.0, 16)]


def _compare(got, ref, rms, rho_i, M):
    gm = {(int(c["tmpl"]), int(c["bin"])): float(c["snr_avg"]) for c in got}
    assert len(gm) > 10
    assert all(M // 2 <= b < M for _, b in gm)
    for key, v in gm.items():
        assert key in ref, key
        assert abs(v - ref[key]) <= 3e-5 * rms[key[0]] + 1e-5 * ref[key], (key, v, ref[key])
    for key, v in ref.items():
        if v >= rho_i * (1 + 1e-3):
            assert key in gm, key


@pytest.mark.parametrize("n,fs,w", CASES)
def test_lowpass_first_stage_vs_oracle(api, n, fs, w):
    # the band below n/w holds about 2/w of a random unit row's power: threshold scaled to match
    T, rho_i = 4, 2.2 * float(np.sqrt(2.0 / w))
    g, psd, x = _case(n, fs, seed=5)
    half, M = n // 2, n // w
    P = inputs.unit_rows(T, half, seed=70 + w).astype(np.complex64)
    d = api.make_desc(g.fs, n, 1, T, w=w, rho_i=rho_i, cand_capacity=1 << 20)
    buf, nc = api.rb_stage1_lowpass(d, torch.from_numpy(P).cuda(), torch.from_numpy(x).cuda(),
                                    torch.from_numpy(psd).cuda())
    got = api.candidates_numpy(buf, nc)
    df = g.fs / n
    scale = np.zeros(g.nf)
    scale[1:half] = np.sqrt(4.0 * df / psd[1:half])
    s_fd = mf.strain_fd(x.astype(np.float64), g.fs)
    ref, rms = {}, np.zeros(T)
    for t in range(T):
        h = np.zeros(g.nf, np.complex128)
        h[1:half] = P[t, 1:].astype(np.complex128) / scale[1:half]
        zb = rb.lowpass_first_stage(s_fd, h, psd, n, g.fs, w)[M // 2:]
        rms[t] = np.sqrt(np.mean(np.abs(zb) ** 2))
        for b in np.nonzero(np.abs(zb) >= rho_i * (1 - 1e-3))[0]:
            ref[(t, int(b) + M // 2)] = abs(zb[b])
    _compare(got, ref, rms, rho_i, M)


@pytest.mark.parametrize("n,fs,w", CASES)
def test_folded_first_stage_vs_oracle(api, n, fs, w):
    # averaging w samples keeps about 2/w of a random unit row's power: threshold scaled to match
    T, rho_i = 5, 1.6 * float(np.sqrt(2.0 / w))
    g, psd, x = _case(n, fs, seed=3)
    half, M = n // 2, n // w
    P = inputs.unit_rows(T, half, seed=90 + w).astype(np.complex64)
    d = api.make_desc(g.fs, n, 1, T, w=w, rho_i=rho_i, cand_capacity=1 << 20)
    buf, nc = api.rb_stage1_folded(d, torch.from_numpy(P).cuda(), torch.from_numpy(x).cuda(),
                                   torch.from_numpy(psd).cuda())
    got = api.candidates_numpy(buf, nc)
    # the oracle takes templates in strain units: h = g / sqrt(4 df / S) for the whitened rows g
    df = g.fs / n
    scale = np.zeros(g.nf)
    scale[1:half] = np.sqrt(4.0 * df / psd[1:half])
    s_fd = mf.strain_fd(x.astype(np.float64), g.fs)
    ref = {}
    rms = np.zeros(T)
    for t in range(T):
        h = np.zeros(g.nf, np.complex128)
        h[1:half] = P[t, 1:].astype(np.complex128) / scale[1:half]
        zb = rb.folded_first_stage(s_fd, h, psd, n, g.fs, w)[M // 2:]
        rms[t] = np.sqrt(np.mean(np.abs(zb) ** 2))
        for b in np.nonzero(np.abs(zb) >= rho_i * (1 - 1e-3))[0]:
            ref[(t, int(b) + M // 2)] = abs(zb[b])
        if t == 0:
            zb0 = zb
    gm = {(int(c["tmpl"]), int(c["bin"])): float(c["snr_avg"]) for c in got}
    assert len(gm) > 10
    assert all(M // 2 <= b < M for _, b in gm)
    for key, v in gm.items():
        assert key in ref, key
        assert abs(v - ref[key]) <= 3e-5 * rms[key[0]] + 1e-5 * ref[key], (key, v, ref[key])
    for key, v in ref.items():
        if v >= rho_i * (1 + 1e-3):
            assert key in gm, key
    # the folded series is the bin mean of the full-rate series (the identity of Eqs. 10-12)
    full = rb.basis_series(s_fd, psd, P[:1].astype(np.complex128), n, g.fs)[0]
    np.testing.assert_allclose(zb0, rb.bin_average(full[None, :], w)[0, M // 2:], atol=1e-9 * np.abs(full).max())


def test_folded_rejects_short_series_and_w1(api):
    from paper_2110_13115_gb300 import _native as N

    n = 1 << 12
    g, psd, x = _case(n, 1024.0, seed=4)
    P = inputs.unit_rows(2, n // 2, seed=5).astype(np.complex64)
    for w, code in ((8, N.RB_ERR_UNSUPPORTED), (1, N.RB_ERR_BAD_INPUT)):
        d = api.make_desc(g.fs, n, 1, 2, w=w, rho_i=2.0)
        with pytest.raises(N.RBError) as e:
            api.rb_stage1_folded(d, torch.from_numpy(P).cuda(), torch.from_numpy(x).cuda(), torch.from_numpy(psd).cuda())
        assert e.value.code == code
