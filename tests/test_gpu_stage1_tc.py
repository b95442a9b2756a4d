"""GPU parity of the tcgen05 first stage (16-bit operands, FP32 accumulation in tensor memory)
against the FP64 oracle, for every precision, on tile-aligned and ragged shapes."""
import numpy as np
import pytest

from oracle import mf, rb, waveform as W
from paper_2110_13115_gb300 import inputs

from parity_util import compare_triggers

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# worst relative error of |z_avg| expected per precision (hi+lo splits keep ~16-22 bits; splitting only
# the coefficients leaves beta_avg's FP16 rounding, about 2^-11 per element, which stays below the
# 1e-3 relative SNR tolerance of the screen)
REL = {"fp16_split": 2e-5, "bf16_split": 1e-4, "fp16": 3e-3, "bf16": 2e-2, "fp16_split_a": 1e-3}
# modes whose screening decisions must agree with the oracle outside a 1e-3 band around rho_I; the
# plain 16-bit modes are reported with a band of twice their own error
SPLIT = ("fp16_split", "bf16_split", "fp16_split_a")


def _band(prec):
    return 1e-3 if prec in SPLIT else max(REL[prec] * 2, 1e-3)


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_13115_gb300 import api as A, _native as N

    N.load()
    return A


def _case(api, T, k, n, w, rho_i, prec, seed=1, variant=0):
    nb = n // (2 * w)
    a = inputs.complex_normal((T, k), seed)
    a = (a / np.linalg.norm(a, axis=1, keepdims=True)).astype(np.complex64)
    bv = inputs.complex_normal((k, nb), seed + 1).astype(np.complex64)
    d = api.make_desc(1024.0, n, k, T, w=w, precision=prec, rho_i=rho_i, cand_capacity=1 << 22)
    basis = api.Basis(torch.zeros((k, n // 2), dtype=torch.complex64, device="cuda"), torch.from_numpy(a).cuda(), n)
    api.rb_pack_coeff(d, basis)
    api.rb_set_stage1_variant(d, variant)
    buf, nc = api.rb_stage1(d, basis, torch.from_numpy(bv).cuda())
    got = api.candidates_numpy(buf, nc)
    full = np.zeros((k, n // w), np.complex128)
    full[:, nb:] = bv
    ref, r = rb.stage1(a.astype(np.complex128), full, n, w, rho_i)
    return got, ref, r, nb


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("prec", ["fp16_split", "bf16_split", "fp16", "bf16", "fp16_split_a"])
@pytest.mark.parametrize("T,k,n,w", [(64, 32, 1 << 14, 16),  # one M tile, two N tiles, K = 64
                                     (200, 24, 1 << 14, 8),  # ragged M (400 rows), ragged K (48 -> 64)
                                     (333, 96, 1 << 15, 4),  # ragged M, N = 4096, K = 192
                                     (1000, 256, 1 << 16, 16)])  # K = 512 (eight K blocks)
def test_stage1_tc_parity(api, prec, T, k, n, w, variant):
    rho_i = 2.6
    got, ref, r, nb = _case(api, T, k, n, w, rho_i, prec, variant=variant)
    band = _band(prec)
    gset = set(zip(got["tmpl"].tolist(), got["bin"].tolist()))
    oset = set(zip(ref["template"].tolist(), ref["bin"].tolist()))
    assert len(oset) > 20
    for t, i in gset ^ oset:
        assert abs(r[t, i - nb] - rho_i) <= band * rho_i, (prec, t, i, r[t, i - nb])
    m = {(int(c["tmpl"]), int(c["bin"])): float(c["snr_avg"]) for c in got}
    errs = [abs(m[(int(c["template"]), int(c["bin"]))] - c["snr_avg"]) / c["snr_avg"] for c in ref
            if (int(c["template"]), int(c["bin"])) in m]
    assert max(errs) < REL[prec], (prec, max(errs))


@pytest.mark.parametrize("variant", [0, 1])
def test_stage1_tc_everything_passes_at_zero_threshold(api, variant):
    """rho_I = 0 keeps every (template, valid bin): exact count, padding rows and columns excluded."""
    T, k, n, w = 70, 40, 1 << 13, 8
    got, ref, r, nb = _case(api, T, k, n, w, 0.0, "fp16_split", variant=variant)
    assert len(got) == T * nb == len(ref)
    assert got["bin"].min() == nb and got["bin"].max() == 2 * nb - 1
    assert got["tmpl"].max() == T - 1


def test_stage1_tc_overflow_reports_count(api):
    from paper_2110_13115_gb300 import _native as N

    T, k, n, w = 64, 32, 1 << 13, 8
    nb = n // (2 * w)
    a = (np.ones((T, k)) / np.sqrt(k)).astype(np.complex64)
    bv = np.ones((k, nb), np.complex64)
    d = api.make_desc(1024.0, n, k, T, w=w, precision="fp16", rho_i=0.0, cand_capacity=100)
    basis = api.Basis(torch.zeros((k, n // 2), dtype=torch.complex64, device="cuda"), torch.from_numpy(a).cuda(), n)
    api.rb_pack_coeff(d, basis)
    with pytest.raises(N.RBError) as e:
        api.rb_stage1(d, basis, torch.from_numpy(bv).cuda())
    assert e.value.code == N.RB_ERR_OVERFLOW


@pytest.mark.parametrize("prec,w,rho_i", [("fp16_split", 8, 2.5), ("fp16", 4, 3.0), ("bf16_split", 16, 2.0),
                                          ("fp16_split_a", 8, 2.5)])
def test_pipeline_tc_real_bank_vs_oracle_rb(api, prec, w, rho_i):
    """GPU rb_build + rb_filter (tensor-core first stage) against the oracle's SVD + hierarchy."""
    k = 40
    wl = inputs.tiny(w=w, k=k)
    g = wl.grid
    psd_d = torch.from_numpy(wl.psd).cuda()
    b = api.Bank(wl.bank, g.fs, g.n, g.f_low, 2)
    basis = api.rb_build(b, psd_d, k, oversample=64, power_iters=1)
    rho_ii = 5.0
    d = api.make_desc(g.fs, g.n, k, len(wl.bank), w=w, precision=prec, rho_i=rho_i, rho_ii=rho_ii,
                      cand_capacity=1 << 18)
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
    band = _band(prec)
    stats = compare_triggers(got, ref, w, rho_ii, ref_rho=zfull, rho_avg=ravg, rho_i=rho_i, band=band)
    assert stats["both"] >= 3, stats


def test_tuner_picks_a_variant(api):
    T, k, n, w = 500, 64, 1 << 15, 8
    nb = n // (2 * w)
    a = inputs.complex_normal((T, k), 5)
    a = (a / np.linalg.norm(a, axis=1, keepdims=True)).astype(np.complex64)
    bv = inputs.complex_normal((k, nb), 6).astype(np.complex64)
    d = api.make_desc(1024.0, n, k, T, w=w, precision="fp16", rho_i=3.0, cand_capacity=1 << 20)
    basis = api.Basis(torch.zeros((k, n // 2), dtype=torch.complex64, device="cuda"), torch.from_numpy(a).cuda(), n)
    api.rb_pack_coeff(d, basis)
    chosen, times = api.rb_tune_stage1(d, basis, torch.from_numpy(bv).cuda())
    assert chosen in (0, 1) and all(t > 0 for t in times)
    assert times[chosen] == min(times)
    # the tuned choice is used afterwards and still gives the oracle's candidates
    buf, nc = api.rb_stage1(d, basis, torch.from_numpy(bv).cuda())
    full = np.zeros((k, n // w), np.complex128)
    full[:, nb:] = bv
    ref, r = rb.stage1(a.astype(np.complex128), full, n, w, 3.0)
    got = api.candidates_numpy(buf, nc)
    diff = set(zip(got["tmpl"].tolist(), got["bin"].tolist())) ^ set(zip(ref["template"].tolist(), ref["bin"].tolist()))
    assert all(abs(r[t, i - nb] - 3.0) <= 6e-3 * 3.0 for t, i in diff)
