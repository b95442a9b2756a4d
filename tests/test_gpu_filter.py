"""GPU parity of the filter path (a1-a5, template method) against the FP64 oracle.

Both sides consume the same seeded inputs; the CUDA path is reached only through the C ABI
(paper_2110_13115_gb300.api -> librbmf.so).
"""
import numpy as np
import pytest

from oracle import mf, rb
from paper_2110_13115_gb300 import inputs

from parity_util import BAND, compare_triggers

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_13115_gb300 import api as A, _native as N

    N.load()
    return A


def _strain(n, fs=1024.0, seed=0, inj=None):
    inj = n >= (1 << 13) if inj is None else inj
    g = inputs.Grid(fs=fs, n=n, f_low=30.0)
    psd = inputs.analytic_psd(g)
    x = inputs.coloured_noise(g, psd, inputs.noise_seed(seed, 0))
    if inj:
        spec = inputs.BankSpec(1, 10.0, 30.0, 0.0, 2)
        for j in inputs.draw_injections(spec, g, 1, 12.0, seed=7 + seed):
            x = x + inputs.injection_series(g, psd, j, 2)
    return g, psd, x.astype(np.float32)


def _dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


@pytest.mark.parametrize("n", [1 << 10, 1 << 11, 1 << 13, 1 << 14, 1 << 16, 1 << 19])
def test_whiten_parity(api, n):
    g, psd, x = _strain(n, fs=2048.0 if n >= (1 << 16) else 1024.0)
    d = api.make_desc(g.fs, n, 1, 1, w=1)
    sh = api.rb_whiten(d, _dev(x), _dev(psd)).cpu().numpy()
    ref = rb.whitened_data(mf.strain_fd(x.astype(np.float64), g.fs), psd, n, g.fs)
    err = np.abs(sh - ref).max() / np.sqrt(np.mean(np.abs(ref) ** 2))
    assert err < 2e-5, err
    assert sh[0] == 0


@pytest.mark.parametrize("n,k,w", [(1 << 12, 8, 1), (1 << 13, 24, 4), (1 << 14, 24, 8), (1 << 17, 16, 16),
                                   (1 << 15, 40, 2)])
def test_basis_filter_parity(api, n, k, w):
    g, psd, x = _strain(n)
    half = n // 2
    P = inputs.unit_rows(k, half, seed=100 + k)
    d = api.make_desc(g.fs, n, k, 1, w=w)
    basis = api.Basis(_dev(P, torch.complex64), _dev(np.ones((1, k)), torch.complex64), n)
    sh = api.rb_whiten(d, _dev(x), _dev(psd))
    beta, bavg = api.rb_basis_filter(d, basis, sh)
    beta, bavg = beta.cpu().numpy(), bavg.cpu().numpy()
    s_fd = mf.strain_fd(x.astype(np.float64), g.fs)
    ref = rb.basis_series(s_fd, psd, P.astype(np.complex64).astype(np.complex128), n, g.fs)
    rref = ref[:, half:]
    scale = np.sqrt(np.mean(np.abs(rref) ** 2))
    assert np.abs(beta - rref).max() / scale < 3e-5
    aref = rb.bin_average(ref, w)[:, n // (2 * w):]
    assert np.abs(bavg - aref).max() / scale < 3e-5


def test_basis_filter_full_size_sampled_rows(api):
    """n = 2^19, k = 256 in the benchmark's launch configuration; 4 rows checked one by one."""
    n, k, w = 1 << 19, 256, 8
    g, psd, x = _strain(n, fs=2048.0)
    half = n // 2
    P = inputs.unit_rows(k, half, seed=5).astype(np.complex64)
    d = api.make_desc(g.fs, n, k, 1, w=w)
    basis = api.Basis(_dev(P), _dev(np.ones((1, k), np.complex64)), n)
    sh = api.rb_whiten(d, _dev(x), _dev(psd))
    beta, bavg = api.rb_basis_filter(d, basis, sh)
    s_fd = mf.strain_fd(x.astype(np.float64), g.fs)
    for row in [0, 77, 200, 255]:
        ref = rb.basis_series(s_fd, psd, P[row:row + 1].astype(np.complex128), n, g.fs)
        rref = ref[0, half:]
        got = beta[row].cpu().numpy()
        scale = np.sqrt(np.mean(np.abs(rref) ** 2))
        assert np.abs(got - rref).max() / scale < 5e-5, row
        aref = rb.bin_average(ref, w)[0, n // (2 * w):]
        assert np.abs(bavg[row].cpu().numpy() - aref).max() / scale < 5e-5, row


def _rand_coeff(T, k, seed):
    a = inputs.complex_normal((T, k), seed)
    return a / np.linalg.norm(a, axis=1, keepdims=True)


@pytest.mark.parametrize("T,k,w,rho_i", [(200, 24, 8, 3.0), (130, 16, 1, 3.3), (64, 40, 16, 2.6)])
def test_stage1_fp32_parity(api, T, k, w, rho_i):
    n = 1 << 14
    nb = n // (2 * w)
    a = _rand_coeff(T, k, 1).astype(np.complex64)
    bv = inputs.complex_normal((k, nb), 2).astype(np.complex64)
    d = api.make_desc(1024.0, n, k, T, w=w, rho_i=rho_i, cand_capacity=1 << 16)
    basis = api.Basis(_dev(np.zeros((k, n // 2), np.complex64)), _dev(a), n)
    buf, nc = api.rb_stage1(d, basis, _dev(bv))
    got = api.candidates_numpy(buf, nc)
    full = np.zeros((k, n // w), np.complex128)
    full[:, nb:] = bv
    ref, r = rb.stage1(a.astype(np.complex128), full, n, w, rho_i)
    gset = set(zip(got["tmpl"].tolist(), got["bin"].tolist()))
    oset = set(zip(ref["template"].tolist(), ref["bin"].tolist()))
    for t, i in gset ^ oset:
        assert abs(r[t, i - nb] - rho_i) <= BAND * rho_i, (t, i)
    assert len(oset) > 20
    m = {(int(c["tmpl"]), int(c["bin"])): float(c["snr_avg"]) for c in got}
    for c in ref:
        key = (int(c["template"]), int(c["bin"]))
        if key in m:
            assert abs(m[key] - c["snr_avg"]) <= 1e-5 * c["snr_avg"]


@pytest.mark.parametrize("w", [1, 2, 4, 8, 16])
def test_stage2_parity(api, w):
    n, k, T = 1 << 14, 24, 50
    half = n // 2
    a = _rand_coeff(T, k, 3).astype(np.complex64)
    beta = inputs.complex_normal((k, half), 4).astype(np.complex64)
    rng = np.random.default_rng(5)
    nb = n // (2 * w)
    cands = np.zeros(400, dtype=api.CANDIDATE_NP)
    cands["tmpl"] = rng.integers(0, T, 400)
    cands["bin"] = nb + rng.integers(0, nb, 400)
    cands = np.unique(cands)
    d = api.make_desc(1024.0, n, k, T, w=w, rho_ii=2.2)
    basis = api.Basis(_dev(np.zeros((k, half), np.complex64)), _dev(a), n)
    api.rb_pack_coeff(d, basis)
    cbuf = _dev(cands.view(np.uint8))
    buf, nt = api.rb_stage2(d, basis, _dev(beta), cbuf, len(cands))
    got = api.triggers_numpy(buf, nt)
    full = np.zeros((k, n), np.complex128)
    full[:, half:] = beta
    oc = np.zeros(len(cands), dtype=rb.CAND_DTYPE)
    oc["template"] = cands["tmpl"]
    oc["bin"] = cands["bin"]
    ref = rb.stage2(a.astype(np.complex128), full, oc, w, 2.2)
    zr = np.abs(np.conj(a.astype(np.complex128)) @ beta.astype(np.complex128))
    stats = compare_triggers(got, ref, w, 2.2, ref_rho=zr)
    assert stats["both"] > 20


@pytest.mark.parametrize("n,k,T,w", [(1 << 14, 24, 40, 8), (1 << 13, 16, 33, 4), (1 << 12, 8, 17, 16),
                                     (1 << 14, 12, 20, 1)])
def test_filter_end_to_end_fp32(api, n, k, T, w):
    g, psd, x = _strain(n, seed=1)
    half = n // 2
    P = inputs.unit_rows(k, half, seed=11).astype(np.complex64)
    a = _rand_coeff(T, k, 12).astype(np.complex64)
    # random white rows decorrelate neighbouring samples, so the bin mean shrinks as 1/sqrt(w)
    rho_i, rho_ii = 2.2 / np.sqrt(w), 3.0
    d = api.make_desc(g.fs, n, k, T, w=w, rho_i=rho_i, rho_ii=rho_ii, cand_capacity=1 << 18)
    basis = api.Basis(_dev(P), _dev(a), n)
    api.rb_pack_coeff(d, basis)
    buf, nt = api.rb_filter(d, basis, _dev(x), _dev(psd))
    got = api.triggers_numpy(buf, nt)
    s_fd = mf.strain_fd(x.astype(np.float64), g.fs)
    P64, a64 = P.astype(np.complex128), a.astype(np.complex128)
    ref, cands, beta = rb.hierarchical_triggers(a64, s_fd, psd, P64, n, g.fs, w, rho_i, rho_ii)
    zfull = np.abs(rb.reconstruct(a64, beta[:, half:]))
    ravg = np.abs(rb.reconstruct(a64, rb.bin_average(beta, w)[:, n // (2 * w):]))
    stats = compare_triggers(got, ref, w, rho_ii, ref_rho=zfull, rho_avg=ravg, rho_i=rho_i)
    assert stats["both"] >= 5, stats


@pytest.mark.parametrize("n,T,w", [(1 << 14, 48, 8), (1 << 12, 20, 1), (1 << 16, 8, 16)])
def test_filter_plain_parity(api, n, T, w):
    g, psd, x = _strain(n, seed=2)
    half = n // 2
    rows = inputs.unit_rows(T, half, seed=21).astype(np.complex64)
    rho_ii = 3.2
    d = api.make_desc(g.fs, n, 1, T, w=w, rho_ii=rho_ii)
    buf, nt = api.rb_filter_plain(d, _dev(rows), _dev(x), _dev(psd))
    got = api.triggers_numpy(buf, nt)
    s_fd = mf.strain_fd(x.astype(np.float64), g.fs)
    z = rb.basis_series(s_fd, psd, rows.astype(np.complex128), n, g.fs)
    rho = np.abs(z)
    ref = np.concatenate([mf.window_triggers(t, rho[t], z[t], n, w, rho_ii) for t in range(T)])
    stats = compare_triggers(got, ref, w, rho_ii, ref_rho=rho[:, half:])
    assert stats["both"] > 10, stats


def test_overflow_and_errors(api):
    from paper_2110_13115_gb300 import _native as N

    n, T = 1 << 12, 8
    g, psd, x = _strain(n, seed=3)
    rows = inputs.unit_rows(T, n // 2, seed=31).astype(np.complex64)
    d = api.make_desc(g.fs, n, 1, T, w=1, rho_ii=0.5)
    _, full = api.rb_filter_plain(d, _dev(rows), _dev(x), _dev(psd))
    assert full > 100
    with pytest.raises(N.RBError) as e:
        api.rb_filter_plain(d, _dev(rows), _dev(x), _dev(psd), capacity=10)
    assert e.value.code == N.RB_ERR_OVERFLOW
    # no triggers at an unreachable threshold
    d2 = api.make_desc(g.fs, n, 1, T, w=1, rho_ii=1e6)
    assert api.rb_filter_plain(d2, _dev(rows), _dev(x), _dev(psd))[1] == 0
    # a negative PSD bin is rejected
    bad = psd.copy()
    bad[100] = -1.0
    with pytest.raises(N.RBError) as e:
        api.rb_whiten(d, _dev(x), _dev(bad))
    assert e.value.code == N.RB_ERR_BAD_INPUT
    # too small a workspace
    with pytest.raises(N.RBError) as e:
        api.rb_whiten(d, _dev(x), _dev(psd), ws=torch.empty(1024, dtype=torch.uint8, device="cuda"))
    assert e.value.code == N.RB_ERR_OOM


@pytest.mark.parametrize("n,w", [(1 << 16, 8), (1 << 19, 2), (1 << 19, 16)])
def test_fft_variants_identical(api, n, w):
    """Every FFT schedule variant runs the same per-column arithmetic, so the basis series and
    bin averages are bit-identical across variants; the tuner picks one of them."""
    from paper_2110_13115_gb300 import _native as N

    k = 20
    g, psd, x = _strain(n, seed=4)
    P = inputs.unit_rows(k, n // 2, seed=41).astype(np.complex64)
    d = api.make_desc(g.fs, n, k, 4, w=w)
    basis = api.Basis(_dev(P), _dev(_rand_coeff(4, k, 42).astype(np.complex64)), n)
    ws = api.workspace(d)
    sh = api.rb_whiten(d, _dev(x), _dev(psd), ws=ws)
    outs = []
    for v in range(N.RB_FFT_VARIANTS):
        api.rb_set_fft_variant(d, v)
        beta, bavg = api.rb_basis_filter(d, basis, sh, ws=ws)
        outs.append((beta.cpu().numpy(), bavg.cpu().numpy()))
    for beta, bavg in outs[1:]:
        assert np.array_equal(beta, outs[0][0]) and np.array_equal(bavg, outs[0][1])
    chosen, times = api.rb_tune_fft(d, basis, sh, ws=ws)
    assert 0 <= chosen < N.RB_FFT_VARIANTS and all(t > 0 for t in times)
    assert times[chosen] == min(times)
    api.rb_set_fft_variant(d, 0)


def test_stage2_order_independent_and_hot_bins(api):
    """The bucketing accepts candidates in any order, and a bin holding thousands of candidates is cut
    into several work pieces: the triggers are bit-identical whatever the order and agree with the
    oracle."""
    n, k, T, w = 1 << 14, 24, 3000, 8
    half, nb = n // 2, n // (2 * w)
    a = _rand_coeff(T, k, 13).astype(np.complex64)
    beta = inputs.complex_normal((k, half), 14).astype(np.complex64)
    rng = np.random.default_rng(15)
    hot = np.zeros(T, dtype=api.CANDIDATE_NP)  # every template in one bin: six pieces of <= 512
    hot["tmpl"] = np.arange(T)
    hot["bin"] = nb + 37
    rest = np.zeros(700, dtype=api.CANDIDATE_NP)
    rest["tmpl"] = rng.integers(0, T, 700)
    rest["bin"] = nb + rng.integers(0, nb, 700)
    cands = np.unique(np.concatenate([hot, rest]))
    d = api.make_desc(1024.0, n, k, T, w=w, rho_ii=2.0, cand_capacity=1 << 14)
    basis = api.Basis(_dev(np.zeros((k, half), np.complex64)), _dev(a), n)
    api.rb_pack_coeff(d, basis)
    outs = []
    for order in (np.arange(len(cands)), rng.permutation(len(cands))):
        c = np.ascontiguousarray(cands[order])
        buf, nt = api.rb_stage2(d, basis, _dev(beta), _dev(c.view(np.uint8)), len(c), capacity=1 << 14)
        outs.append(api.triggers_numpy(buf, nt))
    for f in ("tmpl", "sample", "snr", "phase"):
        assert np.array_equal(outs[0][f], outs[1][f]), f
    full = np.zeros((k, n), np.complex128)
    full[:, half:] = beta
    oc = np.zeros(len(cands), dtype=rb.CAND_DTYPE)
    oc["template"] = cands["tmpl"]
    oc["bin"] = cands["bin"]
    ref = rb.stage2(a.astype(np.complex128), full, oc, w, 2.0)
    zr = np.abs(np.conj(a.astype(np.complex128)) @ beta.astype(np.complex128))
    stats = compare_triggers(outs[0], ref, w, 2.0, ref_rho=zr)
    assert stats["both"] > 500


@pytest.mark.parametrize("w", [1, 8, 16])
def test_stage2_coefficient_ring_depths(api, w):
    """The second stage's coefficient fragments reach the products either straight into registers or
    through each lane's cp.async ring in shared memory (2 to 4 slots): the triggers are bit-identical
    for every depth, on a hot bin (several pieces) and scattered candidates, and agree with the oracle."""
    from paper_2110_13115_gb300 import _native as N

    lib = N.load()
    n, k, T = 1 << 14, 72, 1500
    half, nb = n // 2, n // (2 * w)
    a = _rand_coeff(T, k, 61).astype(np.complex64)
    beta = inputs.complex_normal((k, half), 62).astype(np.complex64)
    rng = np.random.default_rng(63)
    hot = np.zeros(T, dtype=api.CANDIDATE_NP)
    hot["tmpl"] = np.arange(T)
    hot["bin"] = nb + 11
    rest = np.zeros(900, dtype=api.CANDIDATE_NP)
    rest["tmpl"] = rng.integers(0, T, 900)
    rest["bin"] = nb + rng.integers(0, nb, 900)
    cands = np.unique(np.concatenate([hot, rest]))
    d = api.make_desc(1024.0, n, k, T, w=w, rho_ii=1.5, cand_capacity=1 << 14)
    basis = api.Basis(_dev(np.zeros((k, half), np.complex64)), _dev(a), n)
    api.rb_pack_coeff(d, basis)
    depths = (0, 2, 3, 4) if w == 8 else (0, 3)
    outs = []
    try:
        for depth in depths:
            assert lib.rbx_set_stage2_ring(depth) == 0
            buf, nt = api.rb_stage2(d, basis, _dev(beta), _dev(cands.view(np.uint8)), len(cands), capacity=1 << 15)
            outs.append(api.triggers_numpy(buf, nt))
    finally:
        lib.rbx_set_stage2_ring(3)
    assert lib.rbx_set_stage2_ring(5) == N.RB_ERR_BAD_INPUT
    for o in outs[1:]:
        assert len(o) == len(outs[0])
        for f in ("tmpl", "sample", "snr", "phase", "block"):
            assert np.array_equal(o[f], outs[0][f]), f
    full = np.zeros((k, n), np.complex128)
    full[:, half:] = beta
    oc = np.zeros(len(cands), dtype=rb.CAND_DTYPE)
    oc["template"] = cands["tmpl"]
    oc["bin"] = cands["bin"]
    ref = rb.stage2(a.astype(np.complex128), full, oc, w, 1.5)
    zr = np.abs(np.conj(a.astype(np.complex128)) @ beta.astype(np.complex128))
    stats = compare_triggers(outs[0], ref, w, 1.5, ref_rho=zr)
    assert stats["both"] > 500, stats


def test_bucketing_window_and_fallback(api):
    """Bucketing histograms each chunk of consecutive candidates over a 1024-group window from the
    chunk's smallest group; groups beyond it take the per-candidate path. With 8192 valid bins (4096
    groups of two for the tcgen05 second stage), candidates in bin order keep every chunk inside its
    window, a random order sends about three quarters of each chunk's candidates down the other path:
    both orders give bit-identical triggers, which agree with the oracle."""
    n, k, T, w = 1 << 17, 24, 2000, 8
    half, nb = n // 2, n // (2 * w)
    assert nb == 8192
    a = _rand_coeff(T, k, 41).astype(np.complex64)
    beta = inputs.complex_normal((k, half), 42).astype(np.complex64)
    rng = np.random.default_rng(43)
    cands = np.zeros(12000, dtype=api.CANDIDATE_NP)
    cands["tmpl"] = rng.integers(0, T, len(cands))
    cands["bin"] = nb + rng.integers(0, nb, len(cands))
    cands = np.unique(cands)
    d = api.make_desc(1024.0, n, k, T, w=w, rho_ii=2.0, cand_capacity=1 << 15)
    basis = api.Basis(_dev(np.zeros((k, half), np.complex64)), _dev(a), n)
    api.rb_pack_coeff(d, basis)
    by_bin = np.argsort(cands["bin"], kind="stable")
    outs = []
    for order in (by_bin, rng.permutation(len(cands))):
        c = np.ascontiguousarray(cands[order])
        buf, nt = api.rb_stage2(d, basis, _dev(beta), _dev(c.view(np.uint8)), len(c), capacity=1 << 15)
        outs.append(api.triggers_numpy(buf, nt))
    assert len(outs[0]) == len(outs[1])
    for f in ("tmpl", "sample", "snr", "phase"):
        assert np.array_equal(outs[0][f], outs[1][f]), f
    full = np.zeros((k, n), np.complex128)
    full[:, half:] = beta
    oc = np.zeros(len(cands), dtype=rb.CAND_DTYPE)
    oc["template"] = cands["tmpl"]
    oc["bin"] = cands["bin"]
    ref = rb.stage2(a.astype(np.complex128), full, oc, w, 2.0)
    zr = np.abs(np.conj(a.astype(np.complex128)) @ beta.astype(np.complex128))
    stats = compare_triggers(outs[0], ref, w, 2.0, ref_rho=zr)
    assert stats["both"] > 1000


def _runs(T, nb, rng, max_len=40):
    """Candidates as the first stage writes them for clustered triggers: per template, runs of
    consecutive (or every-other) bins in increasing order, starting anywhere, so runs cross the
    second stage's bin groups at every offset."""
    tm, bn = [], []
    for t in range(T):
        for _ in range(int(rng.integers(1, 4))):
            step = int(rng.integers(1, 3))
            length = int(rng.integers(1, max_len))
            start = int(rng.integers(0, nb - step * length))
            tm.append(np.full(length, t))
            bn.append(nb + start + step * np.arange(length))
    return np.concatenate(tm), np.concatenate(bn)


@pytest.mark.parametrize("mode", [16, 32])
@pytest.mark.parametrize("w", [1, 2, 4, 8])
def test_stage2_tc_bin_groups(api, w, mode):
    """The tcgen05 second stage buckets by groups of mode / w bins (16 at most; w = 1 with 32-sample
    groups takes the mma.sync kernel): a run of one template over increasing bins of a group becomes
    one record with a bin mask, whose coefficient row is gathered once. The
    triggers are bit-identical whatever the candidate order (runs intact, shuffled, a run reversed, a
    candidate repeated next to itself, which only repeats its triggers), agree with the oracle, and
    with the per-bin mma.sync second stage within its rounding."""
    from paper_2110_13115_gb300 import _native as N

    lib = N.load()
    n, k, T = 1 << 14, 40, 300
    half, nb = n // 2, n // (2 * w)
    a = _rand_coeff(T, k, 51).astype(np.complex64)
    beta = inputs.complex_normal((k, half), 52).astype(np.complex64)
    rng = np.random.default_rng(53)
    tm, bn = _runs(T, nb, rng, max_len=min(40, nb // 4))
    cands = np.zeros(len(tm), dtype=api.CANDIDATE_NP)
    cands["tmpl"], cands["bin"] = tm, bn
    _, first = np.unique(np.stack([tm, bn], 1), axis=0, return_index=True)
    cands = cands[np.sort(first)]  # one candidate per (template, bin), runs in emission order
    odd = np.concatenate([cands[:9][::-1], cands[9:20], cands[20:21], cands[20:]])
    d = api.make_desc(1024.0, n, k, T, w=w, rho_ii=1.5, cand_capacity=1 << 16)
    basis = api.Basis(_dev(np.zeros((k, half), np.complex64)), _dev(a), n)
    api.rb_pack_coeff(d, basis)

    def run(c, tc):
        assert lib.rbx_set_stage2_tc(mode if tc else 0) == 0
        c = np.ascontiguousarray(c)
        buf, nt = api.rb_stage2(d, basis, _dev(beta), _dev(c.view(np.uint8)), len(c), capacity=1 << 16)
        return api.triggers_numpy(buf, nt)

    try:
        got = run(cands, 1)
        shuffled = run(cands[rng.permutation(len(cands))], 1)
        odd_tc = run(odd, 1)
        mma = run(cands, 0)
    finally:
        lib.rbx_set_stage2_tc(1)
    assert len(shuffled) == len(got)
    for f in ("tmpl", "sample", "snr", "phase", "block"):
        assert np.array_equal(shuffled[f], got[f]), f
    keys = lambda o: list(zip(o["tmpl"].tolist(), o["sample"].tolist(), o["snr"].tolist()))  # noqa: E731
    rep = (int(cands[20]["tmpl"]), int(cands[20]["bin"]))
    extra = sum(1 for t, smp, _ in keys(got) if (t, smp // w) == rep)
    assert len(odd_tc) == len(got) + extra
    assert set(keys(odd_tc)) == set(keys(got))
    full = np.zeros((k, n), np.complex128)
    full[:, half:] = beta
    oc = np.zeros(len(cands), dtype=rb.CAND_DTYPE)
    oc["template"] = cands["tmpl"]
    oc["bin"] = cands["bin"]
    ref = rb.stage2(a.astype(np.complex128), full, oc, w, 1.5)
    zr = np.abs(np.conj(a.astype(np.complex128)) @ beta.astype(np.complex128))
    stats = compare_triggers(got, ref, w, 1.5, ref_rho=zr)
    assert stats["both"] > 1000, stats
    ref2 = np.zeros(len(mma), dtype=mf.TRIGGER_DTYPE)
    ref2["template"], ref2["sample"], ref2["snr"], ref2["phase"] = mma["tmpl"], mma["sample"], mma["snr"], mma["phase"]
    compare_triggers(got, ref2, w, 1.5, ref_rho=zr)


def test_stage2_tc_many_pieces_per_cta(api):
    """Hundreds of bin groups with 1 to 700 records each: every CTA of the persistent tcgen05 second
    stage takes several pieces of one to four tiles, so each tensor-memory slot is reused after pieces
    that left it idle. The triggers agree with the per-bin mma.sync second stage within its rounding."""
    from paper_2110_13115_gb300 import _native as N

    lib = N.load()
    n, k, T, w = 1 << 15, 201, 1200, 8
    half, nb = n // 2, n // (2 * w)
    a = _rand_coeff(T, k, 71).astype(np.complex64)
    beta = inputs.complex_normal((k, half), 72).astype(np.complex64)
    rng = np.random.default_rng(73)
    groups = rng.choice(nb // 2, size=600, replace=False)
    tm, bn = [], []
    for grp in np.sort(groups):
        ts = np.sort(rng.choice(T, size=int(rng.integers(1, 701)), replace=False))
        for t in ts:  # one or both bins of the group, in bin order (a run)
            for b in ((0,), (1,), (0, 1))[int(rng.integers(0, 3))]:
                tm.append(t)
                bn.append(nb + 2 * grp + b)
    cands = np.zeros(len(tm), dtype=api.CANDIDATE_NP)
    cands["tmpl"], cands["bin"] = tm, bn
    d = api.make_desc(1024.0, n, k, T, w=w, rho_ii=2.0, cand_capacity=1 << 20)
    basis = api.Basis(_dev(np.zeros((k, half), np.complex64)), _dev(a), n)
    api.rb_pack_coeff(d, basis)
    outs = []
    try:
        for tc in (1, 0):
            lib.rbx_set_stage2_tc(tc)
            buf, nt = api.rb_stage2(d, basis, _dev(beta), _dev(cands.view(np.uint8)), len(cands), capacity=1 << 20)
            outs.append(api.triggers_numpy(buf, nt))
    finally:
        lib.rbx_set_stage2_tc(1)
    got, mma = outs
    zr = np.abs(np.conj(a.astype(np.complex128)) @ beta.astype(np.complex128))
    ref = np.zeros(len(mma), dtype=mf.TRIGGER_DTYPE)
    ref["template"], ref["sample"], ref["snr"], ref["phase"] = mma["tmpl"], mma["sample"], mma["snr"], mma["phase"]
    stats = compare_triggers(got, ref, w, 2.0, ref_rho=zr)
    assert stats["both"] > 50000, stats


@pytest.mark.parametrize("w", [1, 2, 4, 8])
@pytest.mark.parametrize("k", [24, 40, 256, 400])
def test_stage2_tc_parity(api, w, k):
    """The tcgen05 second stage (tiles of 128 records of a group of 16 / w bins, hi and lo windows side
    by side in one N = 64 operand, two products per K step) against the oracle and against the
    mma.sync second stage on the same candidates, including a hot bin of several tiles. k = 256 and
    below leave room for a 3-stage coefficient ring; at k = 400 the windows leave too little, and the
    call takes the mma.sync kernel."""
    from paper_2110_13115_gb300 import _native as N

    lib = N.load()
    n, T = 1 << 14, 700
    half, nb = n // 2, n // (2 * w)
    a = _rand_coeff(T, k, 31).astype(np.complex64)
    beta = inputs.complex_normal((k, half), 32).astype(np.complex64)
    rng = np.random.default_rng(33)
    hot = np.zeros(T, dtype=api.CANDIDATE_NP)
    hot["tmpl"] = np.arange(T)
    hot["bin"] = nb + 5
    rest = np.zeros(600, dtype=api.CANDIDATE_NP)
    rest["tmpl"] = rng.integers(0, T, 600)
    rest["bin"] = nb + rng.integers(0, nb, 600)
    cands = np.unique(np.concatenate([hot, rest]))
    rho_ii = 1.5  # unit-norm coefficients: |z| is Rayleigh-distributed with scale 1 on these beta
    d = api.make_desc(1024.0, n, k, T, w=w, rho_ii=rho_ii, cand_capacity=1 << 14)
    basis = api.Basis(_dev(np.zeros((k, half), np.complex64)), _dev(a), n)
    api.rb_pack_coeff(d, basis)
    outs = []
    try:
        for tc in (1, 0):
            lib.rbx_set_stage2_tc(tc)
            buf, nt = api.rb_stage2(d, basis, _dev(beta), _dev(cands.view(np.uint8)), len(cands), capacity=1 << 14)
            outs.append(api.triggers_numpy(buf, nt))
    finally:
        lib.rbx_set_stage2_tc(1)
    got, mma = outs
    full = np.zeros((k, n), np.complex128)
    full[:, half:] = beta
    oc = np.zeros(len(cands), dtype=rb.CAND_DTYPE)
    oc["template"] = cands["tmpl"]
    oc["bin"] = cands["bin"]
    ref = rb.stage2(a.astype(np.complex128), full, oc, w, rho_ii)
    zr = np.abs(np.conj(a.astype(np.complex128)) @ beta.astype(np.complex128))
    stats = compare_triggers(got, ref, w, rho_ii, ref_rho=zr)
    assert stats["both"] > 100, stats
    ref2 = np.zeros(len(mma), dtype=mf.TRIGGER_DTYPE)
    ref2["template"], ref2["sample"], ref2["snr"], ref2["phase"] = mma["tmpl"], mma["sample"], mma["snr"], mma["phase"]
    compare_triggers(got, ref2, w, rho_ii, ref_rho=zr)


@pytest.mark.parametrize("n,w", [(1 << 16, 8), (1 << 17, 16), (1 << 18, 1), (1 << 19, 8), (1 << 20, 16), (1 << 20, 4)])
def test_radix32_passes_vs_radix16_and_oracle(api, n, w):
    """The radix-32 four-step passes (every n >= 2^16) against the radix-16 passes and the FP64 oracle:
    basis series, bin means and template-method triggers."""
    from paper_2110_13115_gb300 import _native as N

    k, T = 6, 5
    g, psd, x = _strain(n, fs=2048.0, seed=6)
    half = n // 2
    P = inputs.unit_rows(k, half, seed=61).astype(np.complex64)
    d = api.make_desc(g.fs, n, k, 1, w=w)
    basis = api.Basis(_dev(P), _dev(np.ones((1, k), np.complex64)), n)
    ws = api.workspace(d)
    sh = api.rb_whiten(d, _dev(x), _dev(psd), ws=ws)
    out = {}
    try:
        for r32 in (4, 3, 2, 1, 0):  # radix-32 variants 3..0, then the radix-16 passes
            N.load().rbx_set_fft_radix32(r32)
            beta, bavg = api.rb_basis_filter(d, basis, sh, ws=ws)
            out[r32] = (beta.cpu().numpy(), bavg.cpu().numpy())
    finally:
        N.load().rbx_set_fft_radix32(4)
    s_fd = mf.strain_fd(x.astype(np.float64), g.fs)
    ref = rb.basis_series(s_fd, psd, P.astype(np.complex128), n, g.fs)
    rref = ref[:, half:]
    scale = np.sqrt(np.mean(np.abs(rref) ** 2))
    aref = rb.bin_average(ref, w)[:, n // (2 * w):]
    for r32, (beta, bavg) in out.items():
        assert np.abs(beta - rref).max() / scale < 3e-5, r32
        assert np.abs(bavg - aref).max() / scale < 3e-5, r32
    assert np.abs(out[4][0] - out[0][0]).max() / scale < 3e-5
    # the staged stores change no arithmetic: variants with and without them agree bit for bit
    assert np.array_equal(out[4][0], out[2][0]) and np.array_equal(out[3][0], out[1][0])
    # the template method through the same passes (rows as unit-norm templates)
    rho_ii = 3.0
    dp = api.make_desc(g.fs, n, 1, k, w=w, rho_ii=rho_ii)
    buf, nt = api.rb_filter_plain(dp, _dev(P), _dev(x), _dev(psd))
    got = api.triggers_numpy(buf, nt)
    rho = np.abs(ref)
    tref = np.concatenate([mf.window_triggers(t, rho[t], ref[t], n, w, rho_ii) for t in range(k)])
    stats = compare_triggers(got, tref, w, rho_ii, ref_rho=rho[:, half:])
    assert stats["both"] > 5, stats
