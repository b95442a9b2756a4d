"""Batching (Sec. III.E batches of segments): blocks of uneven segments from two detectors with
per-detector PSD scales and two FFT sizes, several banks concatenated over one basis per FFT size,
filtered by rb_filter_batch and by the recorded CUDA graph (rb_batch_create / rb_batch_run).

Checks: the batch equals block-by-block rb_filter (same kernels, so bit-identical triggers once
each block keeps only its samples from valid_lo on); graph replays equal the eager batch; and
every block agrees with the FP64 oracle's hierarchical pipeline on the same basis."""
import numpy as np
import pytest

from oracle import mf, rb
from paper_2110_13115_gb300 import inputs

from parity_util import compare_triggers

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K, W, RHO_I = 24, 8, 3.2


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_13115_gb300 import api as A, _native as N

    N.load()
    return A


@pytest.fixture(scope="module")
def case(api):
    wl = inputs.batch(n_segments=4, fs=1024.0, f_low=40.0, unit_s=4.0, max_units=10, max_block_s=16.0, n_banks=3,
                      bank_sizes=(30, 60), m_range=(12.0, 30.0), chi_max=0.0, pn_order=2, k=K, w=W,
                      inj_per_segment=1, snr_range=(9.0, 14.0), seed=5)
    assert len(wl.sizes) >= 2
    bank = wl.bank
    T = len(bank)
    descs, bases, where = [], [], {}
    for i, n in enumerate(wl.sizes):
        psd1 = torch.from_numpy(inputs.analytic_psd(inputs.Grid(wl.fs, n, wl.f_low))).cuda()
        b = api.rb_build(api.Bank(bank, wl.fs, n, wl.f_low, wl.bank_spec.pn_order), psd1, K, oversample=64,
                         power_iters=1)
        d = api.make_desc(wl.fs, n, K, T, w=W, precision="fp16_split", rho_i=RHO_I, rho_ii=wl.rho_ii,
                          cand_capacity=1 << 18)
        api.rb_pack_coeff(d, b)
        descs.append(d)
        bases.append(b)
        where[n] = i
    blocks = []
    for j, bb in enumerate(wl.blocks):
        seg = wl.segments[bb.segment]
        blocks.append(api.Block(strain=torch.from_numpy(np.ascontiguousarray(wl.block_strain(bb))).cuda(),
                                psd=torch.from_numpy(wl.block_psd(bb)).cuda(), basis=where[bb.n],
                                sample_offset=seg.start + bb.offset, valid_lo=bb.valid_lo, block_id=j))
    return wl, descs, bases, blocks


def _key_sorted(a):
    return np.sort(a, order=["block", "tmpl", "sample"])


def _per_block(api, wl, descs, bases, blocks):
    out = []
    for j, (bb, blk) in enumerate(zip(wl.blocks, blocks)):
        d = descs[blk.basis]
        dj = api.make_desc(d.fs, d.n, d.k, d.n_templates, w=d.w, precision="fp16_split", rho_i=d.rho_i,
                           rho_ii=d.rho_ii, cand_capacity=d.cand_capacity, sample_offset=blk.sample_offset,
                           block_id=j)
        buf, nt = api.rb_filter(dj, bases[blk.basis], blk.strain, blk.psd, capacity=1 << 18)
        t = api.triggers_numpy(buf, nt)
        out.append(t[t["sample"] - blk.sample_offset >= bb.valid_lo])
    return np.concatenate(out)


def test_batch_equals_block_by_block(api, case):
    wl, descs, bases, blocks = case
    buf, nt = api.rb_filter_batch(descs, bases, blocks, capacity=1 << 20)
    got = _key_sorted(api.triggers_numpy(buf, nt))
    ref = _key_sorted(_per_block(api, wl, descs, bases, blocks))
    assert nt > 0 and len(got) == len(ref)
    for f in ("block", "tmpl", "sample", "snr", "phase"):
        assert np.array_equal(got[f], ref[f]), f
    # every block's triggers lie in its kept range [valid_lo, n)
    for j, bb in enumerate(wl.blocks):
        s = got["sample"][got["block"] == j] - blocks[j].sample_offset
        assert np.all((s >= bb.valid_lo) & (s < bb.n))


def test_graph_replay_equals_eager(api, case):
    wl, descs, bases, blocks = case
    buf, nt = api.rb_filter_batch(descs, bases, blocks, capacity=1 << 20)
    eager = _key_sorted(api.triggers_numpy(buf, nt))
    batch = api.Batch(descs, bases, blocks, capacity=1 << 20)
    try:
        for _ in range(2):
            tb, n2 = batch.run()
            got = _key_sorted(api.triggers_numpy(tb, n2))
            assert n2 == nt
            for f in ("block", "tmpl", "sample", "snr", "phase"):
                assert np.array_equal(got[f], eager[f]), f
    finally:
        batch.close()


def test_batch_blocks_vs_oracle(api, case):
    """Each block against the FP64 oracle pipeline (whitening with the block's scaled PSD, FFT,
    bin average, both stages) on the same basis vectors and coefficients."""
    wl, descs, bases, blocks = case
    buf, nt = api.rb_filter_batch(descs, bases, blocks, capacity=1 << 20)
    got = api.triggers_numpy(buf, nt)
    both = 0
    for j, bb in enumerate(wl.blocks):
        blk = blocks[j]
        n, half = bb.n, bb.n // 2
        P = bases[blk.basis].vectors.cpu().numpy().astype(np.complex128)
        a = bases[blk.basis].coeff.cpu().numpy().astype(np.complex128)
        psd = wl.block_psd(bb)
        s_fd = mf.strain_fd(wl.block_strain(bb).astype(np.float64), wl.fs)
        ref, _, beta = rb.hierarchical_triggers(a, s_fd, psd, P, n, wl.fs, W, RHO_I, wl.rho_ii)
        ref = ref[ref["sample"] >= bb.valid_lo]
        mine = got[got["block"] == j].copy()
        mine["sample"] -= blk.sample_offset
        zfull = np.abs(rb.reconstruct(a, beta[:, half:]))
        ravg = np.abs(rb.reconstruct(a, rb.bin_average(beta, W)[:, n // (2 * W):]))
        stats = compare_triggers(mine, ref, W, wl.rho_ii, ref_rho=zfull, rho_avg=ravg, rho_i=RHO_I)
        both += stats["both"]
    assert both >= 10


def test_batch_fp32_wide_bins_equals_block_by_block(api, case):
    """The same work list with the FP32 first stage and w = 16 (one basis per size reused)."""
    wl, descs, bases, blocks = case
    d2 = [api.make_desc(d.fs, d.n, d.k, d.n_templates, w=16, precision="fp32", rho_i=RHO_I / 1.2,
                        rho_ii=d.rho_ii, cand_capacity=1 << 18) for d in descs]
    for d, b in zip(d2, bases):
        api.rb_pack_coeff(d, b)
    try:
        buf, nt = api.rb_filter_batch(d2, bases, blocks, capacity=1 << 20)
        got = _key_sorted(api.triggers_numpy(buf, nt))
        ref = []
        for j, (bb, blk) in enumerate(zip(wl.blocks, blocks)):
            d = d2[blk.basis]
            dj = api.make_desc(d.fs, d.n, d.k, d.n_templates, w=16, precision="fp32", rho_i=d.rho_i,
                               rho_ii=d.rho_ii, cand_capacity=d.cand_capacity, sample_offset=blk.sample_offset,
                               block_id=j)
            b2, n2 = api.rb_filter(dj, bases[blk.basis], blk.strain, blk.psd, capacity=1 << 18)
            t = api.triggers_numpy(b2, n2)
            ref.append(t[t["sample"] - blk.sample_offset >= bb.valid_lo])
        ref = _key_sorted(np.concatenate(ref))
        assert nt > 0 and len(got) == len(ref)
        for f in ("block", "tmpl", "sample", "snr", "phase"):
            assert np.array_equal(got[f], ref[f]), f
    finally:
        for d, b in zip(descs, bases):  # restore the packing the other tests use
            api.rb_pack_coeff(d, b)


def test_batch_rejects_bad_blocks(api, case):
    from paper_2110_13115_gb300 import _native as N

    wl, descs, bases, blocks = case
    bad = [api.Block(blocks[0].strain, blocks[0].psd, basis=len(descs), valid_lo=None)]
    with pytest.raises(N.RBError) as e:
        api.rb_filter_batch(descs, bases, bad)
    assert e.value.code == N.RB_ERR_BAD_INPUT
    b0 = blocks[0]
    n = descs[b0.basis].n
    for lo in (n // 2 - W, n, n // 2 + 3):
        with pytest.raises(N.RBError) as e:
            api.rb_filter_batch(descs, bases, [api.Block(b0.strain, b0.psd, basis=b0.basis, valid_lo=lo)])
        assert e.value.code == N.RB_ERR_BAD_INPUT
    # a block's candidate overflow is reported once the whole batch has run
    tight = [api.make_desc(d.fs, d.n, d.k, d.n_templates, w=d.w, precision="fp16_split", rho_i=0.0,
                           rho_ii=d.rho_ii, cand_capacity=16) for d in descs]
    with pytest.raises(N.RBError) as e:
        api.rb_filter_batch(tight, bases, blocks[:2], capacity=1 << 20)
    assert e.value.code == N.RB_ERR_OVERFLOW
