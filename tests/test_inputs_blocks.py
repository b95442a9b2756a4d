"""Host logic of the batch work list (no GPU): every segment's samples from its first block's valid
half onwards are covered by exactly one block's kept range, blocks are powers of two that overlap by
half, and a right-aligned tail keeps only what its predecessor did not cover."""
import numpy as np
import pytest

from paper_2110_13115_gb300 import inputs


@pytest.mark.parametrize("length_units", list(range(1, 17)))
def test_segment_blocks_cover_each_valid_sample_once(length_units):
    fs, unit = 2048, 32 * 2048
    length, max_block = length_units * unit, 128 * fs
    blocks = inputs.segment_blocks(length, max_block)
    n = blocks[0][1]
    assert all(b[1] == n for b in blocks)
    assert n & (n - 1) == 0 and n <= min(length, max_block) < 2 * n
    cover = np.zeros(length, np.int32)
    for off, nb, lo in blocks:
        assert nb // 2 <= lo < nb and lo % 8 == 0 and off + nb <= length
        cover[off + lo:off + nb] += 1
    # the first half of the first block is the filter's warm-up: everything after it exactly once
    assert np.all(cover[:n // 2] == 0)
    assert np.all(cover[n // 2:] == 1)
    # consecutive ordinary blocks overlap by half
    for (o1, _, _), (o2, _, lo2) in zip(blocks, blocks[1:]):
        if lo2 == n // 2:
            assert o2 - o1 == n // 2


def test_batch_workload_layout():
    wl = inputs.batch(n_segments=3, fs=1024.0, f_low=40.0, unit_s=4.0, max_units=10, max_block_s=16.0, n_banks=2,
                      bank_sizes=(10, 20), m_range=(12.0, 30.0), chi_max=0.0, pn_order=2, k=16, inj_per_segment=0)
    assert len(wl.segments) == 6 and {s.detector for s in wl.segments} == {0, 1}
    scales = {s.detector: s.psd_scale for s in wl.segments}
    assert all(0.5 <= v <= 2.0 for v in scales.values())
    assert len(wl.bank) == sum(len(b) for b in wl.banks)
    for b in wl.blocks:
        seg = wl.segments[b.segment]
        assert b.offset + b.n <= len(seg.strain)
        psd = wl.block_psd(b)
        assert psd.shape == (b.n // 2 + 1,) and np.isinf(psd[0]) or psd[0] > 0
    secs = wl.valid_seconds
    assert secs == sum(b.n - b.valid_lo for b in wl.blocks) / wl.fs
