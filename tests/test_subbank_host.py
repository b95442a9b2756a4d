"""Sub-banks along iso-tau0 lines and the basis size for a tolerance (Sec. III.B, Table I): the host
functions of the C ABI against the values printed in Table I, the FP64 oracle's waveform phase and
its SVD truncation loss (Eq. 8). No GPU is used."""
import json
import os

import numpy as np
import pytest

from oracle import rb, waveform as W
from paper_2110_13115_gb300 import inputs

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def api():
    from paper_2110_13115_gb300 import _native as N, api as A, build

    if not os.path.exists(N.LIB_PATH):
        build.build()
    N.load()
    return A


def _bank(params, f_low=30.0):
    from paper_2110_13115_gb300 import api as A

    return A.Bank(np.asarray(params, dtype=np.float64), 2048.0, 1 << 16, f_low, 0)


def test_tau0_table1_corners(api):
    """The case-study sub-bank's corners reproduce the tau0 range printed in Table I."""
    g = json.load(open(os.path.join(GOLD, "table1_tau0.json")))
    params = []
    for c in g["corners"]:
        mt, q = c["total_mass"], c["mass_ratio"]
        params.append((mt * q / (1 + q), mt / (1 + q), 0.0, 0.0))
    tau0 = api.rb_bank_tau0(_bank(params), g["f0_hz"])
    for t, c in zip(tau0, g["corners"]):
        assert abs(t / c["tau0_s"] - 1) < g["rel_tol"], (t, c)


def test_tau0_is_the_newtonian_phase_slope(api):
    """tau0 equals -(1/2 pi) dPsi/df of the oracle's Newtonian (0PN) phase at f0, for random masses."""
    rng = np.random.default_rng(7)
    m = rng.uniform(1.0, 60.0, size=(40, 2))
    params = np.column_stack([m.max(1), m.min(1), np.zeros(40), np.zeros(40)])
    f0 = 25.0
    tau0 = api.rb_bank_tau0(_bank(params), f0)
    h = 1e-5 * f0
    for (m1, m2, _, _), t in zip(params, tau0):
        d = (W.phase(f0 + h, m1, m2, pn_order=0) - W.phase(f0 - h, m1, m2, pn_order=0)) / (2 * h)
        assert abs(t / (-d / (2 * np.pi)) - 1) < 1e-6, (m1, m2, t)


def test_tau0_scaling(api):
    """tau0 ~ Mc^(-5/3) f0^(-8/3): doubling f0 divides it by 2^(8/3); equal-mass doubling of M by 2^(5/3)."""
    b = _bank([(10.0, 10.0, 0, 0), (20.0, 20.0, 0, 0)])
    a, c = api.rb_bank_tau0(b, 20.0), api.rb_bank_tau0(b, 40.0)
    np.testing.assert_allclose(a / c, 2.0 ** (8 / 3), rtol=1e-12)
    np.testing.assert_allclose(a[0] / a[1], 2.0 ** (5 / 3), rtol=1e-12)


def test_split_is_an_ordered_equal_count_partition(api):
    rng = np.random.default_rng(8)
    tau0 = np.round(rng.uniform(1.0, 100.0, 1003), 1)  # ties included
    for parts in (1, 2, 7, 64, 1003):
        order, offsets = api.rb_bank_split_tau0(tau0, parts)
        assert sorted(order.tolist()) == list(range(len(tau0)))
        assert offsets[0] == 0 and offsets[-1] == len(tau0)
        sizes = np.diff(offsets)
        assert sizes.min() >= len(tau0) // parts and sizes.max() - sizes.min() <= 1
        t = tau0[order]
        assert np.all(np.diff(t) >= 0)
        for p in range(parts - 1):  # every tau0 of part p <= every tau0 of part p + 1
            assert t[offsets[p]:offsets[p + 1]].max() <= t[offsets[p + 1]:offsets[p + 2]].min()
        ties = order[np.r_[False, np.diff(t) == 0]]  # equal tau0 keep their index order
        prev = order[np.r_[np.diff(t) == 0, False]]
        assert np.all(prev < ties)


def test_k_for_loss_matches_oracle_truncation(api):
    """On a bank's unit-normalised whitened templates, the chosen k is the first whose Eq. 8 loss (the
    oracle's, from all singular values of an exact SVD) is <= tol, and the reported loss is that loss."""
    g = inputs.Grid(fs=512.0, n=4096, f_low=30.0)
    psd = inputs.analytic_psd(g)
    bank = inputs.draw_bank(inputs.BankSpec(48, 8.0, 20.0, 0.0, 2))
    hs = W.bank_templates(bank, g.fs, g.n, g.f_low, 2)
    ghat, _ = rb.whitened_rows(hs, psd, g.n, g.fs)
    _, s, _ = rb.svd_basis(ghat, len(bank))
    T = len(bank)
    for tol in (0.3, 0.1, 1e-2, 1e-3, 1e-4):
        k, loss = api.rb_basis_k_for_loss(s[:40], T, tol)
        assert rb.truncation_loss(s, k) <= tol
        assert k == 1 or rb.truncation_loss(s, k - 1) > tol
        assert abs(loss - rb.truncation_loss(s, k)) < 1e-12


def test_k_for_loss_errors(api):
    from paper_2110_13115_gb300 import _native as N

    sv = np.sqrt(np.array([4.0, 2.0, 1.0]))  # T = 8: losses 0.5, 0.25, 0.125
    assert api.rb_basis_k_for_loss(sv, 8, 0.25) == (2, 0.25)
    with pytest.raises(N.RBError) as e:
        api.rb_basis_k_for_loss(sv, 8, 0.1)
    assert e.value.code == N.RB_ERR_UNSUPPORTED
    for bad in (np.array([1.0, 2.0]), np.array([3.0, 3.0])):  # not descending; sum sv^2 > T
        with pytest.raises(N.RBError) as e:
            api.rb_basis_k_for_loss(bad, 8, 0.1)
        assert e.value.code == N.RB_ERR_BAD_INPUT
    with pytest.raises(N.RBError) as e:
        api.rb_bank_split_tau0(np.ones(3), 4)
    assert e.value.code == N.RB_ERR_BAD_INPUT
    with pytest.raises(N.RBError) as e:
        api.rb_bank_tau0(_bank([(1.0, -1.0, 0, 0)]), 30.0)
    assert e.value.code == N.RB_ERR_BAD_INPUT


def test_banks_plan_shares_one_workspace(api):
    """rb_banks_plan (host only): the workspace of the largest sub-bank, the host trigger staging region
    only when the descriptors ask for host triggers (at an n-only offset, so every sub-bank finds it in
    place), and descriptors that differ in n, w or mem are rejected."""
    from paper_2110_13115_gb300 import _native as N

    fs, n = 2048.0, 1 << 19
    ds = [api.make_desc(fs, n, k, 2500, w=8, precision="fp16_split_a", cand_capacity=1 << 22) for k in (201, 106, 85)]
    one = [api.rb_filter_plan(d).workspace_bytes for d in ds]
    plan = api.rb_banks_plan(ds)
    assert plan.workspace_bytes == max(one)
    assert plan.host_trig_capacity == (96 << 20) // 24
    hs = [N.rb_filter_desc.from_buffer_copy(d) for d in ds]
    for h in hs:
        h.mem = N.RB_MEM_HOST_STRAIN | N.RB_MEM_HOST_TRIGGERS
    assert api.rb_banks_plan(hs).workspace_bytes == plan.workspace_bytes + (96 << 20)
    odd = N.rb_filter_desc.from_buffer_copy(ds[1])
    odd.w = 4
    with pytest.raises(N.RBError):
        api.rb_banks_plan([ds[0], odd])
    odd = N.rb_filter_desc.from_buffer_copy(ds[1])
    odd.mem = N.RB_MEM_HOST_TRIGGERS
    with pytest.raises(N.RBError):
        api.rb_banks_plan([ds[0], odd])
