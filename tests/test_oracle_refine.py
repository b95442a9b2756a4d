"""Pins of the oracle's |Z|^2/sigma^2 objective, its gradient and the ascent (no GPU)."""
import json
import os

import numpy as np

from oracle import cost, mf, refine, waveform as W
from paper_2110_13115_gb300 import inputs


def _injected(mc, eta, tc, phic, amp=1.0):
    g = inputs.Grid(fs=1024.0, n=16384, f_low=30.0)
    psd = inputs.analytic_psd(g)
    mt = mc * eta ** -0.6
    m1 = mt * (1 + np.sqrt(1 - 4 * eta)) / 2
    m2 = mt - m1
    h = W.template((m1, m2, 0, 0), g.fs, g.n, g.f_low, 2, tc=tc, phic=phic)
    return g, psd, amp * h


def test_gradient_matches_finite_differences():
    g, psd, h = _injected(12.0, 0.21, 12.3, 0.5)
    rng = np.random.default_rng(0)
    s_fd = h + 0.05 * (rng.standard_normal(h.size) + 1j * rng.standard_normal(h.size)) * np.abs(h).max()
    th = np.array([12.03, 0.208, 12.3004, 0.1])
    f, ws, amp, sig2 = refine.setup(s_fd, psd, g.fs, g.n, g.f_low, th[0], th[1])
    j0, grad = refine.gradient(th, f, ws, amp, sig2, 2)
    for i in range(3):
        e = np.zeros(4)
        e[i] = 1e-6 * max(abs(th[i]), 1.0)
        jp, _ = refine.objective(th + e, f, ws, amp, sig2, 2)
        jm, _ = refine.objective(th - e, f, ws, amp, sig2, 2)
        fd = (jp - jm) / (2 * e[i])
        assert abs(grad[i] - fd) <= 1e-5 * abs(fd) + 1e-9 * j0 / e[i], (i, grad[i], fd)
    assert grad[3] == 0.0 or abs(grad[3]) < 1e-12 * j0  # |Z| does not depend on phi_c


def test_stationary_at_truth_and_matches_template_method():
    mc, eta, tc = 10.0, 0.24, 12.0
    g, psd, h = _injected(mc, eta, tc, 0.9, amp=0.5)
    th = np.array([mc, eta, tc, 0.0])
    f, ws, amp, sig2 = refine.setup(h, psd, g.fs, g.n, g.f_low, mc, eta)
    j, grad = refine.gradient(th, f, ws, amp, sig2, 2)
    np.testing.assert_allclose(j, 0.25 * sig2, rtol=1e-12)  # J = A^2 sigma^2
    scale = np.array([mc, 1.0, 1.0 / refine.F_REF, 1.0])
    assert np.max(np.abs(grad * scale)) < 1e-6 * j
    # J at an integer-sample t_c equals the template method's |z|^2 / sigma^2
    m = int(tc * g.fs) + 3
    mt = mc * eta ** -0.6
    m1 = mt * (1 + np.sqrt(1 - 4 * eta)) / 2
    z, sig = mf.snr_series(h, W.template((m1, mt - m1, 0, 0), g.fs, g.n, g.f_low, 2), psd, g.n, g.fs)
    jm, _ = refine.objective(np.array([mc, eta, m / g.fs, 0.0]), f, ws, amp, sig2, 2)
    np.testing.assert_allclose(jm, np.abs(z[m]) ** 2 / sig ** 2, rtol=1e-10)


def test_ascent_is_monotone_and_converges():
    mc, eta, tc = 10.0, 0.24, 12.0
    g, psd, h = _injected(mc, eta, tc, 0.9)
    th0 = np.array([mc * 1.002, 0.235, tc + 0.4e-3, 0.0])
    th, j, hist = refine.ascend(th0, h, psd, g.fs, g.n, g.f_low, 2, steps=60)
    assert np.all(np.diff(hist) >= 0)
    f, ws, amp, sig2 = refine.setup(h, psd, g.fs, g.n, g.f_low, th0[0], th0[1])
    assert hist[-1] > hist[0]
    assert j > 0.97 * sig2


def test_throughput_definition_table2():
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "throughput_table2.json")))
    v = cost.throughput(gold["seconds"], gold["templates"], gold["wall_s"])
    assert abs(v / gold["throughput"] - 1) < 1e-12


def test_cost_model_limits():
    n, t = 262144, 6250
    # w = 1 folded first stage is the template method plus the 2 N T averaging term
    assert abs(cost.z_first(n, t, 1) - (cost.z_basic(n, t) + 2 * n * t)) < 1e-3 * cost.z_basic(n, t)
    assert cost.z_first(n, t, 16) < cost.z_first(n, t, 8) < cost.z_basic(n, t)
    assert cost.z_total(n, t, 8, 254, 0.0) > cost.z_first(n, t, 8)
