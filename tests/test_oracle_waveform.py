"""Pins of the oracle's chirp templates (no GPU)."""
import json
import os

import numpy as np
import pytest

from oracle import waveform as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _tau_textbook(f, m1, m2, chi1, chi2, order):
    """Stationary-phase time before coalescence (textbook PN series, through 1.5PN):
    tau = 5 M/(256 eta) v^-8 [1 + (4/3)(743/336 + 11 eta/4) v^2 - (8/5)(4 pi - beta) v^3]."""
    m = m1 + m2
    eta = m1 * m2 / m ** 2
    ms = m * W.MSUN_S
    beta = (chi1 * (113 * (m1 / m) ** 2 + 75 * eta) + chi2 * (113 * (m2 / m) ** 2 + 75 * eta)) / 12
    v = (np.pi * ms * f) ** (1 / 3)
    series = 1.0
    if order >= 2:
        series = series + 4 / 3 * (743 / 336 + 11 / 4 * eta) * v ** 2
    if order >= 3:
        series = series - 8 / 5 * (4 * np.pi - beta) * v ** 3
    return 5 * ms / (256 * eta) * v ** -8 * series


@pytest.mark.parametrize("order", [0, 2, 3])
@pytest.mark.parametrize("params", [(1.4, 1.3, 0.0, 0.0), (30.0, 5.0, 0.4, -0.3), (12.0, 11.0, -0.5, 0.5)])
def test_stationary_phase_relation(order, params):
    """dPsi/df = 2 pi (t_c - tau(f)) with the textbook tau(f) series."""
    m1, m2, c1, c2 = params
    tc = 3.25
    f = np.linspace(20.0, 0.9 * W.f_isco(m1, m2), 50)
    h = 1e-4 * f
    dpsi = (W.phase(f + h, m1, m2, c1, c2, tc, 0.7, order) - W.phase(f - h, m1, m2, c1, c2, tc, 0.7, order)) / (2 * h)
    expect = 2 * np.pi * (tc - _tau_textbook(f, m1, m2, c1, c2, order))
    np.testing.assert_allclose(dpsi, expect, rtol=1e-6, atol=1e-7 * np.abs(expect).max())


def test_table1_newtonian_chirp_time():
    """Case-study sub-bank corners reproduce the tau0 range printed in Table I."""
    g = json.load(open(os.path.join(GOLD, "table1_tau0.json")))
    f0 = g["f0_hz"]
    for c in g["corners"]:
        mt, q = c["total_mass"], c["mass_ratio"]
        m1, m2 = mt * q / (1 + q), mt / (1 + q)
        h = 1e-5
        d = (W.phase(f0 + h, m1, m2, pn_order=0) - W.phase(f0 - h, m1, m2, pn_order=0)) / (2 * h)
        tau0 = -d / (2 * np.pi)
        assert abs(tau0 / c["tau0_s"] - 1) < g["rel_tol"], (c, tau0)


def test_spin_exchange_symmetry():
    f = np.linspace(30, 300, 20)
    a = W.phase(f, 20.0, 8.0, 0.3, -0.2, 0.0, 0.0, 3)
    b = W.phase(f, 8.0, 20.0, -0.2, 0.3, 0.0, 0.0, 3)
    np.testing.assert_allclose(a, b, rtol=1e-14)
    # the spin term is not symmetric under exchanging only the spins
    c = W.phase(f, 20.0, 8.0, -0.2, 0.3, 0.0, 0.0, 3)
    assert np.max(np.abs(a - c)) > 1e-3


def test_time_shift_and_isco():
    fs, n = 1024.0, 4096
    p = (15.0, 12.0, 0.0, 0.0)
    h0 = W.template(p, fs, n, 30.0, 2)
    h1 = W.template(p, fs, n, 30.0, 2, tc=0.37, phic=0.4)
    f = np.arange(n // 2 + 1) * fs / n
    np.testing.assert_allclose(h1, h0 * np.exp(-2j * np.pi * f * 0.37 + 0.4j), atol=1e-14)
    # f_isco ~ 4.4 kHz for one solar mass (textbook value 4397 Hz)
    assert abs(W.f_isco(0.5, 0.5) - 4397.0) < 2.0
    # support: f_low <= f < f_isco, Nyquist and DC excluded
    nz = np.nonzero(h0)[0]
    assert f[nz[0]] >= 30.0 and f[nz[0] - 1] < 30.0
    assert f[nz[-1]] < W.f_isco(15.0, 12.0) <= f[nz[-1] + 1]
    # amplitude f^(-7/6)
    np.testing.assert_allclose(np.abs(h0[nz]), f[nz] ** (-7 / 6), rtol=1e-13)


@pytest.mark.parametrize("order", [2, 3])
def test_phase_gradient_finite_difference(order):
    f = np.linspace(30.0, 200.0, 40)
    mc, eta, tc, phic = 9.0, 0.22, 1.5, 0.3
    d = W.phase_grad_mc_eta(f, mc, eta, order)
    th = np.array([mc, eta, tc, phic])
    for i in range(4):
        e = np.zeros(4)
        e[i] = 1e-6 * max(abs(th[i]), 1.0)
        p = W.phase_mc_eta(f, *(th + e), order)
        m = W.phase_mc_eta(f, *(th - e), order)
        fd = (p - m) / (2 * e[i])
        np.testing.assert_allclose(d[i], fd, rtol=1e-6, atol=1e-6 * np.abs(fd).max())


def test_mc_eta_form_matches_component_form():
    f = np.linspace(30.0, 200.0, 40)
    m1, m2 = 17.0, 6.0
    _, eta, mc = W.mass_params(m1, m2)
    np.testing.assert_allclose(W.phase_mc_eta(f, mc, eta, 0.2, 0.1, 3), W.phase(f, m1, m2, 0, 0, 0.2, 0.1, 3), rtol=1e-12)
    # chirp mass of 1.4 + 1.4 is 1.2188 (textbook)
    assert abs(W.mass_params(1.4, 1.4)[2] - 1.2188) < 1e-4
