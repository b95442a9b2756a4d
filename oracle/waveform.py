"""Closed-form stationary-phase chirp templates, FP64 (test infrastructure only).

The paper generates its bank with IMRPhenomPv2 (Sec. III.B), which is not
available here.  The templates are the closed-form stationary-phase (TaylorF2)
chirp ``h(f) = f^(-7/6) exp(-i Psi(f))`` with the post-Newtonian phase

    Psi(f) = 2 pi f t_c - phi_c - pi/4
             + 3/(128 eta v^5) [1 + (20/9)(743/336 + 11 eta/4) v^2
                                 + (4 beta - 16 pi) v^3]

with ``v = (pi M f)^(1/3)``, ``M`` the total mass in seconds, ``eta`` the
symmetric mass ratio and ``beta`` the aligned-spin spin-orbit coefficient.
Order 0 is the Newtonian phase alone, order 2 keeps the phase through 1PN
(drops the ``v^3`` term), order 3 keeps the 1.5PN tail and spin-orbit term.  The template is supported on
``f_low <= f < f_isco`` with ``f_isco = 1/(6^(3/2) pi M)`` and ``0 < j < n/2``.
The extrinsic form of Eq. (3) holds: ``t_c`` enters as ``exp(-2 pi i f t_c)``.

Pinned by: the stationary-phase relation dPsi/df = 2 pi (t_c - tau(f)) against
the textbook time-to-coalescence series, the Newtonian chirp times printed in
Table I for the case-study sub-bank, exchange symmetry of the spin term, and
finite differences of the phase derivatives (tests/test_oracle_waveform.py).
"""
from __future__ import annotations

import numpy as np

MSUN_S = 4.925491025543576e-06  # G M_sun / c^3 [s]


def mass_params(m1, m2):
    """Total mass [s], symmetric mass ratio, chirp mass [M_sun]."""
    m = m1 + m2
    eta = m1 * m2 / (m * m)
    mc = m * eta ** 0.6
    return m * MSUN_S, eta, mc


def spin_orbit_beta(m1, m2, chi1, chi2):
    """1.5PN aligned-spin spin-orbit coefficient beta = sum_i chi_i [113 (m_i/M)^2 + 75 eta] / 12."""
    m = m1 + m2
    eta = m1 * m2 / (m * m)
    return (chi1 * (113.0 * (m1 / m) ** 2 + 75.0 * eta) + chi2 * (113.0 * (m2 / m) ** 2 + 75.0 * eta)) / 12.0


def f_isco(m1, m2):
    """Innermost-stable-circular-orbit frequency 1/(6^(3/2) pi M) [Hz]."""
    return 1.0 / (6.0 ** 1.5 * np.pi * (m1 + m2) * MSUN_S)


def pn_phase(f, mt_s, eta, beta, pn_order):
    """Intrinsic PN part of Psi (without 2 pi f t_c - phi_c - pi/4)."""
    v = np.cbrt(np.pi * mt_s * f)
    c2 = (20.0 / 9.0) * (743.0 / 336.0 + 11.0 * eta / 4.0) if pn_order >= 2 else 0.0
    c3 = (4.0 * beta - 16.0 * np.pi) if pn_order >= 3 else 0.0
    return 3.0 / (128.0 * eta) * (v ** -5 + c2 * v ** -3 + c3 * v ** -2)


def phase(f, m1, m2, chi1=0.0, chi2=0.0, tc=0.0, phic=0.0, pn_order=2):
    mt, eta, _ = mass_params(m1, m2)
    beta = spin_orbit_beta(m1, m2, chi1, chi2)
    return 2.0 * np.pi * f * tc - phic - np.pi / 4.0 + pn_phase(f, mt, eta, beta, pn_order)


def support(nf, n, df, f_low, fcut):
    """Boolean mask of template support: f_low <= f_j < fcut, 0 < j < n/2."""
    j = np.arange(nf)
    f = j * df
    return (f >= f_low) & (f < fcut) & (j > 0) & (j < n // 2)


def template(params, fs, n, f_low, pn_order, tc=0.0, phic=0.0):
    """h(f_j) for j in [0, n/2], complex128; zero off support."""
    m1, m2, chi1, chi2 = (float(x) for x in params)
    nf = n // 2 + 1
    df = fs / n
    mask = support(nf, n, df, f_low, f_isco(m1, m2))
    f = np.arange(nf) * df
    h = np.zeros(nf, dtype=np.complex128)
    fb = f[mask]
    h[mask] = fb ** (-7.0 / 6.0) * np.exp(-1j * phase(fb, m1, m2, chi1, chi2, tc, phic, pn_order))
    return h


def bank_templates(bank, fs, n, f_low, pn_order):
    """All templates of a bank as a [T, n/2 + 1] complex128 array."""
    return np.stack([template(p, fs, n, f_low, pn_order) for p in bank])


# --- chirp-parameter form used by refinement -------------------------------------------

def phase_mc_eta(f, mc, eta, tc, phic, pn_order):
    """Psi(f) for non-spinning systems parametrised by chirp mass [M_sun] and eta."""
    mt = mc * eta ** -0.6 * MSUN_S
    return 2.0 * np.pi * f * tc - phic - np.pi / 4.0 + pn_phase(f, mt, eta, 0.0, pn_order)


def phase_grad_mc_eta(f, mc, eta, pn_order):
    """Partial derivatives of Psi with respect to (mc, eta, tc, phic), non-spinning.

    With M = mc eta^(-3/5), v = (pi M f)^(1/3) and the PN series
    Psi_PN = 3/(128 eta) [v^-5 + c2 v^-3 + c3 v^-2]:
      dPsi_PN/dM|eta  = 1/(128 eta M) [-5 v^-5 - 3 c2 v^-3 - 2 c3 v^-2]
      dPsi_PN/deta|M  = -Psi_PN/eta + 3/(128 eta) (20/9)(11/4) v^-3
      dM/dmc = M/mc, dM/deta = -(3/5) M/eta.
    Returns four arrays shaped like f.
    """
    mt = mc * eta ** -0.6 * MSUN_S
    v = np.cbrt(np.pi * mt * f)
    c2 = (20.0 / 9.0) * (743.0 / 336.0 + 11.0 * eta / 4.0) if pn_order >= 2 else 0.0
    c3 = -16.0 * np.pi if pn_order >= 3 else 0.0
    psi_pn = 3.0 / (128.0 * eta) * (v ** -5 + c2 * v ** -3 + c3 * v ** -2)
    dpsi_dm = (-5.0 * v ** -5 - 3.0 * c2 * v ** -3 - 2.0 * c3 * v ** -2) / (128.0 * eta * mt)
    dc2 = (20.0 / 9.0) * (11.0 / 4.0) if pn_order >= 2 else 0.0
    dpsi_deta_m = -psi_pn / eta + 3.0 / (128.0 * eta) * dc2 * v ** -3
    d_mc = dpsi_dm * mt / mc
    d_eta = dpsi_deta_m + dpsi_dm * (-0.6 * mt / eta)
    d_tc = 2.0 * np.pi * f
    d_phic = -np.ones_like(f)
    return d_mc, d_eta, d_tc, d_phic

