"""Peak |SNR|^2 of a chirp template and its gradient, FP64 (test infrastructure only).

For a candidate theta = (mc, eta, t_c, phi_c) of a non-spinning chirp, the
matched filter of Eq. (1) evaluated at the template's own coalescence time
(Eq. 3-4 with t_0 folded into Psi) is

    Z(theta) = sum_j w_j s_j conj(h_j(theta)),   w_j = 4 df / S_j,
    J(theta) = |Z|^2 / sigma^2,                  sigma^2 = sum_j w_j |h_j|^2,

with h_j = f_j^(-7/6) exp(-i Psi(f_j; theta)) on the support frozen at the
starting point (f_low <= f < f_isco(theta_0)), so sigma does not depend on
theta.  Since dh/dtheta = -i (dPsi/dtheta) h,

    dZ/dtheta = sum_j w_j s_j (i dPsi_j/dtheta) conj(h_j),
    dJ/dtheta = 2 Re(conj(Z) dZ/dtheta) / sigma^2.

The ascent rule (not in the paper; see the design notes) works in scaled
coordinates u = (mc/mc_0, eta, t_c f_ref, phi_c): a step of length alpha along
the normalised gradient is taken only if J increases (then alpha doubles, up
to alpha_max); otherwise alpha halves.  eta is clamped to [eta_min, 0.25].

Pinned by: central finite differences of J, dJ/dphi_c == 0, dJ/dt_c == 0 at
the true t_c of a noiseless self-injection, and J equal to the template
method's |z|^2/sigma^2 at integer samples (tests/test_oracle_refine.py).
"""
from __future__ import annotations

import numpy as np

from . import waveform

F_REF = 100.0
ETA_MIN = 0.05


def setup(s_fd, psd, fs, n, f_low, mc0, eta0):
    """Frequencies, weights w_j s_j and |h_j|^2 weights on the support frozen at (mc0, eta0)."""
    df = fs / n
    mt0 = mc0 * eta0 ** -0.6 * waveform.MSUN_S
    fcut = 1.0 / (6.0 ** 1.5 * np.pi * mt0)
    mask = waveform.support(n // 2 + 1, n, df, f_low, fcut)
    f = np.arange(n // 2 + 1)[mask] * df
    wgt = 4.0 * df / np.asarray(psd, dtype=np.float64)[mask]
    ws = wgt * s_fd[mask]
    amp = f ** (-7.0 / 6.0)
    sig2 = float(np.sum(wgt * amp * amp))
    return f, ws, amp, sig2


def objective(theta, f, ws, amp, sig2, pn_order):
    mc, eta, tc, phic = theta
    psi = waveform.phase_mc_eta(f, mc, eta, tc, phic, pn_order)
    hc = amp * np.exp(1j * psi)  # conj(h)
    z = np.sum(ws * hc)
    return float(np.abs(z) ** 2 / sig2), z


def gradient(theta, f, ws, amp, sig2, pn_order):
    """(J, dJ/dtheta[4]) at theta."""
    mc, eta, tc, phic = theta
    psi = waveform.phase_mc_eta(f, mc, eta, tc, phic, pn_order)
    hc = amp * np.exp(1j * psi)
    z = np.sum(ws * hc)
    dpsi = waveform.phase_grad_mc_eta(f, mc, eta, pn_order)
    g = np.empty(4)
    for i in range(4):
        dz = np.sum(ws * 1j * dpsi[i] * hc)
        g[i] = 2.0 * np.real(np.conj(z) * dz) / sig2
    return float(np.abs(z) ** 2 / sig2), g


def ascend(theta0, s_fd, psd, fs, n, f_low, pn_order, steps=20, alpha0=1e-3, alpha_max=0.05):
    """Gradient ascent of J from theta0; returns (theta, J, history of J)."""
    theta = np.array(theta0, dtype=np.float64)
    mc0 = theta[0]
    f, ws, amp, sig2 = setup(s_fd, psd, fs, n, f_low, theta[0], theta[1])
    scale = np.array([mc0, 1.0, 1.0 / F_REF, 1.0])  # theta = u * scale
    u = theta / scale
    j, g = gradient(theta, f, ws, amp, sig2, pn_order)
    hist = [j]
    alpha = alpha0
    for _ in range(steps):
        gu = g * scale
        norm = np.sqrt(np.sum(gu * gu))
        if not norm > 0.0:
            hist.append(j)
            continue
        u_try = u + alpha * gu / norm
        u_try[1] = min(max(u_try[1], ETA_MIN), 0.25)
        th_try = u_try * scale
        j_try, g_try = gradient(th_try, f, ws, amp, sig2, pn_order)
        if j_try > j:
            u, j, g = u_try, j_try, g_try
            alpha = min(2.0 * alpha, alpha_max)
        else:
            alpha = 0.5 * alpha
        hist.append(j)
    return u * scale, j, np.array(hist)
