"""Shared helpers of the parity tests (comparison rules only; no filter arithmetic)."""
from __future__ import annotations

import numpy as np

SNR_RTOL = 1e-4  # FP32 SNR parity with the FP64 oracle
BAND = 1e-3  # trigger decisions within this relative distance of a threshold may differ


def rel_close(a, b, rtol):
    return abs(a - b) <= rtol * max(abs(a), abs(b))


def compare_triggers(gpu, ref, w, rho_ii, ref_rho=None, rtol=SNR_RTOL, band=BAND, rho_avg=None, rho_i=None):
    """Compare trigger sets keyed by (template, bin = sample // w).

    gpu: structured array with fields tmpl, sample, snr, phase (block-relative samples).
    ref: oracle structured array with fields template, sample, snr, phase.
    ref_rho[t, m] (optional): oracle full-rate SNR over the valid half (index m - n/2) used to
      accept an arg-max that differs where two samples are within rtol.
    rho_avg[t, i] / rho_i (optional): oracle bin-averaged SNR; a trigger missing on one side is
      accepted when its bin's averaged SNR lies within `band` of rho_i.
    Returns a dict of counts; raises AssertionError with the first offending key.
    """
    g = {(int(r["tmpl"]), int(r["sample"]) // w): r for r in gpu}
    o = {(int(r["template"]), int(r["sample"]) // w): r for r in ref}
    stats = dict(both=0, only_gpu=0, only_ref=0, argmax_tie=0)
    for key in set(g) | set(o):
        if key in g and key in o:
            stats["both"] += 1
            a, b = g[key], o[key]
            assert rel_close(float(a["snr"]), float(b["snr"]), rtol), ("snr", key, a, b)
            if int(a["sample"]) != int(b["sample"]):
                assert ref_rho is not None, ("argmax", key, a, b)
                n_half_off = ref_rho.shape[1]
                r_at = ref_rho[key[0], int(a["sample"]) - n_half_off]
                assert rel_close(r_at, float(b["snr"]), rtol), ("argmax", key, a, b, r_at)
                stats["argmax_tie"] += 1
            else:
                dphi = np.angle(np.exp(1j * (float(a["phase"]) - float(b["phase"]))))
                assert abs(dphi) < 1e-3, ("phase", key, a, b)
        else:
            r = g.get(key) if key in g else o.get(key)
            val = float(r["snr"])
            near_ii = abs(val - rho_ii) <= band * rho_ii
            near_i = False
            if rho_avg is not None and rho_i is not None:
                nb_off = rho_avg.shape[1]
                ra = rho_avg[key[0], key[1] - nb_off]
                near_i = abs(ra - rho_i) <= band * max(rho_i, 1e-30)
            if key in g and ref_rho is not None:
                # the oracle's maximum over this bin must sit at the threshold
                n_half_off = ref_rho.shape[1]
                m0 = key[1] * w - n_half_off
                near_ii = near_ii or abs(ref_rho[key[0], m0:m0 + w].max() - rho_ii) <= band * rho_ii
            assert near_ii or near_i, ("only_" + ("gpu" if key in g else "ref"), key, r)
            stats["only_gpu" if key in g else "only_ref"] += 1
    return stats
