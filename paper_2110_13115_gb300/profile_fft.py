"""Timing driver of the basis filter's four-step passes, for profiling them one at a time.

``python -m paper_2110_13115_gb300.profile_fft [mode]`` filters one n = 2^19 block (w = 8) with 64
unit-norm random basis vectors through rb_basis_filter, two warm-up calls then five timed ones, and
the same vectors as templates through rb_filter_plain; mode 0 selects the radix-16 passes, 1 + v the
radix-32 passes in variant v (bit 0: running-product twiddles, bit 1: pass A's rows staged in shared
memory); "all" runs modes 4, 3, 2, 1 and 0. Prints microseconds per vector for each mode.
"""
from __future__ import annotations

import sys

import numpy as np
import torch

from . import api, inputs, _native


def main(argv):
    lib = _native.load()
    n, k, w = 1 << 19, 64, 8
    g = inputs.Grid(2048.0, n, 30.0)
    psd = inputs.analytic_psd(g)
    x = torch.from_numpy(inputs.coloured_noise(g, psd, 5).astype(np.float32)).cuda()
    psd_d = torch.from_numpy(psd).cuda()
    P = inputs.unit_rows(k, n // 2, seed=3).astype(np.complex64)
    d = api.make_desc(g.fs, n, k, 1, w=w)
    basis = api.Basis(torch.from_numpy(P).cuda(), torch.ones((1, k), dtype=torch.complex64, device="cuda"), n)
    ws = api.workspace(d)
    sh = api.rb_whiten(d, x, psd_d, ws=ws)
    arg = argv[1] if len(argv) > 1 else "all"
    modes = (4, 3, 2, 1, 0) if arg == "all" else (int(arg),)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dp = api.make_desc(g.fs, n, 1, k, w=w, rho_ii=6.0)
    wsp = api.workspace(dp)
    trig = torch.empty((1 << 16) * 24, dtype=torch.uint8, device="cuda")
    try:
        for mode in modes:
            lib.rbx_set_fft_radix32(mode)
            for fn, what in ((lambda: api.rb_basis_filter(d, basis, sh, ws=ws), "basis vector"),
                             (lambda: api.rb_filter_plain(dp, basis.vectors, x, psd_d, capacity=1 << 16, ws=wsp,
                                                          trig=trig), "template")):
                for _ in range(2):
                    fn()
                torch.cuda.synchronize()
                e0.record()
                for _ in range(5):
                    fn()
                e1.record()
                torch.cuda.synchronize()
                print(f"mode {mode}: {e0.elapsed_time(e1) / 5 / k * 1e3:.2f} us per {what}", flush=True)
    finally:
        lib.rbx_set_fft_radix32(4)


if __name__ == "__main__":
    main(sys.argv)
