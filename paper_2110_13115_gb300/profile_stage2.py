"""Timing driver of the second stage on real clustered candidates, for profiling it alone.

``python -m paper_2110_13115_gb300.profile_stage2 [kernel ...]`` takes the full-size block (10,000
templates, 256 s at 2048 Hz, w = 8, 20 injections), the first of its four tau0 sub-banks (2,500
templates) with a GPU basis of at most 320 vectors truncated to the fewest that hold every template's
SNR loss within 1e-3, and its first-stage candidates at rho_I = 4.378 (FP16 split-A); then, for each
second-stage kernel given ("tc": the tcgen05 kernel over bin groups of the automatic width, "tc16"
or "tc32": of 16 or 32 samples; a number: the mma.sync kernel with that coefficient-ring depth, 0
for loads into registers, else 2, 3 or 4 slots; "tc 2" if none), two warm-up rb_stage2 calls and
five timed ones. Prints the candidates and the milliseconds per call (bucketing + reconstruction)
for each, then the GPU's mma.sync m16n8k16 FP16 issue rate (register-only products, the ceiling of
the mma.sync kernel).
"""
from __future__ import annotations

import ctypes
import sys

import numpy as np
import torch

from . import api, inputs, _native


def main(argv):
    lib = _native.load()
    wl = inputs.full(w=8, k=256, n_templates=10000, n=524288, segment=0)
    g = wl.grid
    psd_d = torch.from_numpy(wl.psd).cuda()
    strain_d = torch.from_numpy(wl.strain).cuda()
    pn = wl.bank_spec.pn_order
    order, offs = api.rb_bank_split_tau0(api.rb_bank_tau0(api.Bank(wl.bank, g.fs, g.n, g.f_low, pn), g.f_low), 4)
    idx = order[offs[0]:offs[1]]
    full = api.rb_build(api.Bank(np.ascontiguousarray(wl.bank[idx]), g.fs, g.n, g.f_low, pn), psd_d, 320,
                        oversample=64, power_iters=1)
    loss = api.rb_basis_max_loss(full)
    k = int(np.nonzero(loss <= 1e-3)[0][0]) + 1
    basis = api.truncate(full, k)
    del full
    d = api.make_desc(g.fs, g.n, k, len(idx), w=8, precision="fp16_split_a", rho_i=4.378, rho_ii=wl.rho_ii,
                      cand_capacity=1 << 22)
    api.rb_pack_coeff(d, basis)
    ws = api.workspace(d)
    sh = api.rb_whiten(d, strain_d, psd_d, ws=ws)
    beta, bavg = api.rb_basis_filter(d, basis, sh, ws=ws)
    cand, nc = api.rb_stage1(d, basis, bavg, ws=ws)
    del bavg, sh
    c = api.candidates_numpy(cand, nc)
    print(f"k = {k}, {len(idx)} templates, {nc} candidates in {len(np.unique(c['bin']))} bins", flush=True)
    kernels = argv[1:] or ["tc", "2"]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    try:
        for s in kernels:
            tc = {"tc": 1, "tc16": 16, "tc32": 32}.get(s, 0)
            _native.check("rbx_set_stage2_tc", lib.rbx_set_stage2_tc(tc))
            if not tc:
                _native.check("rbx_set_stage2_ring", lib.rbx_set_stage2_ring(int(s)))
            for _ in range(2):
                api.rb_stage2(d, basis, beta, cand, nc, capacity=1 << 22, ws=ws)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(5):
                _, nt = api.rb_stage2(d, basis, beta, cand, nc, capacity=1 << 22, ws=ws)
            e1.record()
            torch.cuda.synchronize()
            print(f"kernel {s}: {nt} triggers, {e0.elapsed_time(e1) / 5:.4f} ms per rb_stage2", flush=True)
    finally:
        lib.rbx_set_stage2_tc(1)
        lib.rbx_set_stage2_ring(2)
    rate = ctypes.c_double(0.0)
    _native.check("rbx_mma_sync_rate", lib.rbx_mma_sync_rate(4000, ctypes.byref(rate)))
    print(f"mma.sync m16n8k16 FP16: {rate.value / 1e9:.1f} G products/s = {rate.value * 4096 * 2 / 1e12:.0f} TFLOP/s",
          flush=True)


if __name__ == "__main__":
    main(sys.argv)
