"""The seeded synthetic workloads: identical on every call (parity runs are reproducible), bank draws
inside their stated ranges, and injections at the optimal SNR they state (reading 16), measured
with the oracle's inner product on the strain after its float32 round trip. No GPU."""
import numpy as np

from oracle import mf
from paper_2110_13115_gb300 import inputs


def test_workloads_are_deterministic():
    a, b = inputs.tiny(), inputs.tiny()
    for f in ("bank", "psd", "strain"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f
    assert a.injections == b.injections
    c, d = inputs.full(n_templates=64), inputs.full(n_templates=64)
    assert np.array_equal(c.strain, d.strain) and np.array_equal(c.bank, d.bank)
    e = inputs.full(n_templates=64, segment=1)  # another segment draws other noise
    assert not np.array_equal(c.strain, e.strain)


def test_bank_draws_stay_in_range():
    spec = inputs.BankSpec(2000, 3.0, 50.0, 0.5, 3)
    bank = inputs.draw_bank(spec)
    assert bank.shape == (2000, 4)
    assert np.all(bank[:, 0] >= bank[:, 1])
    assert np.all((bank[:, :2] >= 3.0) & (bank[:, :2] <= 50.0))
    assert np.all(np.abs(bank[:, 2:]) <= 0.5)
    assert np.all(inputs.draw_bank(inputs.BankSpec(100, 10.0, 30.0))[:, 2:] == 0.0)


def test_injections_have_their_stated_optimal_snr():
    for wl in (inputs.tiny(noise=False), inputs.full(n_templates=16, n_inj=5, noise=False)):
        g = wl.grid
        total = mf.sigma2(mf.strain_fd(wl.strain, g.fs), wl.psd, g.n, g.fs)
        if len(wl.injections) == 1:
            assert abs(np.sqrt(total) / wl.injections[0].snr - 1) < 1e-4
        for inj in wl.injections:
            h = inputs.injection_series(g, wl.psd, inj, wl.bank_spec.pn_order)
            rho = np.sqrt(mf.sigma2(mf.strain_fd(h.astype(np.float32), g.fs), wl.psd, g.n, g.fs))
            assert abs(rho / inj.snr - 1) < 1e-4, (inj, rho)
            assert g.n // 2 * g.dt <= inj.tc < g.n * g.dt  # in the valid half
