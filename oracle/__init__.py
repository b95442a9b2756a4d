"""CPU FP64 oracle for the hierarchical reduced-basis matched filter.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, links or
executes this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use it.  It shares no code with the CUDA
path; both sides consume the seeded arrays of ``paper_2110_13115_gb300.inputs``.

Modules (each function cites the passage of arXiv:2110.13115 it follows):

* ``waveform`` - the closed-form stationary-phase templates and the analytic
  derivatives of their phase (stand-in for the paper's IMRPhenomPv2 bank).
* ``mf``       - the template method: Eq. (1) matched filter, Eq. (2)/(4) SNR
  time series by inverse FFT, per-window triggers.
* ``rb``       - the reduced basis (Eq. 5b SVD, Eq. 7 reconstruction, Eq. 8
  truncation loss) and the two-stage hierarchy of Sec. III.C, plus the
  folded first stage of Sec. III.D (Eqs. 10-12).
* ``refine``   - |Z|^2/sigma^2 and its gradient with respect to the chirp
  parameters, with a fixed-step-rule gradient ascent.
* ``cost``     - the operation counts of Sec. III.F (Eqs. 13-15) and the
  throughput definition of Sec. IV.B.2.

Parity status per function is stated in each module header; every function
here is pinned by the ``-m "not gpu"`` tests in ``tests/test_oracle_*.py``.
"""
from . import waveform, mf, rb, refine, cost  # noqa: F401
