"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke run.

This module draws the workload only: bank parameters, coloured Gaussian noise,
injected chirp signals and the analytic noise spectrum.  It holds none of the
matched-filter arithmetic (no whitening, no filtering, no basis, no
thresholds); the CUDA path and the CPU oracle both consume what it returns.

The paper filters PyCBC-generated coloured Gaussian noise against an O2
template bank (Sec. IV, its comparison with the template-by-template matched
filter).  Neither is available here, so the synthetic workloads below stand in
for them:

* noise: stationary Gaussian noise coloured by the analytic one-sided PSD
  ``S(f) = A [(f/40)^-4 + 2 + 2 (f/40)^2]`` with ``A = 1`` (internal units),
  drawn in the frequency domain and band-limited to ``f >= f_low / 2`` so
  that single-precision strain keeps full precision in band;
* signals: closed-form stationary-phase (TaylorF2) chirps,
  ``h(f) = f^(-7/6) exp(-i Psi(f))``, scaled to a stated optimal SNR.

All randomness comes from ``numpy.random.default_rng(seed)`` with the seeds
fixed per workload (bank 0, injections 2, noise ``1000 + 2*segment +
detector``).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

MSUN_S = 4.925491025543576e-06  # G M_sun / c^3 in seconds

SEED_BANK = 0
SEED_INJ = 2


def noise_seed(segment: int = 0, detector: int = 0) -> int:
    return 1000 + 2 * segment + detector


@dataclasses.dataclass(frozen=True)
class Grid:
    """Uniform sampling of one filtering block: ``n`` samples at ``fs`` Hz."""

    fs: float
    n: int
    f_low: float

    @property
    def dt(self) -> float:
        return 1.0 / self.fs

    @property
    def df(self) -> float:
        return self.fs / self.n

    @property
    def nf(self) -> int:
        return self.n // 2 + 1

    @property
    def freqs(self) -> np.ndarray:
        return np.arange(self.nf, dtype=np.float64) * self.df


def analytic_psd(grid: Grid, amplitude: float = 1.0) -> np.ndarray:
    """One-sided PSD on the grid's frequencies; ``inf`` at DC.

    ``S(f) = A [(f/40)^-4 + 2 + 2 (f/40)^2]`` (the analytic spectrum of the
    synthetic workloads).  Returned as float64 of length ``n/2 + 1``.
    """
    f = grid.freqs
    x = np.empty_like(f)
    x[0] = np.inf
    r = f[1:] / 40.0
    x[1:] = amplitude * (r ** -4 + 2.0 + 2.0 * r * r)
    return x


@dataclasses.dataclass(frozen=True)
class BankSpec:
    n_templates: int
    m_min: float
    m_max: float
    chi_max: float = 0.0  # aligned spins uniform in [-chi_max, chi_max]
    pn_order: int = 2  # 2: Newtonian+1PN phase, 3: adds the 1.5PN tail and spin-orbit terms


def draw_bank(spec: BankSpec, seed: int = SEED_BANK) -> np.ndarray:
    """Template parameters ``[T, 4] = (m1, m2, chi1, chi2)``, m1 >= m2, in solar masses.

    Component masses uniform in ``[m_min, m_max]``; aligned spins uniform in
    ``[-chi_max, chi_max]`` (zero when ``chi_max == 0``).
    """
    rng = np.random.default_rng(seed)
    m = rng.uniform(spec.m_min, spec.m_max, size=(spec.n_templates, 2))
    chi = rng.uniform(-spec.chi_max, spec.chi_max, size=(spec.n_templates, 2)) if spec.chi_max > 0 else np.zeros((spec.n_templates, 2))
    swap = m[:, 1] > m[:, 0]
    m[swap] = m[swap][:, ::-1]
    chi[swap] = chi[swap][:, ::-1]
    return np.ascontiguousarray(np.concatenate([m, chi], axis=1))


def white_draws(nf: int, seed: int) -> np.ndarray:
    """Standard-normal complex draws ``x + i y`` for ``nf`` frequency bins."""
    rng = np.random.default_rng(seed)
    xy = rng.standard_normal(size=(2, nf))
    return xy[0] + 1j * xy[1]


def complex_normal(shape, seed: int) -> np.ndarray:
    """Standard complex normal draws (E|x|^2 = 2) of the given shape, complex128."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(size=shape) + 1j * rng.standard_normal(size=shape)


def unit_rows(rows: int, cols: int, seed: int) -> np.ndarray:
    """Rows of complex normal draws scaled to unit Euclidean norm, column 0 zero (DC)."""
    x = complex_normal((rows, cols), seed)
    x[:, 0] = 0.0
    return x / np.linalg.norm(x, axis=1, keepdims=True)


def coloured_noise(grid: Grid, psd: np.ndarray, seed: int, scale: float = 1.0) -> np.ndarray:
    """Gaussian noise with one-sided PSD ``scale * psd`` as a float64 time series.

    Frequency-domain draw ``n(f_j) = sqrt(scale S_j n dt / 4) (x + i y)`` so that
    ``E|n(f)|^2 = scale S T_obs / 2`` with ``n(f) = dt * DFT(n)``; DC, Nyquist and
    everything below ``f_low / 2`` are zero.
    """
    w = white_draws(grid.nf, seed)
    f = grid.freqs
    amp = np.zeros(grid.nf)
    band = (f >= 0.5 * grid.f_low) & (np.arange(grid.nf) < grid.n // 2)
    amp[band] = np.sqrt(scale * psd[band] * grid.n * grid.dt / 4.0)
    nt = np.fft.irfft(amp * w, n=grid.n) / grid.dt
    return nt


# --- source model for injections -------------------------------------------------
# The injected signals use the same closed-form stationary-phase chirp as the
# template bank (the paper injects IMRPhenomPv2 signals through PyCBC, which is
# not available; TaylorF2 stands in for it).


def _source_phase(f, m1, m2, chi1, chi2, tc, phic, pn_order):
    mt = (m1 + m2) * MSUN_S
    eta = m1 * m2 / (m1 + m2) ** 2
    v = np.cbrt(np.pi * mt * f)
    v2 = v * v
    series = 1.0 + (20.0 / 9.0) * (743.0 / 336.0 + 11.0 * eta / 4.0) * v2
    if pn_order >= 3:
        q1, q2 = m1 / (m1 + m2), m2 / (m1 + m2)
        so = (chi1 * (113.0 * q1 * q1 + 75.0 * eta) + chi2 * (113.0 * q2 * q2 + 75.0 * eta)) / 12.0
        series = series - (16.0 * np.pi - 4.0 * so) * v2 * v
    return 2.0 * np.pi * f * tc - phic - np.pi / 4.0 + 3.0 / (128.0 * eta * v2 * v2 * v) * series


def _source_fisco(m1, m2):
    return 1.0 / (6.0 ** 1.5 * np.pi * (m1 + m2) * MSUN_S)


def source_fd(grid: Grid, params, tc: float, phic: float, pn_order: int) -> np.ndarray:
    """Frequency-domain chirp ``f^(-7/6) exp(-i Psi)`` on ``f_low <= f < min(f_isco, fs/2)``."""
    m1, m2, chi1, chi2 = (float(x) for x in params)
    f = grid.freqs
    j = np.arange(grid.nf)
    band = (f >= grid.f_low) & (f < _source_fisco(m1, m2)) & (j < grid.n // 2) & (j > 0)
    h = np.zeros(grid.nf, dtype=np.complex128)
    fb = f[band]
    h[band] = fb ** (-7.0 / 6.0) * np.exp(-1j * _source_phase(fb, m1, m2, chi1, chi2, tc, phic, pn_order))
    return h


def _source_norm(grid: Grid, h: np.ndarray, psd: np.ndarray) -> float:
    band = h != 0
    return math.sqrt(4.0 * grid.df * float(np.sum(np.abs(h[band]) ** 2 / psd[band])))


@dataclasses.dataclass(frozen=True)
class Injection:
    params: tuple  # (m1, m2, chi1, chi2)
    tc: float  # seconds from block start
    phic: float
    snr: float


def draw_injections(spec: BankSpec, grid: Grid, n_inj: int, snr_range, seed: int = SEED_INJ,
                    min_sep: float = 0.0, integer_tc: bool = False) -> list:
    """Injection parameters: masses/spins from the bank's distribution (off the
    bank's own grid), coalescence times uniform over the valid half of the block
    (at least ``min_sep`` s apart), phases uniform, SNRs uniform in ``snr_range``."""
    rng = np.random.default_rng(seed)
    t0 = grid.n // 2 * grid.dt + 0.25
    t1 = grid.n * grid.dt - 0.5
    out, tcs = [], []
    tries = 0
    while len(out) < n_inj:
        tries += 1
        if tries > 100000:
            raise RuntimeError("could not place injections")
        m = np.sort(rng.uniform(spec.m_min, spec.m_max, size=2))[::-1]
        chi = rng.uniform(-spec.chi_max, spec.chi_max, size=2) if spec.chi_max > 0 else np.zeros(2)
        tc = rng.uniform(t0, t1)
        if integer_tc:
            tc = round(tc * grid.fs) / grid.fs
        if any(abs(tc - x) < min_sep for x in tcs):
            continue
        phic = rng.uniform(0.0, 2.0 * np.pi)
        snr = rng.uniform(*snr_range) if np.ndim(snr_range) else float(snr_range)
        tcs.append(tc)
        out.append(Injection((float(m[0]), float(m[1]), float(chi[0]), float(chi[1])), float(tc), float(phic), float(snr)))
    return out


def injection_series(grid: Grid, psd: np.ndarray, inj: Injection, pn_order: int) -> np.ndarray:
    """Time series of one injection scaled to optimal SNR ``inj.snr`` against ``psd``."""
    h = source_fd(grid, inj.params, inj.tc, inj.phic, pn_order)
    h *= inj.snr / _source_norm(grid, h, psd)
    return np.fft.irfft(h, n=grid.n) / grid.dt


@dataclasses.dataclass
class Workload:
    """One block of strain with everything needed to filter it."""

    name: str
    grid: Grid
    bank_spec: BankSpec
    bank: np.ndarray  # [T, 4] float64
    psd: np.ndarray  # [nf] float64 (inf at DC)
    strain: np.ndarray  # [n] float32
    injections: list
    k: int
    w: int
    rho_ii: float


def make_workload(name: str, grid: Grid, bank_spec: BankSpec, k: int, w: int, rho_ii: float,
                  n_inj: int = 0, snr_range=(10.0, 10.0), min_sep: float = 0.0,
                  segment: int = 0, detector: int = 0, psd_scale: float = 1.0,
                  integer_tc: bool = False, noise: bool = True) -> Workload:
    psd = analytic_psd(grid)
    bank = draw_bank(bank_spec)
    x = coloured_noise(grid, psd * psd_scale, noise_seed(segment, detector)) if noise else np.zeros(grid.n)
    injs = draw_injections(bank_spec, grid, n_inj, snr_range, min_sep=min_sep, integer_tc=integer_tc) if n_inj else []
    for inj in injs:
        x = x + injection_series(grid, psd * psd_scale, inj, bank_spec.pn_order)
    return Workload(name, grid, bank_spec, bank, psd * psd_scale, x.astype(np.float32), injs, k, w, rho_ii)


# --- the named workloads ------------------------------------------------------------

def tiny(w: int = 8, k: int = 16, noise: bool = True, n_templates: int = 64) -> Workload:
    """64 templates (masses 10-30, Newtonian+1PN), 16 s at 1024 Hz, one SNR-10 injection."""
    grid = Grid(fs=1024.0, n=16384, f_low=30.0)
    spec = BankSpec(n_templates, 10.0, 30.0, 0.0, 2)
    return make_workload("tiny-64x16s@1024Hz", grid, spec, k=k, w=w, rho_ii=5.0, n_inj=1,
                         snr_range=10.0, noise=noise)


def full(w: int = 8, k: int = 256, n_templates: int = 10000, n_inj: int = 20, segment: int = 0,
         noise: bool = True, n: int = 524288) -> Workload:
    """10,000 templates (masses 3-50, aligned spins, 1.5PN), 256 s at 2048 Hz, 20 injections SNR 5-20."""
    grid = Grid(fs=2048.0, n=n, f_low=30.0)
    spec = BankSpec(n_templates, 3.0, 50.0, 0.5, 3)
    return make_workload(f"full-{n_templates}x{int(n / 2048)}s@2048Hz", grid, spec, k=k, w=w, rho_ii=5.0,
                         n_inj=n_inj, snr_range=(5.0, 20.0), min_sep=4.0, segment=segment, noise=noise)


def precision(k: int = 400, w: int = 8, n_templates: int = 50000, n_inj: int = 3,
              noise: bool = True) -> Workload:
    """50,000 templates (masses 1-50, non-spinning, 1.5PN), 128 s at 4096 Hz with f_low = 40 Hz
    (so the longest template, 43.6 s, fits the 64-s valid half), 3 injections SNR 10-20."""
    grid = Grid(fs=4096.0, n=524288, f_low=40.0)
    spec = BankSpec(n_templates, 1.0, 50.0, 0.0, 3)
    return make_workload(f"precision-{n_templates}x128s@4096Hz", grid, spec, k=k, w=w, rho_ii=5.0,
                         n_inj=n_inj, snr_range=(10.0, 20.0), min_sep=4.0, noise=noise)


def scaled(name: str, fs: float, n: int, n_templates: int, m_range=(3.0, 50.0), chi_max=0.5, pn_order=3,
           f_low=30.0, k=64, w=8, n_inj=2, snr_range=(8.0, 15.0), rho_ii=5.0, min_sep=1.0,
           segment=0, detector=0, psd_scale=1.0, noise=True) -> Workload:
    """A workload with the full-size recipe at a smaller block and bank (parity cases); noise=False
    leaves the injections alone in the block."""
    grid = Grid(fs=fs, n=n, f_low=f_low)
    spec = BankSpec(n_templates, m_range[0], m_range[1], chi_max, pn_order)
    return make_workload(name, grid, spec, k=k, w=w, rho_ii=rho_ii, n_inj=n_inj, snr_range=snr_range,
                         min_sep=min_sep, segment=segment, detector=detector, psd_scale=psd_scale, noise=noise)


# --- batches of uneven segments from two detectors ----------------------------------------

@dataclasses.dataclass
class Segment:
    """One detector's strain over one segment (float32, ``length`` samples from ``start``)."""

    index: int
    detector: int
    start: int  # global sample index of the segment's first sample
    strain: np.ndarray
    psd_scale: float
    injections: list


@dataclasses.dataclass
class BatchBlock:
    """A filtering block of a segment: samples [offset, offset + n) of the segment, keeping
    triggers at block samples >= valid_lo (n/2, or more for a right-aligned tail block)."""

    segment: int  # index into BatchWorkload.segments
    offset: int
    n: int
    valid_lo: int


@dataclasses.dataclass
class BatchWorkload:
    name: str
    fs: float
    f_low: float
    bank_spec: BankSpec  # parameter ranges of every bank (sizes differ)
    banks: list  # [T_b, 4] float64 per bank, concatenated in this order for filtering
    segments: list
    blocks: list
    k: int
    w: int
    rho_ii: float

    @property
    def bank(self) -> np.ndarray:
        return np.concatenate(self.banks, axis=0)

    def block_psd(self, b: BatchBlock) -> np.ndarray:
        seg = self.segments[b.segment]
        return analytic_psd(Grid(self.fs, b.n, self.f_low)) * seg.psd_scale

    def block_strain(self, b: BatchBlock) -> np.ndarray:
        return self.segments[b.segment].strain[b.offset:b.offset + b.n]

    @property
    def sizes(self) -> list:
        return sorted({b.n for b in self.blocks})

    @property
    def valid_seconds(self) -> float:
        return sum(b.n - b.valid_lo for b in self.blocks) / self.fs


def segment_blocks(length: int, max_block: int) -> list:
    """(offset, n, valid_lo) of the blocks of a segment of ``length`` samples: n is the largest
    power of two <= min(length, max_block); blocks overlap by half; a last block is right-aligned
    and keeps only the samples the block before it did not already cover."""
    n = 1 << (min(length, max_block).bit_length() - 1)
    out = []
    off = 0
    while off + n <= length:
        out.append((off, n, n // 2))
        off += n // 2
    last_end = out[-1][0] + n
    if last_end < length:
        tail = length - n
        out.append((tail, n, last_end - tail))
    return out


def batch(n_segments: int = 64, fs: float = 2048.0, f_low: float = 30.0, unit_s: float = 32.0,
          max_units: int = 16, max_block_s: float = 128.0, n_banks: int = 4, bank_sizes=(5000, 20000),
          m_range=(3.0, 50.0), chi_max: float = 0.5, pn_order: int = 3, k: int = 256, w: int = 8,
          rho_ii: float = 5.0, inj_per_segment: int = 1, snr_range=(8.0, 15.0),
          psd_scales=(0.5, 2.0), seed: int = 4) -> BatchWorkload:
    """Segments of uneven length (uniform multiples of ``unit_s`` in [unit_s, max_units unit_s]) seen by
    two detectors with independent noise and per-detector PSD scale factors, cut into blocks of
    min(max_block_s, 2^floor(log2 L)) with half overlap; ``n_banks`` banks of sizes uniform in
    ``bank_sizes`` drawn from the same parameter ranges (one basis serves all of them)."""
    rng = np.random.default_rng(seed)
    scales = rng.uniform(psd_scales[0], psd_scales[1], size=2)
    sizes = rng.integers(bank_sizes[0], bank_sizes[1] + 1, size=n_banks)
    spec = BankSpec(int(sizes.max()), m_range[0], m_range[1], chi_max, pn_order)
    banks = [draw_bank(BankSpec(int(t), m_range[0], m_range[1], chi_max, pn_order), seed=SEED_BANK + 10 * b)
             for b, t in enumerate(sizes)]
    unit = int(round(unit_s * fs))
    max_block = int(round(max_block_s * fs))
    lengths = rng.integers(1, max_units + 1, size=n_segments) * unit
    segments, blocks = [], []
    start = 0
    for s, length in enumerate(lengths):
        for det in range(2):
            grid = Grid(fs, int(length), f_low)
            psd = analytic_psd(grid) * scales[det]
            x = coloured_noise(grid, psd, noise_seed(s, det))
            injs = draw_injections(spec, grid, inj_per_segment, snr_range, seed=SEED_INJ + 100 * s + det) \
                if inj_per_segment else []
            for inj in injs:
                x = x + injection_series(grid, psd, inj, pn_order)
            seg_index = len(segments)
            segments.append(Segment(s, det, start, x.astype(np.float32), float(scales[det]), injs))
            for off, n, lo in segment_blocks(int(length), max_block):
                blocks.append(BatchBlock(seg_index, off, n, lo))
        start += int(length)
    name = f"batch-{n_segments}seg-x2det-{int(sum(sizes))}tmpl"
    return BatchWorkload(name, fs, f_low, spec, banks, segments, blocks, k, w, rho_ii)
