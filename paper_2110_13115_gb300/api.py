"""Python binding of the C ABI: same names, torch tensors for device memory and streams.

Every function only marshals arguments (device pointers, sizes, the current CUDA
stream) and calls the shared library; all arithmetic runs in the sm_103a kernels.
"""
from __future__ import annotations

import ctypes as C
import dataclasses

import numpy as np
import torch

from . import _native as N

TRIGGER_NP = np.dtype([("sample", np.int64), ("tmpl", np.int32), ("block", np.int32), ("snr", np.float32),
                       ("phase", np.float32)])
CANDIDATE_NP = np.dtype([("tmpl", np.int32), ("bin", np.int32), ("snr_avg", np.float32), ("block", np.int32)])


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _lib():
    return N.load()


def make_desc(fs, n, k, n_templates, w=8, precision="fp32", rho_i=0.0, rho_ii=5.0, cand_capacity=1 << 20,
              sample_offset=0, block_id=0, mem=0) -> N.rb_filter_desc:
    prec = N.PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    return N.rb_filter_desc(float(fs), int(n), int(k), int(n_templates), int(w), prec, float(rho_i), float(rho_ii),
                            int(cand_capacity), int(sample_offset), int(block_id), int(mem))


def rb_filter_plan(desc) -> N.rb_filter_sizes:
    out = N.rb_filter_sizes()
    N.check("rb_filter_plan", _lib().rb_filter_plan(C.byref(desc), C.byref(out)))
    return out


def _with_host_mem(desc):
    d = N.rb_filter_desc.from_buffer_copy(desc)
    d.mem = N.RB_MEM_HOST_STRAIN | N.RB_MEM_HOST_TRIGGERS
    return d


def workspace(desc, device="cuda", host=False) -> torch.Tensor:
    """Workspace for desc; host=True sizes it for calls with host buffers (desc.mem set), which also
    serves the device-buffer calls."""
    d = _with_host_mem(desc) if host else desc
    return torch.empty(rb_filter_plan(d).workspace_bytes, dtype=torch.uint8, device=device)


@dataclasses.dataclass
class Basis:
    """Device arrays of a reduced basis (see rb_basis in include/rbmf.h)."""

    vectors: torch.Tensor  # complex64 [k][n/2]
    coeff: torch.Tensor  # complex64 [T][k]
    n: int
    coeff_op: torch.Tensor | None = None
    coeff_op_precision: int = 0
    sigma2: torch.Tensor | None = None  # float64 [T]
    singular_values: np.ndarray | None = None

    @property
    def k(self):
        return self.vectors.shape[0]

    @property
    def n_templates(self):
        return self.coeff.shape[0]

    def c_struct(self) -> N.rb_basis:
        assert self.vectors.is_contiguous() and self.coeff.is_contiguous()
        assert self.vectors.dtype == torch.complex64 and self.coeff.dtype == torch.complex64
        return N.rb_basis(self.k, self.n_templates, int(self.n), self.vectors.data_ptr(), self.coeff.data_ptr(),
                          self.coeff_op.data_ptr() if self.coeff_op is not None else None,
                          int(self.coeff_op_precision), 0)


def rb_whiten(desc, strain: torch.Tensor, psd: torch.Tensor, ws: torch.Tensor | None = None) -> torch.Tensor:
    ws = workspace(desc) if ws is None else ws
    out = torch.empty(desc.n // 2, dtype=torch.complex64, device=strain.device)
    rc = _lib().rb_whiten(C.byref(desc), _p(strain), _p(psd), _p(out), _p(ws), ws.numel(), _stream())
    N.check("rb_whiten", rc)
    return out


def rb_basis_filter(desc, basis: Basis, s_hat: torch.Tensor, keep_beta=True, ws=None):
    ws = workspace(desc) if ws is None else ws
    dev = s_hat.device
    half = desc.n // 2
    nb = rb_filter_plan(desc).n_bins
    beta = torch.empty((desc.k, half), dtype=torch.complex64, device=dev) if keep_beta else None
    bavg = torch.empty((desc.k, nb), dtype=torch.complex64, device=dev)
    b = basis.c_struct()
    rc = _lib().rb_basis_filter(C.byref(desc), C.byref(b), _p(s_hat), _p(beta), _p(bavg), _p(ws), ws.numel(),
                                _stream())
    N.check("rb_basis_filter", rc)
    return beta, bavg


def rb_pack_coeff(desc, basis: Basis) -> Basis:
    """Pack the coefficient operands of both stages for desc.precision into basis.coeff_op
    (in place); rb_filter and rb_stage2 need it for every precision."""
    sizes = rb_filter_plan(desc)
    op = torch.empty(sizes.coeff_op_bytes, dtype=torch.uint8, device=basis.coeff.device)
    b = basis.c_struct()
    N.check("rb_pack_coeff", _lib().rb_pack_coeff(C.byref(desc), C.byref(b), _p(op), _stream()))
    basis.coeff_op = op
    basis.coeff_op_precision = desc.precision
    return basis


def _as_np(buf: torch.Tensor, n: int, dt) -> np.ndarray:
    raw = buf[: n * dt.itemsize].cpu().numpy()
    return raw.view(dt).copy()


def rb_stage1(desc, basis: Basis, beta_avg: torch.Tensor, ws=None):
    """Returns (candidates device buffer, count)."""
    ws = workspace(desc) if ws is None else ws
    cand = torch.empty(max(desc.cand_capacity, 1) * 16, dtype=torch.uint8, device=beta_avg.device)
    n = C.c_int64(0)
    b = basis.c_struct()
    rc = _lib().rb_stage1(C.byref(desc), C.byref(b), _p(beta_avg), _p(cand), C.byref(n), _p(ws), ws.numel(),
                          _stream())
    N.check("rb_stage1", rc)
    return cand, n.value


def rb_stage2(desc, basis: Basis, beta: torch.Tensor, cand: torch.Tensor, n_cand: int, capacity=1 << 20, ws=None):
    ws = workspace(desc) if ws is None else ws
    trig = torch.empty(max(capacity, 1) * 24, dtype=torch.uint8, device=beta.device)
    n = C.c_int64(0)
    b = basis.c_struct()
    rc = _lib().rb_stage2(C.byref(desc), C.byref(b), _p(beta), _p(cand), int(n_cand), _p(trig), int(capacity),
                          C.byref(n), _p(ws), ws.numel(), _stream())
    N.check("rb_stage2", rc)
    return trig, n.value


def rb_filter(desc, basis: Basis, strain: torch.Tensor, psd: torch.Tensor, capacity=1 << 20, ws=None, trig=None):
    """Whole hierarchical filter of one block; returns (trigger buffer, count)."""
    ws = workspace(desc) if ws is None else ws
    trig = torch.empty(max(capacity, 1) * 24, dtype=torch.uint8, device=strain.device) if trig is None else trig
    n = C.c_int64(0)
    b = basis.c_struct()
    rc = _lib().rb_filter(C.byref(desc), C.byref(b), _p(strain), _p(psd), _p(trig), int(capacity), C.byref(n),
                          _p(ws), ws.numel(), _stream())
    N.check("rb_filter", rc)
    return trig, n.value


def _host_ptr(x):
    """Address of a host buffer: a C-contiguous numpy array or a contiguous CPU torch tensor."""
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return C.c_void_p(x.ctypes.data)
    assert x.device.type == "cpu" and x.is_contiguous()
    return C.c_void_p(x.data_ptr())


def rb_filter_host(desc, basis: Basis, strain, psd: torch.Tensor, trig, capacity=None, ws=None) -> int:
    """rb_filter with the strain and the triggers in host memory (desc.mem gets both RB_MEM_* bits):
    the library copies the strain in and the triggers out on the current stream inside the one call.
    strain: float32 [n] host buffer; trig: host buffer of `capacity` records (TRIGGER_NP numpy array
    or a uint8 CPU tensor of capacity * 24 bytes). Returns the trigger count."""
    ws = workspace(desc, host=True) if ws is None else ws
    if capacity is None:
        capacity = len(trig) if isinstance(trig, np.ndarray) and trig.dtype == TRIGGER_NP else trig.numel() // 24
    d = _with_host_mem(desc)
    n = C.c_int64(0)
    b = basis.c_struct()
    rc = _lib().rb_filter(C.byref(d), C.byref(b), _host_ptr(strain), _p(psd), _host_ptr(trig), int(capacity),
                          C.byref(n), _p(ws), ws.numel(), _stream())
    N.check("rb_filter", rc)
    return n.value


# --- sub-banks --------------------------------------------------------------------------------

def rb_banks_plan(descs) -> N.rb_filter_sizes:
    d = (N.rb_filter_desc * len(descs))(*descs)
    out = N.rb_filter_sizes()
    N.check("rb_banks_plan", _lib().rb_banks_plan(d, len(descs), C.byref(out)))
    return out


def banks_workspace(descs, device="cuda", host=False) -> torch.Tensor:
    """Workspace for rb_filter_banks; host=True sizes it for host buffers (it serves both kinds)."""
    ds = [_with_host_mem(d) for d in descs] if host else descs
    return torch.empty(rb_banks_plan(ds).workspace_bytes, dtype=torch.uint8, device=device)


def rb_filter_banks(descs, bases, strain, psd: torch.Tensor, capacity=1 << 22, ws=None, trig=None, host=False):
    """One block through every sub-bank (whitened once); returns (trigger buffer, count). Template rows
    of the triggers index the concatenation of the sub-banks. With host=True, `strain` and `trig` are
    host buffers (numpy or CPU tensors) and the library copies them on the current stream."""
    ws = banks_workspace(descs, host=host) if ws is None else ws
    descs = [N.rb_filter_desc.from_buffer_copy(d) for d in descs]
    for d in descs:
        d.mem = (N.RB_MEM_HOST_STRAIN | N.RB_MEM_HOST_TRIGGERS) if host else 0
    if trig is None:
        trig = (np.zeros(capacity, dtype=TRIGGER_NP) if host else
                torch.empty(max(capacity, 1) * 24, dtype=torch.uint8, device=ws.device))
    d, b = _pairs(descs, bases)
    n = C.c_int64(0)
    sp = _host_ptr(strain) if host else _p(strain)
    tp = _host_ptr(trig) if host else _p(trig)
    rc = _lib().rb_filter_banks(d, b, len(descs), sp, _p(psd), tp, int(capacity), C.byref(n), _p(ws), ws.numel(),
                                _stream())
    N.check("rb_filter_banks", rc)
    return trig, n.value


def rb_basis_max_loss(basis: Basis) -> np.ndarray:
    """Worst single-template truncation loss for every basis size 1..k (float64 [k], host)."""
    ws = torch.empty(max(8 * basis.k, 256), dtype=torch.uint8, device=basis.coeff.device)
    out = np.zeros(basis.k, dtype=np.float64)
    b = basis.c_struct()
    N.check("rb_basis_max_loss", _lib().rb_basis_max_loss(C.byref(b), out.ctypes.data_as(C.POINTER(C.c_double)),
                                                          _p(ws), ws.numel(), _stream()))
    return out


def truncate(basis: Basis, k: int) -> Basis:
    """The first k vectors of a basis (vectors are ordered by singular value) and their coefficients."""
    sv = None if basis.singular_values is None else basis.singular_values[:k]
    return Basis(basis.vectors[:k].contiguous(), basis.coeff[:, :k].contiguous(), basis.n, sigma2=basis.sigma2,
                 singular_values=sv)


def rb_folded_plan(desc) -> int:
    """Workspace bytes of rb_stage1_folded / rb_stage1_lowpass."""
    nbytes = C.c_size_t(0)
    N.check("rb_folded_plan", _lib().rb_folded_plan(C.byref(desc), C.byref(nbytes)))
    return nbytes.value


def rb_stage1_lowpass(desc, templates: torch.Tensor, strain: torch.Tensor, psd: torch.Tensor, ws=None, cand=None):
    """The low-pass and decimation first stage (the paper's comparison); as rb_stage1_folded."""
    return rb_stage1_folded(desc, templates, strain, psd, ws=ws, cand=cand, _entry="rb_stage1_lowpass")


def rb_stage1_folded(desc, templates: torch.Tensor, strain: torch.Tensor, psd: torch.Tensor, ws=None, cand=None,
                     _entry="rb_stage1_folded"):
    """First stage by the template method (folded spectrum, length n/w inverse transforms); returns
    (candidate device buffer, count). templates: complex64 [T][n/2] whitened unit-norm rows."""
    if ws is None:
        ws = torch.empty(rb_folded_plan(desc), dtype=torch.uint8, device=strain.device)
    cand = torch.empty(max(desc.cand_capacity, 1) * 16, dtype=torch.uint8, device=strain.device) if cand is None else cand
    n = C.c_int64(0)
    rc = getattr(_lib(), _entry)(C.byref(desc), _p(templates), _p(strain), _p(psd), _p(cand), C.byref(n), _p(ws),
                                 ws.numel(), _stream())
    N.check(_entry, rc)
    return cand, n.value


def rb_filter_plain(desc, templates: torch.Tensor, strain: torch.Tensor, psd: torch.Tensor, capacity=1 << 20,
                    ws=None, trig=None):
    """Template-method comparator; templates complex64 [T][n/2] unit-norm whitened."""
    ws = workspace(desc) if ws is None else ws
    trig = torch.empty(max(capacity, 1) * 24, dtype=torch.uint8, device=strain.device) if trig is None else trig
    n = C.c_int64(0)
    rc = _lib().rb_filter_plain(C.byref(desc), _p(templates), _p(strain), _p(psd), _p(trig), int(capacity),
                                C.byref(n), _p(ws), ws.numel(), _stream())
    N.check("rb_filter_plain", rc)
    return trig, n.value


# --- batching -------------------------------------------------------------------------------

@dataclasses.dataclass
class Block:
    """One filtering block of a batch (see rb_block): device strain [n] float32 and PSD [n/2+1]
    float64, the index of its (desc, basis) pair, its global sample offset, the first block
    sample whose triggers are kept, and the id copied into its triggers."""

    strain: torch.Tensor
    psd: torch.Tensor
    basis: int
    sample_offset: int = 0
    valid_lo: int | None = None  # default n/2
    block_id: int = 0


def _blocks(descs, blocks):
    arr = (N.rb_block * max(len(blocks), 1))()
    for i, b in enumerate(blocks):
        if b.valid_lo is not None:
            lo = int(b.valid_lo)
        else:  # n/2 of the block's desc; an out-of-range index is left for the library to reject
            lo = descs[b.basis].n // 2 if 0 <= b.basis < len(descs) else 0
        arr[i] = N.rb_block(b.strain.data_ptr(), b.psd.data_ptr(), int(b.sample_offset), lo, int(b.basis),
                            int(b.block_id))
    return arr


def _pairs(descs, bases):
    assert len(descs) == len(bases) and len(descs) > 0
    d = (N.rb_filter_desc * len(descs))(*descs)
    b = (N.rb_basis * len(bases))(*[x.c_struct() for x in bases])
    return d, b


def rb_batch_plan(descs) -> int:
    d = (N.rb_filter_desc * len(descs))(*descs)
    out = C.c_size_t(0)
    N.check("rb_batch_plan", _lib().rb_batch_plan(d, len(descs), C.byref(out)))
    return out.value


def batch_workspace(descs, device="cuda") -> torch.Tensor:
    return torch.empty(rb_batch_plan(descs), dtype=torch.uint8, device=device)


def rb_filter_batch(descs, bases, blocks, capacity=1 << 22, ws=None, trig=None):
    """Every block through the hierarchical filter in one call; returns (trigger buffer, count)."""
    ws = batch_workspace(descs) if ws is None else ws
    trig = torch.empty(max(capacity, 1) * 24, dtype=torch.uint8, device=ws.device) if trig is None else trig
    d, b = _pairs(descs, bases)
    arr = _blocks(descs, blocks)
    n = C.c_int64(0)
    rc = _lib().rb_filter_batch(d, b, len(descs), arr, len(blocks), _p(trig), int(capacity), C.byref(n), _p(ws),
                                ws.numel(), _stream())
    N.check("rb_filter_batch", rc)
    return trig, n.value


class Batch:
    """A batch recorded as one CUDA graph (rb_batch_create); run() replays it with one graph
    launch. Holds references to every device buffer the graph uses."""

    def __init__(self, descs, bases, blocks, capacity=1 << 22, ws=None, trig=None):
        self.ws = batch_workspace(descs) if ws is None else ws
        self.trig = torch.empty(max(capacity, 1) * 24, dtype=torch.uint8, device=self.ws.device) if trig is None else trig
        self.capacity = int(capacity)
        self._keep = (list(descs), list(bases), list(blocks))
        d, b = _pairs(descs, bases)
        arr = _blocks(descs, blocks)
        h = C.c_void_p()
        rc = _lib().rb_batch_create(d, b, len(descs), arr, len(blocks), _p(self.trig), self.capacity, _p(self.ws),
                                    self.ws.numel(), C.byref(h))
        N.check("rb_batch_create", rc)
        self._h = h

    def run(self):
        """Replays the graph on the current stream; returns (trigger buffer, count)."""
        n = C.c_int64(0)
        N.check("rb_batch_run", _lib().rb_batch_run(self._h, C.byref(n), _stream()))
        return self.trig, n.value

    def close(self):
        if getattr(self, "_h", None):
            N.check("rb_batch_destroy", _lib().rb_batch_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def triggers_numpy(buf: torch.Tensor, n: int) -> np.ndarray:
    """Device trigger buffer -> numpy structured array sorted by (tmpl, sample)."""
    a = _as_np(buf, n, TRIGGER_NP)
    return np.sort(a, order=["tmpl", "sample"])


def candidates_numpy(buf: torch.Tensor, n: int) -> np.ndarray:
    a = _as_np(buf, n, CANDIDATE_NP)
    return np.sort(a, order=["tmpl", "bin"])


# --- bank and basis construction ----------------------------------------------------------

class Bank:
    """Host-side bank description (parameters stay on the host, as the C ABI states)."""

    def __init__(self, params: np.ndarray, fs: float, n: int, f_low: float, pn_order: int):
        self.params = np.ascontiguousarray(params, dtype=np.float64)
        assert self.params.ndim == 2 and self.params.shape[1] == 4
        self.fs, self.n, self.f_low, self.pn_order = float(fs), int(n), float(f_low), int(pn_order)

    def c_struct(self) -> N.rb_bank_desc:
        return N.rb_bank_desc(self.fs, self.n, self.f_low, self.params.shape[0], self.pn_order,
                              self.params.ctypes.data)


def rb_build_plan(bank: Bank, k: int, oversample: int = 64):
    t = C.c_size_t(0)
    b = C.c_size_t(0)
    bd = bank.c_struct()
    N.check("rb_build_plan", _lib().rb_build_plan(C.byref(bd), int(k), int(oversample), C.byref(t), C.byref(b)))
    return t.value, b.value


def rb_bank_tau0(bank: Bank, f0: float) -> np.ndarray:
    """Newtonian chirp time of every template from f0 to coalescence [s] (host)."""
    out = np.empty(bank.params.shape[0], dtype=np.float64)
    bd = bank.c_struct()
    N.check("rb_bank_tau0", _lib().rb_bank_tau0(C.byref(bd), float(f0), out.ctypes.data))
    return out


def rb_bank_split_tau0(tau0: np.ndarray, parts: int):
    """Templates in ascending tau0 order cut into `parts` equal-count sub-banks: (order, offsets);
    sub-bank p is order[offsets[p]:offsets[p + 1]] (host)."""
    tau0 = np.ascontiguousarray(tau0, dtype=np.float64)
    order = np.empty(len(tau0), dtype=np.int64)
    offsets = np.empty(int(parts) + 1, dtype=np.int64)
    N.check("rb_bank_split_tau0", _lib().rb_bank_split_tau0(tau0.ctypes.data, len(tau0), int(parts),
                                                            order.ctypes.data, offsets.ctypes.data))
    return order, offsets


def rb_basis_k_for_loss(sv: np.ndarray, n_templates: int, tol: float):
    """Fewest basis vectors whose Eq. 8 loss is <= tol, from rb_build's singular values: (k, loss).
    Raises RBError(RB_ERR_UNSUPPORTED) when all of sv do not reach tol."""
    sv = np.ascontiguousarray(sv, dtype=np.float64)
    k, loss = C.c_int32(0), C.c_double(0.0)
    N.check("rb_basis_k_for_loss", _lib().rb_basis_k_for_loss(sv.ctypes.data, len(sv), int(n_templates), float(tol),
                                                              C.byref(k), C.byref(loss)))
    return k.value, loss.value


def rb_templates(bank: Bank, psd: torch.Tensor):
    """Whitened unit-norm templates [T][n/2] complex64 and sigma^2 [T] float64 (device)."""
    tb, _ = rb_build_plan(bank, 1, 0)
    ws = torch.empty(tb, dtype=torch.uint8, device=psd.device)
    T = bank.params.shape[0]
    out = torch.empty((T, bank.n // 2), dtype=torch.complex64, device=psd.device)
    s2 = torch.empty(T, dtype=torch.float64, device=psd.device)
    bd = bank.c_struct()
    N.check("rb_templates", _lib().rb_templates(C.byref(bd), _p(psd), _p(out), _p(s2), _p(ws), ws.numel(), _stream()))
    return out, s2


def rb_build(bank: Bank, psd: torch.Tensor, k: int, oversample: int = 64, power_iters: int = 1, seed: int = 12345):
    """Reduced basis of the bank (step a0); returns a Basis with sigma2 and singular values."""
    _, bb = rb_build_plan(bank, k, oversample)
    ws = torch.empty(bb, dtype=torch.uint8, device=psd.device)
    T = bank.params.shape[0]
    vec = torch.empty((k, bank.n // 2), dtype=torch.complex64, device=psd.device)
    coeff = torch.empty((T, k), dtype=torch.complex64, device=psd.device)
    s2 = torch.empty(T, dtype=torch.float64, device=psd.device)
    sv = (C.c_double * k)()
    bd = bank.c_struct()
    rc = _lib().rb_build(C.byref(bd), _p(psd), int(k), int(oversample), int(power_iters), C.c_uint64(seed), _p(vec),
                         _p(coeff), _p(s2), sv, _p(ws), ws.numel(), _stream())
    N.check("rb_build", rc)
    del ws
    return Basis(vec, coeff, bank.n, sigma2=s2, singular_values=np.array(sv[:]))


# --- measurement support -------------------------------------------------------------------

def rb_profile_start():
    N.check("rb_profile_start", _lib().rb_profile_start())


def rb_profile_stop():
    """Mean milliseconds per rb_filter stage since rb_profile_start, and the call count."""
    ms = (C.c_double * N.RB_STAGES)()
    calls = C.c_int64(0)
    N.check("rb_profile_stop", _lib().rb_profile_stop(ms, C.byref(calls)))
    return dict(zip(N.STAGE_NAMES, ms[:])), calls.value


def rb_kernel_launches() -> int:
    return int(_lib().rb_kernel_launches())


# --- candidate refinement (step a8) --------------------------------------------------------

def make_refine_desc(fs, n, f_low, pn_order=2, steps=20, alpha0=1e-3, alpha_max=0.05) -> N.rb_refine_desc:
    return N.rb_refine_desc(float(fs), int(n), float(f_low), int(pn_order), int(steps), float(alpha0),
                            float(alpha_max))


def _refine_ws(desc, device):
    return torch.empty(int(_lib().rb_refine_workspace_bytes(C.byref(desc))), dtype=torch.uint8, device=device)


def rb_refine_eval(desc, s_hat: torch.Tensor, psd: torch.Tensor, theta: torch.Tensor):
    """J [n] and Z [n] complex128 at theta [n, 4] float64 (device)."""
    theta = theta.contiguous()
    n = theta.shape[0]
    J = torch.empty(n, dtype=torch.float64, device=theta.device)
    Z = torch.empty(n, dtype=torch.complex128, device=theta.device)
    ws = _refine_ws(desc, theta.device)
    rc = _lib().rb_refine_eval(C.byref(desc), _p(s_hat), _p(psd), _p(theta), _p(J), _p(Z), n, _p(ws), ws.numel(),
                               _stream())
    N.check("rb_refine_eval", rc)
    return J, Z


def rb_refine_adjoint(desc, s_hat, psd, theta, Z, dJ):
    theta = theta.contiguous()
    n = theta.shape[0]
    dtheta = torch.empty((n, 4), dtype=torch.float64, device=theta.device)
    ws = _refine_ws(desc, theta.device)
    rc = _lib().rb_refine_adjoint(C.byref(desc), _p(s_hat), _p(psd), _p(theta), _p(Z.contiguous()),
                                  _p(dJ.contiguous()), _p(dtheta), n, _p(ws), ws.numel(), _stream())
    N.check("rb_refine_adjoint", rc)
    return dtheta


def rb_refine(desc, s_hat: torch.Tensor, psd: torch.Tensor, theta: torch.Tensor):
    """desc.steps of gradient ascent; returns (refined theta [n, 4], J [n]) (device, new tensors)."""
    th = theta.detach().clone().contiguous()
    n = th.shape[0]
    J = torch.empty(n, dtype=torch.float64, device=th.device)
    ws = _refine_ws(desc, th.device)
    rc = _lib().rb_refine(C.byref(desc), _p(s_hat), _p(psd), _p(th), _p(J), n, _p(ws), ws.numel(), _stream())
    N.check("rb_refine", rc)
    return th, J


class PeakSNR2(torch.autograd.Function):
    """J(theta) = |Z|^2 / sigma^2 per candidate; backward runs the adjoint kernel (templates recomputed)."""

    @staticmethod
    def forward(ctx, theta, s_hat, psd, desc):
        J, Z = rb_refine_eval(desc, s_hat, psd, theta.detach())
        ctx.save_for_backward(theta.detach(), Z)
        ctx.s_hat, ctx.psd, ctx.desc = s_hat, psd, desc
        return J

    @staticmethod
    def backward(ctx, gJ):
        theta, Z = ctx.saved_tensors
        dtheta = rb_refine_adjoint(ctx.desc, ctx.s_hat, ctx.psd, theta, Z, gJ.to(torch.float64))
        return dtheta, None, None, None


def peak_snr2(theta, s_hat, psd, desc):
    return PeakSNR2.apply(theta, s_hat, psd, desc)


def rb_tune_stage1(desc, basis: Basis, beta_avg: torch.Tensor, ws=None):
    """Time the first-stage tile variants on these operands; returns (chosen variant, times in ms)."""
    ws = workspace(desc) if ws is None else ws
    times = (C.c_double * 2)()
    chosen = C.c_int32(0)
    b = basis.c_struct()
    rc = _lib().rb_tune_stage1(C.byref(desc), C.byref(b), _p(beta_avg), times, C.byref(chosen), _p(ws), ws.numel(),
                               _stream())
    N.check("rb_tune_stage1", rc)
    return chosen.value, list(times)


def rb_tune_fft(desc, basis: Basis, s_hat: torch.Tensor, ws=None):
    """Times every FFT schedule variant of the basis filter; returns (chosen, ms per variant)."""
    ws = workspace(desc) if ws is None else ws
    times = (C.c_double * N.RB_FFT_VARIANTS)()
    chosen = C.c_int32(-1)
    b = basis.c_struct()
    rc = _lib().rb_tune_fft(C.byref(desc), C.byref(b), _p(s_hat), times, C.byref(chosen), _p(ws), ws.numel(),
                            _stream())
    N.check("rb_tune_fft", rc)
    return chosen.value, list(times)


def rb_set_fft_variant(desc, variant: int):
    N.check("rb_set_fft_variant", _lib().rb_set_fft_variant(C.byref(desc), int(variant)))


def rb_set_stage1_variant(desc, variant: int):
    N.check("rb_set_stage1_variant", _lib().rb_set_stage1_variant(C.byref(desc), int(variant)))
