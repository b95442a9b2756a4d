"""ctypes declarations of the C ABI in include/rbmf.h (argument marshalling only).

The shared library is built in-tree by ``paper_2110_13115_gb300.build`` into
``paper_2110_13115_gb300/_lib/librbmf.so``.  Loading fails loudly when it is
missing: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "librbmf.so")

RB_OK = 0
RB_ERR_BAD_INPUT = -1
RB_ERR_OOM = -2
RB_ERR_OVERFLOW = -3
RB_ERR_TIMEOUT = -4
RB_ERR_CUDA = -5
RB_ERR_UNSUPPORTED = -6

RB_STAGES = 7
RB_FFT_VARIANTS = 8
STAGE_NAMES = ["setup", "whiten", "basis_filter", "pack", "first_stage", "bucket", "second_stage"]

RB_PREC_FP32 = 0
RB_PREC_FP16_SPLIT = 1
RB_PREC_BF16_SPLIT = 2
RB_PREC_FP16 = 3
RB_PREC_BF16 = 4
RB_PREC_FP16_SPLIT_A = 5
RB_MEM_HOST_STRAIN = 1
RB_MEM_HOST_TRIGGERS = 2

PRECISIONS = {"fp32": 0, "fp16_split": 1, "bf16_split": 2, "fp16": 3, "bf16": 4, "fp16_split_a": 5}


class rb_filter_desc(C.Structure):
    _fields_ = [("fs", C.c_double), ("n", C.c_int64), ("k", C.c_int32), ("n_templates", C.c_int32),
                ("w", C.c_int32), ("precision", C.c_int32), ("rho_i", C.c_float), ("rho_ii", C.c_float),
                ("cand_capacity", C.c_int64), ("sample_offset", C.c_int64), ("block_id", C.c_int32),
                ("mem", C.c_int32)]


class rb_basis(C.Structure):
    _fields_ = [("k", C.c_int32), ("n_templates", C.c_int32), ("n", C.c_int64), ("vectors", C.c_void_p),
                ("coeff", C.c_void_p), ("coeff_op", C.c_void_p), ("coeff_op_precision", C.c_int32),
                ("reserved", C.c_int32)]


class rb_trigger(C.Structure):
    _fields_ = [("sample", C.c_int64), ("tmpl", C.c_int32), ("block", C.c_int32), ("snr", C.c_float),
                ("phase", C.c_float)]


class rb_candidate(C.Structure):
    _fields_ = [("tmpl", C.c_int32), ("bin", C.c_int32), ("snr_avg", C.c_float), ("block", C.c_int32)]


class rb_filter_sizes(C.Structure):
    _fields_ = [("workspace_bytes", C.c_size_t), ("n_bins", C.c_int64), ("n1", C.c_int32), ("n2", C.c_int32),
                ("kp", C.c_int32), ("coeff_op_bytes", C.c_size_t), ("host_trig_capacity", C.c_int64)]


class rb_bank_desc(C.Structure):
    _fields_ = [("fs", C.c_double), ("n", C.c_int64), ("f_low", C.c_double), ("n_templates", C.c_int32),
                ("pn_order", C.c_int32), ("params", C.c_void_p)]


class rb_refine_desc(C.Structure):
    _fields_ = [("fs", C.c_double), ("n", C.c_int64), ("f_low", C.c_double), ("pn_order", C.c_int32),
                ("steps", C.c_int32), ("alpha0", C.c_double), ("alpha_max", C.c_double)]


class rb_block(C.Structure):
    _fields_ = [("strain", C.c_void_p), ("psd", C.c_void_p), ("sample_offset", C.c_int64), ("valid_lo", C.c_int64),
                ("basis", C.c_int32), ("block_id", C.c_int32)]


EXTRA_STRUCTS = {"rb_bank_desc": rb_bank_desc, "rb_refine_desc": rb_refine_desc, "rb_block": rb_block}

assert C.sizeof(rb_trigger) == 24 and C.sizeof(rb_candidate) == 16

_P = C.c_void_p
_D = C.POINTER(rb_filter_desc)
_B = C.POINTER(rb_basis)
_I64P = C.POINTER(C.c_int64)

# name -> (restype, argtypes); every symbol the header declares
SIGNATURES = {
    "rb_strerror": (C.c_char_p, [C.c_int]),
    "rb_last_error_detail": (C.c_char_p, []),
    "rb_version": (C.c_int, []),
    "rb_filter_plan": (C.c_int, [_D, C.POINTER(rb_filter_sizes)]),
    "rb_whiten": (C.c_int, [_D, _P, _P, _P, _P, C.c_size_t, _P]),
    "rb_basis_filter": (C.c_int, [_D, _B, _P, _P, _P, _P, C.c_size_t, _P]),
    "rb_pack_coeff": (C.c_int, [_D, _B, _P, _P]),
    "rb_stage1": (C.c_int, [_D, _B, _P, _P, _I64P, _P, C.c_size_t, _P]),
    "rb_stage2": (C.c_int, [_D, _B, _P, _P, C.c_int64, _P, C.c_int64, _I64P, _P, C.c_size_t, _P]),
    "rb_filter": (C.c_int, [_D, _B, _P, _P, _P, C.c_int64, _I64P, _P, C.c_size_t, _P]),
    "rb_filter_plain": (C.c_int, [_D, _P, _P, _P, _P, C.c_int64, _I64P, _P, C.c_size_t, _P]),
    "rb_filter_static": (C.c_int, [_D, _B, _P, _P, _P, C.c_int64, _I64P, _P]),
    "rb_banks_plan": (C.c_int, [_D, C.c_int32, C.POINTER(rb_filter_sizes)]),
    "rb_folded_plan": (C.c_int, [_D, C.POINTER(C.c_size_t)]),
    "rb_stage1_folded": (C.c_int, [_D, _P, _P, _P, _P, _I64P, _P, C.c_size_t, _P]),
    "rb_stage1_lowpass": (C.c_int, [_D, _P, _P, _P, _P, _I64P, _P, C.c_size_t, _P]),
    "rb_filter_banks": (C.c_int, [_D, _B, C.c_int32, _P, _P, _P, C.c_int64, _I64P, _P, C.c_size_t, _P]),
    "rb_basis_max_loss": (C.c_int, [_B, C.POINTER(C.c_double), _P, C.c_size_t, _P]),
    "rb_batch_plan": (C.c_int, [_D, C.c_int32, C.POINTER(C.c_size_t)]),
    "rb_filter_batch": (C.c_int, [_D, _B, C.c_int32, C.POINTER(rb_block), C.c_int64, _P, C.c_int64, _I64P, _P,
                                  C.c_size_t, _P]),
    "rb_batch_create": (C.c_int, [_D, _B, C.c_int32, C.POINTER(rb_block), C.c_int64, _P, C.c_int64, _P, C.c_size_t,
                                  C.POINTER(C.c_void_p)]),
    "rb_batch_run": (C.c_int, [_P, _I64P, _P]),
    "rb_batch_destroy": (C.c_int, [_P]),
    "rb_set_stage1_variant": (C.c_int, [_D, C.c_int32]),
    "rb_set_fft_variant": (C.c_int, [_D, C.c_int32]),
    "rb_tune_fft": (C.c_int, [_D, _B, _P, C.POINTER(C.c_double), C.POINTER(C.c_int32), _P, C.c_size_t, _P]),
    "rb_tune_stage1": (C.c_int, [_D, _B, _P, C.POINTER(C.c_double), C.POINTER(C.c_int32), _P, C.c_size_t, _P]),
    "rb_refine_workspace_bytes": (C.c_size_t, [C.POINTER(rb_refine_desc)]),
    "rb_refine_eval": (C.c_int, [C.POINTER(rb_refine_desc), _P, _P, _P, _P, _P, C.c_int64, _P, C.c_size_t, _P]),
    "rb_refine_adjoint": (C.c_int, [C.POINTER(rb_refine_desc), _P, _P, _P, _P, _P, _P, C.c_int64, _P, C.c_size_t,
                                    _P]),
    "rb_refine": (C.c_int, [C.POINTER(rb_refine_desc), _P, _P, _P, _P, C.c_int64, _P, C.c_size_t, _P]),
    "rb_profile_start": (C.c_int, []),
    "rb_profile_stop": (C.c_int, [C.POINTER(C.c_double), _I64P]),
    "rb_kernel_launches": (C.c_uint64, []),
    "rb_build_plan": (C.c_int, [C.POINTER(rb_bank_desc), C.c_int32, C.c_int32, C.POINTER(C.c_size_t),
                                C.POINTER(C.c_size_t)]),
    "rb_templates": (C.c_int, [C.POINTER(rb_bank_desc), _P, _P, _P, _P, C.c_size_t, _P]),
    "rb_bank_tau0": (C.c_int, [C.POINTER(rb_bank_desc), C.c_double, _P]),
    "rb_bank_split_tau0": (C.c_int, [_P, C.c_int64, C.c_int32, _P, _P]),
    "rb_basis_k_for_loss": (C.c_int, [_P, C.c_int32, C.c_int64, C.c_double, C.POINTER(C.c_int32),
                                      C.POINTER(C.c_double)]),
    "rb_build": (C.c_int, [C.POINTER(rb_bank_desc), _P, C.c_int32, C.c_int32, C.c_int32, C.c_uint64, _P, _P, _P,
                           C.POINTER(C.c_double), _P, C.c_size_t, _P]),
}

# host-only helpers exported for the CPU tests of the FP64 linear algebra (not in the header)
HOST_HOOKS = {
    "rbx_herm_eig": (C.c_int, [C.c_int, _P, _P, _P]),
    "rbx_cholesky": (C.c_int, [C.c_int, _P, _P]),
    "rbx_stage1_withhold_copies": (C.c_int, [C.c_int]),
    "rbx_set_stage2_tc": (C.c_int, [C.c_int]),
    "rbx_stage2_withhold_copies": (C.c_int, [C.c_int]),
    "rbx_set_fft_radix32": (C.c_int, [C.c_int]),
    "rbx_set_stage2_ring": (C.c_int, [C.c_int]),
    "rbx_set_stage2_tc_piece": (C.c_int, [C.c_int]),
    "rbx_set_stage2_tc_windows": (C.c_int, [C.c_int]),
    "rbx_mma_sync_rate": (C.c_int, [C.c_int, C.POINTER(C.c_double)]),
}

_lib = None


class RBError(RuntimeError):
    def __init__(self, name, code, detail):
        super().__init__(f"{name} failed: {code} ({detail})")
        self.code = code


def load(path: str = LIB_PATH):
    """Load the shared library (raises if it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is not built: run `python -m paper_2110_13115_gb300.build`")
    lib = C.CDLL(path)
    for name, (res, args) in list(SIGNATURES.items()) + list(HOST_HOOKS.items()):
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(name: str, rc: int, allow=()):
    if rc == RB_OK or rc in allow:
        return rc
    lib = load()
    raise RBError(name, rc, f"{lib.rb_strerror(rc).decode()}: {lib.rb_last_error_detail().decode()}")
