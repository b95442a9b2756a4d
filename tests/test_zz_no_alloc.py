"""rb_filter_static: the allocation-free variant of rb_filter, for callers that cannot allocate
device memory (hosts that own the whole GPU pool, latency-critical loops, plugins whose host
forbids allocation calls). Its scratch is a 32 MiB static device array inside the library.

Collected last on purpose (file name): if it fails, a run that stops at the first failure has
already run every other test. It must pass alone in a fresh process and after the other tests.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2110_13115_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_13115_gb300 import api as A, _native as N

    N.load()
    return A


def _static_call(api, d, basis, strain, psd, cap, trig=None):
    from paper_2110_13115_gb300 import _native as N

    trig = torch.empty(cap * 24, dtype=torch.uint8, device="cuda") if trig is None else trig
    n = C.c_int64(0)
    b = basis.c_struct()
    rc = N.load().rb_filter_static(C.byref(d), C.byref(b), C.c_void_p(strain.data_ptr()), C.c_void_p(psd.data_ptr()),
                                   C.c_void_p(trig.data_ptr()), cap, C.byref(n),
                                   C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, trig, n.value


@pytest.mark.parametrize("prec", ["fp32", "fp16_split"])
def test_static_scratch_matches_workspace_path(api, prec):
    from paper_2110_13115_gb300 import _native as N

    k, w = 24, 8
    wl = inputs.tiny(w=w, k=k)
    g = wl.grid
    psd = torch.from_numpy(wl.psd).cuda()
    strain = torch.from_numpy(wl.strain).cuda()
    basis = api.rb_build(api.Bank(wl.bank, g.fs, g.n, g.f_low, 2), psd, k, oversample=64, power_iters=1)
    d = api.make_desc(g.fs, g.n, k, len(wl.bank), w=w, precision=prec, rho_i=2.5, rho_ii=4.0,
                      cand_capacity=1 << 16)
    api.rb_pack_coeff(d, basis)
    assert api.rb_filter_plan(d).workspace_bytes <= (32 << 20)
    cap = 1 << 16
    ref_buf, n_ref = api.rb_filter(d, basis, strain, psd, capacity=cap)
    ref = api.triggers_numpy(ref_buf, n_ref)
    assert n_ref > 0
    trig = torch.empty(cap * 24, dtype=torch.uint8, device="cuda")
    for call in range(2):  # two calls in a row: the shared array keeps no state that matters
        torch.cuda.synchronize()
        alloc0, reserved0 = torch.cuda.memory_allocated(), torch.cuda.memory_reserved()
        free0, total = torch.cuda.mem_get_info()
        rc, buf, n = _static_call(api, d, basis, strain, psd, cap, trig=trig)
        torch.cuda.synchronize()
        assert rc == N.RB_OK, N.load().rb_last_error_detail()
        if call == 1:  # the call itself allocates nothing (the first may still grow driver-side pools)
            assert torch.cuda.memory_allocated() == alloc0 and torch.cuda.memory_reserved() == reserved0
            free1, _ = torch.cuda.mem_get_info()
            assert free0 - free1 <= (2 << 20), (free0, free1)
        got = api.triggers_numpy(buf, n)
        assert n == n_ref
        assert np.array_equal(got["tmpl"], ref["tmpl"]) and np.array_equal(got["sample"], ref["sample"])
        np.testing.assert_allclose(got["snr"], ref["snr"], rtol=1e-4)
        np.testing.assert_allclose(got["phase"], ref["phase"], atol=1e-3)


def test_static_scratch_rejects_oversized_problems(api):
    from paper_2110_13115_gb300 import _native as N

    n, k, T = 1 << 19, 256, 100
    d = api.make_desc(2048.0, n, k, T, w=8)
    assert api.rb_filter_plan(d).workspace_bytes > (32 << 20)
    basis = api.Basis(torch.zeros((k, n // 2), dtype=torch.complex64, device="cuda"),
                      torch.zeros((T, k), dtype=torch.complex64, device="cuda"), n)
    strain = torch.zeros(n, dtype=torch.float32, device="cuda")
    psd = torch.ones(n // 2 + 1, dtype=torch.float64, device="cuda")
    rc, _, _ = _static_call(api, d, basis, strain, psd, 16)
    assert rc == N.RB_ERR_UNSUPPORTED
    assert b"static scratch" in N.load().rb_last_error_detail()
