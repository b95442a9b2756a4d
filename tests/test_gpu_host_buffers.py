"""rb_filter with host buffers (rb_filter_desc.mem, the host/device tagging of the C ABI): strain in host
memory in, triggers in host memory out, in one call whose copies run on the caller's stream. The
result must equal the device-buffer call's, bit for bit."""
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


@pytest.fixture(scope="module")
def case(api):
    k, w = 24, 8
    wl = inputs.tiny(w=w, k=k)
    g = wl.grid
    psd = torch.from_numpy(wl.psd).cuda()
    basis = api.rb_build(api.Bank(wl.bank, g.fs, g.n, g.f_low, 2), psd, k, oversample=64, power_iters=1)
    d = api.make_desc(g.fs, g.n, k, len(wl.bank), w=w, precision="fp16_split_a", rho_i=2.5, rho_ii=4.0,
                      cand_capacity=1 << 16)
    api.rb_pack_coeff(d, basis)
    buf, n = api.rb_filter(d, basis, torch.from_numpy(wl.strain).cuda(), psd, capacity=1 << 16)
    ref = api.triggers_numpy(buf, n)
    assert n > 0
    return wl, psd, basis, d, ref


def test_host_buffers_match_device_call_numpy(api, case):
    """Pageable numpy buffers, called through ctypes with plain host addresses."""
    from paper_2110_13115_gb300 import _native as N

    wl, psd, basis, d, ref = case
    strain = np.ascontiguousarray(wl.strain, dtype=np.float32)
    cap = 1 << 14
    trig = np.zeros(cap, dtype=api.TRIGGER_NP)
    ws = api.workspace(d, host=True)
    dh = N.rb_filter_desc.from_buffer_copy(d)
    dh.mem = N.RB_MEM_HOST_STRAIN | N.RB_MEM_HOST_TRIGGERS
    n = C.c_int64(0)
    b = basis.c_struct()
    for _ in range(2):
        rc = N.load().rb_filter(C.byref(dh), C.byref(b), C.c_void_p(strain.ctypes.data), C.c_void_p(psd.data_ptr()),
                                C.c_void_p(trig.ctypes.data), cap, C.byref(n), C.c_void_p(ws.data_ptr()), ws.numel(),
                                C.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == N.RB_OK, N.load().rb_last_error_detail()
        got = np.sort(trig[: n.value], order=["tmpl", "sample"])
        assert n.value == len(ref)
        assert np.array_equal(got, ref)


def test_host_buffers_pinned_and_one_sided(api, case):
    """Pinned torch host tensors through the binding; each host bit also works alone."""
    from paper_2110_13115_gb300 import _native as N

    wl, psd, basis, d, ref = case
    strain_h = torch.from_numpy(wl.strain).pin_memory()
    cap = 1 << 14
    trig_h = torch.zeros(cap * 24, dtype=torch.uint8).pin_memory()
    n = api.rb_filter_host(d, basis, strain_h, psd, trig_h)
    got = np.sort(trig_h[: n * 24].numpy().view(api.TRIGGER_NP), order=["tmpl", "sample"])
    assert np.array_equal(got, ref)
    ws = api.workspace(d, host=True)
    for mem in (N.RB_MEM_HOST_STRAIN, N.RB_MEM_HOST_TRIGGERS):
        dh = N.rb_filter_desc.from_buffer_copy(d)
        dh.mem = mem
        strain = strain_h if mem == N.RB_MEM_HOST_STRAIN else strain_h.cuda()
        out = trig_h if mem == N.RB_MEM_HOST_TRIGGERS else torch.zeros(cap * 24, dtype=torch.uint8, device="cuda")
        cnt = C.c_int64(0)
        b = basis.c_struct()
        rc = N.load().rb_filter(C.byref(dh), C.byref(b), C.c_void_p(strain.data_ptr()), C.c_void_p(psd.data_ptr()),
                                C.c_void_p(out.data_ptr()), cap, C.byref(cnt), C.c_void_p(ws.data_ptr()), ws.numel(),
                                C.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == N.RB_OK, N.load().rb_last_error_detail()
        got = np.sort(out[: cnt.value * 24].cpu().numpy().view(api.TRIGGER_NP), order=["tmpl", "sample"])
        assert np.array_equal(got, ref), mem


def test_host_trigger_capacity_and_other_calls(api, case):
    from paper_2110_13115_gb300 import _native as N

    wl, psd, basis, d, ref = case
    plan = api.rb_filter_plan(d)
    too_many = plan.host_trig_capacity + 1
    trig = np.zeros(1, dtype=api.TRIGGER_NP)
    with pytest.raises(N.RBError) as e:
        api.rb_filter_host(d, basis, np.ascontiguousarray(wl.strain), psd, trig, capacity=too_many)
    assert e.value.code == N.RB_ERR_BAD_INPUT
    # overflow with host triggers: the count is reported and the first `capacity` records are copied
    small = np.zeros(3, dtype=api.TRIGGER_NP)
    with pytest.raises(N.RBError) as e:
        api.rb_filter_host(d, basis, np.ascontiguousarray(wl.strain), psd, small)
    assert e.value.code == N.RB_ERR_OVERFLOW
    assert all(int(t["tmpl"]) in set(ref["tmpl"].tolist()) for t in small)
    # the stage calls take device pointers only
    dh = N.rb_filter_desc.from_buffer_copy(d)
    dh.mem = N.RB_MEM_HOST_STRAIN
    with pytest.raises(N.RBError) as e:
        api.rb_whiten(dh, torch.from_numpy(wl.strain).cuda(), psd)
    assert e.value.code == N.RB_ERR_BAD_INPUT
