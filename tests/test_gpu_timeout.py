"""Failure detection without a GPU fault: every device-side wait of the tensor-core first stage is
bounded (1 s of %globaltimer). A host-only test hook makes the next launch's producer issue no copy,
so the MMA warp waits on a barrier that nothing completes; the wait runs out, the kernel stops every
role, frees its tensor memory and returns, and rb_stage1 reports RB_ERR_TIMEOUT. The context stays
usable: the same call then succeeds and matches a call made before."""
import time

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


def test_bounded_wait_reports_timeout_and_context_survives(api):
    from paper_2110_13115_gb300 import _native as N

    lib = N.load()
    n, k, T, w = 1 << 14, 24, 64, 8
    g = inputs.Grid(fs=1024.0, n=n, f_low=30.0)
    psd = inputs.analytic_psd(g)
    x = inputs.coloured_noise(g, psd, inputs.noise_seed(3, 0)).astype(np.float32)
    P = inputs.unit_rows(k, n // 2, seed=31).astype(np.complex64)
    a = inputs.complex_normal((T, k), 32)
    a = (a / np.linalg.norm(a, axis=1, keepdims=True)).astype(np.complex64)
    d = api.make_desc(g.fs, n, k, T, w=w, precision="fp16_split", rho_i=1.5, cand_capacity=1 << 18)
    basis = api.Basis(torch.from_numpy(P).cuda(), torch.from_numpy(a).cuda(), n)
    api.rb_pack_coeff(d, basis)
    ws = api.workspace(d)
    sh = api.rb_whiten(d, torch.from_numpy(x).cuda(), torch.from_numpy(psd).cuda(), ws=ws)
    _, bavg = api.rb_basis_filter(d, basis, sh, keep_beta=False, ws=ws)
    ref_buf, n_ref = api.rb_stage1(d, basis, bavg, ws=ws)
    ref = api.candidates_numpy(ref_buf, n_ref)
    assert n_ref > 0

    lib.rbx_stage1_withhold_copies(1)
    t0 = time.perf_counter()
    with pytest.raises(N.RBError) as e:
        api.rb_stage1(d, basis, bavg, ws=ws)
    waited = time.perf_counter() - t0
    assert e.value.code == N.RB_ERR_TIMEOUT
    assert b"timed out" in lib.rb_last_error_detail()
    assert 0.5 < waited < 30.0

    # the context is intact: the device still runs work and the same call succeeds again
    torch.cuda.synchronize()
    buf, n2 = api.rb_stage1(d, basis, bavg, ws=ws)
    got = api.candidates_numpy(buf, n2)
    assert n2 == n_ref
    assert np.array_equal(got["tmpl"], ref["tmpl"]) and np.array_equal(got["bin"], ref["bin"])
    np.testing.assert_array_equal(got["snr_avg"], ref["snr_avg"])


def test_stage2_tc_bounded_wait_reports_timeout(api):
    """The same for the tcgen05 second stage: with its coefficient producers withholding every copy the
    MMA thread's first wait runs out, rb_stage2 reports RB_ERR_TIMEOUT, and the next call matches."""
    from paper_2110_13115_gb300 import _native as N

    lib = N.load()
    n, k, T, w = 1 << 14, 24, 500, 8
    half, nb = n // 2, n // (2 * w)
    a = inputs.complex_normal((T, k), 51)
    a = (a / np.linalg.norm(a, axis=1, keepdims=True)).astype(np.complex64)
    beta = torch.from_numpy(inputs.complex_normal((k, half), 52).astype(np.complex64)).cuda()
    rng = np.random.default_rng(53)
    cands = np.zeros(3000, dtype=api.CANDIDATE_NP)
    cands["tmpl"] = rng.integers(0, T, len(cands))
    cands["bin"] = nb + rng.integers(0, nb, len(cands))
    cands = np.unique(cands)
    cd = torch.from_numpy(np.ascontiguousarray(cands).view(np.uint8)).cuda()
    d = api.make_desc(1024.0, n, k, T, w=w, rho_ii=1.5, cand_capacity=1 << 14)
    basis = api.Basis(torch.zeros((k, half), dtype=torch.complex64, device="cuda"), torch.from_numpy(a).cuda(), n)
    api.rb_pack_coeff(d, basis)
    lib.rbx_set_stage2_tc(1)
    try:
        buf, n_ref = api.rb_stage2(d, basis, beta, cd, len(cands), capacity=1 << 14)
        ref = api.triggers_numpy(buf, n_ref)
        assert n_ref > 0
        lib.rbx_stage2_withhold_copies(1)
        t0 = time.perf_counter()
        with pytest.raises(N.RBError) as e:
            api.rb_stage2(d, basis, beta, cd, len(cands), capacity=1 << 14)
        waited = time.perf_counter() - t0
        assert e.value.code == N.RB_ERR_TIMEOUT
        assert b"timed out" in lib.rb_last_error_detail()
        assert 0.5 < waited < 30.0
        torch.cuda.synchronize()
        buf, n2 = api.rb_stage2(d, basis, beta, cd, len(cands), capacity=1 << 14)
        got = api.triggers_numpy(buf, n2)
        assert n2 == n_ref
        for f in ("tmpl", "sample", "snr", "phase"):
            assert np.array_equal(got[f], ref[f]), f
    finally:
        lib.rbx_stage2_withhold_copies(0)
        lib.rbx_set_stage2_tc(1)
