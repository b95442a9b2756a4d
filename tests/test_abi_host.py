"""C ABI checks that need no GPU: the library loads, exports every declared symbol,
its structs match the header's layout, and host-side validation behaves."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in sorted(os.listdir(os.path.join(ROOT, "include"))) if h.endswith(".h")]


@pytest.fixture(scope="module")
def lib():
    from paper_2110_13115_gb300 import _native as N, build

    if not os.path.exists(N.LIB_PATH):
        build.build()
    return N.load()


def _declared_functions():
    names = []
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[\w]+\s*\**\s*(rb_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    from paper_2110_13115_gb300 import _native as N

    names = _declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
        assert name in N.SIGNATURES, f"{name} has no binding"
    out = subprocess.run(["nm", "-D", "--defined-only", N.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\s[TW]\s(rb_\w+)$", out, flags=re.M))
    assert set(names) <= exported


def test_struct_layout_matches_header():
    from paper_2110_13115_gb300 import _native as N

    structs = {"rb_filter_desc": N.rb_filter_desc, "rb_basis": N.rb_basis, "rb_trigger": N.rb_trigger,
               "rb_candidate": N.rb_candidate, "rb_filter_sizes": N.rb_filter_sizes}
    extra = getattr(N, "EXTRA_STRUCTS", {})
    structs.update(extra)
    lines = ['#include <stdio.h>', '#include <stddef.h>']
    lines += [f'#include "{h}"' for h in HEADERS]
    lines.append("int main(void) {")
    for name, cls in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines.append("return 0; }")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "l.c")
        exe = os.path.join(d, "l")
        open(src, "w").write("\n".join(lines))
        subprocess.run(["gcc", "-std=c11", src, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    got = dict(line.rsplit(" ", 1) for line in out if line)
    for name, cls in structs.items():
        assert int(got[f"{name} size"]) == C.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(cls, f).offset, (name, f)


def test_plan_validation(lib):
    from paper_2110_13115_gb300 import _native as N
    from paper_2110_13115_gb300.api import make_desc

    def plan(**kw):
        base = dict(fs=1024.0, n=16384, k=16, n_templates=64, w=8)
        base.update(kw)
        d = make_desc(**base)
        out = N.rb_filter_sizes()
        return lib.rb_filter_plan(C.byref(d), C.byref(out)), out

    rc, s = plan()
    assert rc == 0
    assert (s.n1, s.n2, s.n_bins, s.kp) == (128, 128, 1024, 64)
    assert plan(n=12000)[0] == N.RB_ERR_BAD_INPUT
    assert plan(n=1 << 21)[0] == N.RB_ERR_BAD_INPUT
    assert plan(w=3)[0] == N.RB_ERR_BAD_INPUT
    assert plan(k=0)[0] == N.RB_ERR_BAD_INPUT
    assert plan(rho_i=float("nan"))[0] == N.RB_ERR_BAD_INPUT
    assert plan(precision=9)[0] == N.RB_ERR_UNSUPPORTED
    rc, s2 = plan(n=524288, k=256, n_templates=10000, precision="fp16_split")
    assert rc == 0 and (s2.n1, s2.n2, s2.kp) == (512, 1024, 512)
    # second-stage planes (hi, lo) of [T][2 k16] FP16, then first-stage planes (2 x 2T x kp)
    assert s2.coeff_op_bytes == 2 * 10000 * 512 * 2 + 2 * 2 * 10000 * 512 * 2
    rc, s3 = plan(n=524288, k=256, n_templates=10000, precision="fp32")
    assert rc == 0 and s3.coeff_op_bytes == 2 * 10000 * 512 * 2
    # beta (k n/2 complex64) dominates the workspace
    assert s2.workspace_bytes >= 256 * 262144 * 8
    # host trigger staging: a region of max(96 MB, 8 n bytes), carved only when mem asks for host triggers
    assert s2.host_trig_capacity == (96 << 20) // 24
    rc, s4 = plan(n=524288, k=256, n_templates=10000, precision="fp16_split", mem=N.RB_MEM_HOST_TRIGGERS)
    assert rc == 0 and s4.workspace_bytes == s2.workspace_bytes + (96 << 20) // 24 * 24
    assert plan(mem=N.RB_MEM_HOST_STRAIN | N.RB_MEM_HOST_TRIGGERS)[0] == 0
    assert plan(mem=4)[0] == N.RB_ERR_BAD_INPUT
    assert lib.rb_strerror(N.RB_ERR_OVERFLOW) == b"output overflow"
    assert lib.rb_version() >= 100


def test_workspace_per_candidate(lib):
    """Each unit of cand_capacity costs a 16-byte candidate, a 12-byte bucketed (template, block, bin
    mask) record and 1/128 of a 16-byte work piece (buffers are 256-byte aligned). The plan is the larger
    of the hierarchical and the template-method carvings: from 2^20 candidates on, the hierarchical one."""
    from paper_2110_13115_gb300 import _native as N
    from paper_2110_13115_gb300.api import make_desc

    def ws(cap):
        d = make_desc(fs=1024.0, n=16384, k=16, n_templates=64, w=8, cand_capacity=cap)
        out = N.rb_filter_sizes()
        assert lib.rb_filter_plan(C.byref(d), C.byref(out)) == 0
        return out.workspace_bytes

    c0, extra = 1 << 20, 512 * 4096
    grow = ws(c0 + extra) - ws(c0)
    expect = extra * (16 + 12) + extra // 128 * 16
    assert abs(grow - expect) <= 3 * 256, (grow, expect)
    d = make_desc(fs=1024.0, n=16384, k=16, n_templates=64, w=8, cand_capacity=1 << 31)
    out = N.rb_filter_sizes()
    assert lib.rb_filter_plan(C.byref(d), C.byref(out)) == N.RB_ERR_BAD_INPUT


def test_null_arguments_rejected_without_gpu(lib):
    from paper_2110_13115_gb300 import _native as N

    assert lib.rb_filter_plan(None, None) == N.RB_ERR_BAD_INPUT
    assert b"NULL" in lib.rb_last_error_detail()


def test_second_stage_hooks_validate_without_gpu(lib):
    """The host-only second-stage hooks check their arguments on the host (no CUDA call) and leave the
    defaults in place: tcgen05 kernel on, two-slot mma.sync ring, 256-record tcgen05 pieces."""
    from paper_2110_13115_gb300 import _native as N

    for bad in (2, 7, 32 + 1, -1):
        assert lib.rbx_set_stage2_tc(bad) == N.RB_ERR_BAD_INPUT
    for bad in (1, 5, -2):
        assert lib.rbx_set_stage2_ring(bad) == N.RB_ERR_BAD_INPUT
    for bad in (0, 64, 100, 300, 4224, 8192):
        assert lib.rbx_set_stage2_tc_piece(bad) == N.RB_ERR_BAD_INPUT
    for bad in (-1, 3):
        assert lib.rbx_set_stage2_tc_windows(bad) == N.RB_ERR_BAD_INPUT
    try:
        for ok in (128, 384, 4096):
            assert lib.rbx_set_stage2_tc_piece(ok) == 0
        for ok in (0, 16, 32, 1):
            assert lib.rbx_set_stage2_tc(ok) == 0
        for ok in (0, 3, 4, 2):
            assert lib.rbx_set_stage2_ring(ok) == 0
    finally:
        lib.rbx_set_stage2_tc_piece(256)
        lib.rbx_set_stage2_tc(1)
        lib.rbx_set_stage2_ring(2)
        lib.rbx_set_stage2_tc_windows(0)
