"""Host-side checks of the C-ABI library: it builds for sm_103a, loads, exports every entry
point declared in include/ntf.h, the binding's structures match the header's, and it rejects
bad arguments before touching the GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1409_2383_gb300 import build, ntf
    build.build()
    return ntf.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "ntf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ntf_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "ntf_create" in names and "ntf_mttkrp" in names and "ntf_admm_update" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    from paper_1409_2383_gb300 import ntf
    assert set(_declared()) == set(ntf._SIGS)


def test_default_params(lib):
    from paper_1409_2383_gb300 import ntf
    p = ntf.default_params(paper_mode=True)
    assert (p.inner_iters, p.kr_source, p.rho_policy) == (1, ntf.NTF_KR_PRIMAL, ntf.NTF_RHO_ADAPTIVE)
    assert (p.rho0, p.mu, p.tau_incr, p.tau_decr, p.eps_abs, p.eps_rel) == (1, 8, 4, 2, 1e-4, 1e-4)
    q = ntf.default_params(paper_mode=False)
    assert (q.inner_iters, q.kr_source, q.rho_policy) == (5, ntf.NTF_KR_AUX, ntf.NTF_RHO_TRACE)


@pytest.mark.parametrize("order,rank,dtype,ptr", [(5, 3, 0, 16), (2, 3, 0, 16), (3, 0, 0, 16),
                                                   (3, 65, 0, 16), (3, 3, 7, 16), (3, 3, 0, 0)])
def test_create_rejects_bad_arguments_before_any_launch(lib, order, rank, dtype, ptr):
    from paper_1409_2383_gb300 import ntf
    h = ctypes.c_void_p()
    dims = (ctypes.c_int64 * 5)(4, 5, 6, 7, 8)
    p = ntf.default_params()
    st = lib.ntf_create(ctypes.byref(h), order, dims, rank, dtype, ptr or None, ctypes.byref(p), None)
    assert st == 1 and not h.value
    assert lib.ntf_last_error()


@pytest.mark.parametrize("dims", [(1 << 30, 1 << 30, 1 << 30), (1 << 16, 1 << 16, 2),
                                  (2, 1 << 16, 1 << 16), (1 << 30,) * 4])
def test_create_rejects_oversized_halves_before_any_launch(lib, dims):
    """A half of the tensor's matrix views with 2^31 or more entries is refused as
    unsupported (without forming the overflowing size of the whole tensor)."""
    from paper_1409_2383_gb300 import ntf
    h = ctypes.c_void_p()
    d = (ctypes.c_int64 * len(dims))(*dims)
    p = ntf.default_params()
    st = lib.ntf_create(ctypes.byref(h), len(dims), d, 3, 0, 16, ctypes.byref(p), None)
    assert st == 8 and not h.value
    assert b"2^31" in lib.ntf_last_error()


def test_noalloc_mttkrp_rejects_oversized_halves_before_any_launch(lib):
    dims = (ctypes.c_int64 * 3)(1 << 30, 1 << 30, 1 << 30)
    F = (ctypes.c_void_p * 3)(16, 16, 16)
    assert lib.ntf_mttkrp_noalloc(3, dims, 3, 0, 16, 0, F, 16, None) == 8
    dims4 = (ctypes.c_int64 * 4)(*(1 << 30,) * 4)
    F4 = (ctypes.c_void_p * 4)(16, 16, 16, 16)
    assert lib.ntf_mttkrp_noalloc(4, dims4, 3, 0, 16, 3, F4, 16, None) == 8


def test_create_rejects_bad_params(lib):
    from paper_1409_2383_gb300 import ntf
    h = ctypes.c_void_p()
    dims = (ctypes.c_int64 * 3)(4, 5, 6)
    for bad in (dict(inner_iters=0), dict(rho0=-1.0), dict(mu=1.0, rho_policy=0),
                dict(kr_source=3), dict(rho_policy=9), dict(eps_abs=-1.0),
                dict(fuse_level=2), dict(tensor_copy=-2)):
        p = ntf.default_params(**bad)
        assert lib.ntf_create(ctypes.byref(h), 3, dims, 3, 0, 16, ctypes.byref(p), None) == 1


def test_null_context_calls_fail_cleanly(lib):
    assert lib.ntf_destroy(None) == 0
    assert lib.ntf_sync(None) == 1
    assert lib.ntf_watchdog_check(None, ctypes.c_double(10.0)) == 1
    assert lib.ntf_mttkrp(None, 0, None, None) == 1
    assert lib.ntf_to_bf16(None, None, 4, None) == 1
    assert lib.ntf_status_string(4) == b"coefficient matrix not positive definite"


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes structures have the size and field offsets of the header's
    structs (compiled with the host C compiler against include/ntf.h)."""
    import shutil
    import subprocess
    from paper_1409_2383_gb300 import ntf
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    pairs = {"ntf_params": ntf.Params, "ntf_update_stats": ntf.UpdateStats,
             "ntf_run_stats": ntf.RunStats, "ntf_profile": ntf.Profile,
             "ntf_trace_entry": ntf.TraceEntry}
    lines = ["#include <stdio.h>", '#include "ntf.h"', "int main(void) {"]
    for cname, py in pairs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in py._fields_:
            lines.append(f'  printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-std=c11", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], check=True, capture_output=True,
                             text=True).stdout.splitlines():
        cname, key, val = ln.split()
        got[(cname, key)] = int(val)
    for cname, py in pairs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for field, _ in py._fields_:
            assert got[(cname, field)] == getattr(py, field).offset, (cname, field)


def test_binding_constants_match_the_header():
    """Every enum constant of the header has the same value in the binding (status codes in
    its STATUS table, the others as module constants)."""
    from paper_1409_2383_gb300 import ntf
    with open(os.path.join(ROOT, "include", "ntf.h")) as f:
        consts = {k: int(v) for k, v in re.findall(r"\b(NTF_[A-Z0-9_]+)\s*=\s*(\d+)", f.read())}
    assert len(consts) >= 19
    for name, value in consts.items():
        if name == "NTF_OK" or name.startswith("NTF_ERR_"):
            assert ntf.STATUS[value] == name
        else:
            assert getattr(ntf, name) == value, name


def test_misaligned_pointers_are_refused_before_any_launch(lib):
    """Pointers that are not multiples of their element size are invalid arguments (the
    kernels read every array with loads of its element type at least)."""
    from paper_1409_2383_gb300 import ntf
    h = ctypes.c_void_p()
    dims = (ctypes.c_int64 * 3)(4, 5, 6)
    p = ntf.default_params()
    for dtype, ptr in ((0, 18), (0, 17), (1, 17)):
        st = lib.ntf_create(ctypes.byref(h), 3, dims, 3, dtype, ptr, ctypes.byref(p), None)
        assert st == 1 and not h.value and b"aligned" in lib.ntf_last_error()
    assert lib.ntf_to_bf16(18, 16, 4, None) == 1
    assert lib.ntf_to_bf16(16, 17, 4, None) == 1
    ok = (ctypes.c_void_p * 3)(16, 16, 16)
    bad = (ctypes.c_void_p * 3)(16, 18, 16)
    assert lib.ntf_mttkrp_noalloc(3, dims, 3, 0, 18, 0, ok, 16, None) == 1   # tensor
    assert lib.ntf_mttkrp_noalloc(3, dims, 3, 0, 16, 0, bad, 16, None) == 1  # factor 1
    assert lib.ntf_mttkrp_noalloc(3, dims, 3, 0, 16, 0, ok, 18, None) == 1   # output
