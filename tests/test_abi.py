"""The C-ABI library without a GPU: it loads, exports every entry point that
include/tosolve.h declares, its structs have the layout the binding uses,
and host-only validation works (no compute call is made here)."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


@pytest.fixture(scope="module")
def lib():
    from paper_2311_05595_gb300 import build as b

    b.build()
    from paper_2311_05595_gb300 import tosolve as T

    return T


def _declared():
    names = set()
    for hpath in HEADERS:
        src = open(hpath).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(tosolve_\w+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    cdll = ctypes.CDLL(lib._LIB_PATH)
    names = _declared()
    assert "tosolve_create" in names and "tosolve_solve" in names
    for n in names:
        assert hasattr(cdll, n), n


def test_struct_layout_matches_header(lib, tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    prog = tmp_path / "layout.c"
    prog.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "tosolve.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n\","
        " sizeof(tosolve_desc), offsetof(tosolve_desc, E0), offsetof(tosolve_desc, mg_levels),"
        " offsetof(tosolve_desc, max_rhs), sizeof(tosolve_info), offsetof(tosolve_info, status),"
        " sizeof(tosolve_server_desc), offsetof(tosolve_server_desc, maxit),"
        " sizeof(tosolve_request_result), offsetof(tosolve_request_result, t_end),"
        " sizeof(tosolve_server_info), offsetof(tosolve_server_info, now));"
        "return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.check_call([gcc, "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    T = lib
    want = [ctypes.sizeof(T.tosolve_desc), T.tosolve_desc.E0.offset, T.tosolve_desc.mg_levels.offset,
            T.tosolve_desc.max_rhs.offset, ctypes.sizeof(T.tosolve_info), T.tosolve_info.status.offset,
            ctypes.sizeof(T.tosolve_server_desc), T.tosolve_server_desc.maxit.offset,
            ctypes.sizeof(T.tosolve_request_result), T.tosolve_request_result.t_end.offset,
            ctypes.sizeof(T.tosolve_server_info), T.tosolve_server_info.now.offset]
    assert got == want


def test_footprint_and_validation_without_gpu(lib):
    T = lib
    b0 = T.tosolve_footprint(T.make_desc(24, 12, 12, mg_levels=3))
    b1 = T.tosolve_footprint(T.make_desc(48, 24, 24, n_mr=2, rmin=1.5, mg_levels=4,
                                         precision=T.PREC_FP32))
    assert 0 < b0 < b1
    bad = [
        T.make_desc(24, 12, 12, mg_levels=5),      # 12 not divisible by 16
        T.make_desc(0, 12, 12),                    # empty mesh
        T.make_desc(24, 12, 12, degree=4),         # degree not built
        T.make_desc(24, 12, 12, degree=3, mg_levels=1),  # cubic needs its degree-2 level
        T.make_desc(24, 12, 12, degree=1, family=1),     # no linear serendipity element
        T.make_desc(24, 12, 12, nu=0.5),           # incompressible
        T.make_desc(24, 12, 12, Emin=0.0),         # singular void
        T.make_desc(24, 12, 12, cycle_gamma=2),    # W-cycle not built
        T.make_desc(200, 100, 100, mg_levels=1),   # coarse dense solve too large
    ]
    for d in bad:
        with pytest.raises(T.TosolveError) as e:
            T.tosolve_footprint(d)
        assert e.value.status == T.EINVAL
    # create rejects the same descriptors before touching the GPU
    import numpy as np

    with pytest.raises(T.TosolveError) as e:
        T.tosolve_create(bad[0], np.zeros(3 * 25 * 13 * 13, np.uint8))
    assert e.value.status == T.EINVAL


def test_server_validation_without_gpu(lib):
    """Host-side checks of the serving runtime: no request reaches a GPU."""
    import numpy as np

    T = lib
    for bad in [(0, 1 << 30, 1e-8, 100), (4, 0, 1e-8, 100), (4, 1 << 30, 0.0, 100),
                (4, 1 << 30, 1e-8, 0)]:
        with pytest.raises(T.TosolveError) as e:
            T.tosolve_server_create(*bad)
        assert e.value.status == T.EINVAL
    s = T.tosolve_server_create(2, 1 << 30, 1e-8, 100)
    try:
        d = T.make_desc(4, 2, 2, mg_levels=1)
        nd = 3 * 5 * 3 * 3
        T.tosolve_server_add_design(s, 7, d, np.zeros(nd, np.uint8), np.zeros((1, nd)), 1)
        with pytest.raises(T.TosolveError) as e:  # duplicate id
            T.tosolve_server_add_design(s, 7, d, np.zeros(nd, np.uint8), np.zeros((1, nd)), 1)
        assert e.value.status == T.EINVAL
        with pytest.raises(T.TosolveError) as e:  # invalid descriptor
            T.tosolve_server_add_design(s, 8, T.make_desc(4, 2, 2, degree=4), np.zeros(nd, np.uint8),
                                        np.zeros((1, nd)), 1)
        assert e.value.status == T.EINVAL
        with pytest.raises(T.TosolveError) as e:  # unknown design
            T.tosolve_server_submit(s, 9, np.zeros(16))
        assert e.value.status == T.EINVAL
        info = T.tosolve_server_stats(s)
        assert info.designs == 1 and info.resident_designs == 0 and info.pending == 0
        assert T.tosolve_server_poll(s, 4, 0) == []
    finally:
        T.tosolve_server_destroy(s)
