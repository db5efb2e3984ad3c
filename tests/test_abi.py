"""The C-ABI library builds for sm_103a and exports every entry point that
include/figaro.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "figaro.h")


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"FIGARO_API\s+[\w\s\*]+?\b(figaro_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2503_23385_gb300 import _build
    return _build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["figaro_join_qr_r", "figaro_join_singular_values", "figaro_join_group", "figaro_join_head_tail",
                 "figaro_batch_join", "figaro_workspace_size", "figaro_get_status"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(figaro_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_library_loads_and_answers_host_only_calls(lib_path):
    import paper_2503_23385_gb300 as fg
    lib = fg.library()
    for name in declared_functions():
        assert hasattr(lib, name)
    assert lib.figaro_version() > 0
    assert lib.figaro_status_string(0) == b"ok"
    o = fg.Options()
    assert lib.figaro_default_options(ctypes.byref(o)) == 0
    assert o.path == fg.PATH_MIXED
    # argument checks happen on the host, before any device work
    assert lib.figaro_default_options(None) == 1


def test_workspace_size_and_argument_checks_on_host(lib_path):
    import paper_2503_23385_gb300 as fg
    lib = fg.library()
    A = fg.Table(None, None, 1000, 16, 16, fg.F32, fg.MEM_DEVICE, 0)
    B = fg.Table(None, None, 0, 16, 16, fg.F32, fg.MEM_DEVICE, 0)
    sz = ctypes.c_size_t(0)
    # m > 0 with null pointers is an invalid argument
    assert lib.figaro_workspace_size(ctypes.byref(A), ctypes.byref(B), None, ctypes.byref(sz)) == 1
    A.x, A.key = 16, 16  # non-null placeholders: the size query never dereferences them
    assert lib.figaro_workspace_size(ctypes.byref(A), ctypes.byref(B), None, ctypes.byref(sz)) == 0
    assert sz.value > 1000 * 16 * 4
    # widths: n1 + n2 <= 512 with each table at most 256 columns once n1 + n2 > 128
    for (na, nb), code in (((100, 100), 0), ((256, 256), 0), ((300, 10), 7), ((257, 200), 7), ((300, 300), 7),
                           ((64, 64), 0), ((120, 8), 0)):
        ta = fg.Table(16, 16, 10, na, na, fg.F32, fg.MEM_DEVICE, 0)
        tb = fg.Table(16, 16, 10, nb, nb, fg.F32, fg.MEM_DEVICE, 0)
        assert lib.figaro_workspace_size(ctypes.byref(ta), ctypes.byref(tb), None, ctypes.byref(sz)) == code, (na, nb)
    bad = fg.Table(16, 16, 10, 3, 4, fg.F32, fg.MEM_DEVICE, 0)  # ld < n
    assert lib.figaro_workspace_size(ctypes.byref(bad), ctypes.byref(A), None, ctypes.byref(sz)) == 1
    mixed = fg.Table(16, 16, 10, 4, 4, fg.F64, fg.MEM_DEVICE, 0)  # dtype mismatch with A
    assert lib.figaro_workspace_size(ctypes.byref(A), ctypes.byref(mixed), None, ctypes.byref(sz)) == 1


def test_batch_schedule_query_on_host(lib_path):
    """Without a tuned entry the batch schedule is the default one (host-only call)."""
    import paper_2503_23385_gb300 as fg
    lib = fg.library()
    TA = (fg.Table * 2)(fg.Table(16, 16, 1000, 8, 8, fg.F32, fg.MEM_DEVICE, 0),
                        fg.Table(16, 16, 5000, 16, 16, fg.F32, fg.MEM_DEVICE, 0))
    TB = (fg.Table * 2)(fg.Table(16, 16, 2000, 8, 8, fg.F32, fg.MEM_DEVICE, 0),
                        fg.Table(16, 16, 300, 32, 32, fg.F32, fg.MEM_DEVICE, 0))
    rpc, hts = ctypes.c_int64(0), ctypes.c_int32(0)
    assert lib.figaro_batch_schedule(2, TA, TB, None, ctypes.byref(rpc), ctypes.byref(hts)) == 0
    assert (rpc.value, hts.value) == (4096, 2)
    assert lib.figaro_batch_schedule(2, TA, TB, None, None, ctypes.byref(hts)) == 1
