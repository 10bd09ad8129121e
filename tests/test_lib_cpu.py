"""Host-side checks of the C-ABI library (no GPU): it loads, exports every declared symbol, and the
binding rejects bad arguments before reaching the device."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1711_08935_gb300 import build_lib, dftu
    if not os.path.exists(dftu.LIB_PATH):
        build_lib.build()
    return dftu.load()


def test_header_declarations_are_exported(lib):
    from paper_1711_08935_gb300 import dftu
    hdr = open(os.path.join(ROOT, "include", "dftu.h")).read()
    declared = set(re.findall(r"^\s*(?:dftu_status|int|void|const char\*)\s+(dftu_\w+)\s*\(", hdr, re.M))
    assert declared == set(dftu.EXPORTED)
    out = subprocess.run(["nm", "-D", "--defined-only", dftu.LIB_PATH], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if l.split() and l.split()[-1].startswith("dftu_")}
    assert declared <= exported
    for name in declared:
        assert hasattr(lib, name)


def test_null_handle_calls_are_rejected(lib):
    assert lib.dftu_project(None, None, 0, 1, 1, None) == 1
    assert lib.dftu_occupations(None, None, None) == 1
    assert lib.dftu_acbn0_uj(None, None) == 1
    assert lib.dftu_apply(None, None, 0, 1, 1, None, 1, None) == 1
    assert lib.dftu_sync_status(None) == 1
    assert lib.dftu_last_error(None) == b"null handle"
    lib.dftu_destroy(None)


def test_create_without_gpu_fails_cleanly(lib):
    """No CUDA device here: creation must fail with an error code, not crash."""
    import ctypes as C
    import torch
    from paper_1711_08935_gb300 import dftu
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    g = dftu.DftuGrid((C.c_int * 3)(8, 8, 8), (C.c_double * 3)(0.3, 0.3, 0.3), (C.c_double * 3)(0, 0, 0), 1)
    h = C.c_void_p()
    k = (C.c_double * 3)(0, 0, 0)
    w = (C.c_double * 1)(1.0)
    st = lib.dftu_create(C.byref(h), C.byref(g), 1, k, w, 0, 4, 0)
    assert st == dftu.DFTU_ERR_INVALID_ARG and not h.value
