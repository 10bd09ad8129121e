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
    declared = set(re.findall(r"^\s*(?:dftu_status|int64_t|int|void|double|const char\*)\s+(dftu_\w+)\s*\(", hdr, re.M))
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
    assert lib.dftu_taylor_step(None, None, None, 0, 1, 1, None, 0.01, 4, None) == 1
    assert lib.dftu_taylor_steps(None, None, 0, 1, 1, None, 0.01, 4, 10, None) == 1
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


def test_radius_methods_match_oracle(lib):
    """Sec. II radius methods 2 and 3 (host functions of the library) against the oracle's statement,
    and the threshold radius against the analytic tail of a hydrogen-like 3d radial."""
    import math
    import numpy as np
    from oracle import dftu_oracle as O
    from paper_1711_08935_gb300 import dftu, synth
    g = synth.Grid((40, 48, 36), (0.3, 0.25, 0.35), periodic=True)
    assert dftu.radius_cell(g) == O.radius_from_cell(g) == min(12.0, 12.0, 12.6)
    rad = synth.hydrogenic_radial(3, 2, 4.0)
    for thr in (1e-2, 1e-3, 1e-5):
        r_lib = dftu.radius_threshold(rad, thr)
        assert r_lib == O.radius_from_threshold(rad.dr, rad.R, thr)
        # R_32 ~ c (8r/3)^2 exp(-4r/3) is monotone beyond its maximum at r = 1.5: the crossing is the root
        c = (8.0 / 3.0) ** 1.5 * math.sqrt(1 / (6 * 120))
        f = lambda r: c * (8 * r / 3) ** 2 * math.exp(-4 * r / 3) - thr
        lo, hi = 1.5, 12.0
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            lo, hi = (mid, hi) if f(mid) > 0 else (lo, mid)
        assert abs(r_lib - lo) <= 2 * rad.dr
    assert dftu.radius_threshold(rad, 1e9) == 0.0
