"""The allocation-free projection entry point (dftu_project_sphere_noalloc), called through the C ABI.

It serves callers that cannot allocate GPU memory; its scratch is a fixed array in the library's
device image.  Its projections of each atom must match the handle-based dftu_project within the
FP64 tolerance of the other parity tests, on two calls in a row (the second call reuses scratch that
still holds the first call's partial sums).  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_1711_08935_gb300 import dftu
from tests import _cases

pytestmark = pytest.mark.gpu


def _noalloc(lib, psi_rows, idx_d, ph_d, phi_d, M, dV, out):
    nb, ld = psi_rows.shape
    prec = dftu.C128 if psi_rows.dtype == torch.complex128 else dftu.C64
    st = torch.cuda.current_stream().cuda_stream
    return lib.dftu_project_sphere_noalloc(C.c_void_p(psi_rows.data_ptr()), prec, nb, ld, C.c_void_p(idx_d.data_ptr()),
                                           C.c_void_p(ph_d.data_ptr()) if ph_d is not None else None,
                                           C.c_void_p(phi_d.data_ptr()), idx_d.numel(), M, dV,
                                           C.c_void_p(out.data_ptr()), C.c_void_p(st))


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_noalloc_projection_matches_handle_projection(dtype):
    s = _cases.periodic_two_atoms()
    nb = 9
    psi = torch.from_numpy(_cases.states_np(s, nb, seed=17)).cuda().to(dtype)
    h = dftu.handle_for_system(s, nb)
    h.project(psi)
    p_ref = h.projections(nb)                                    # [k*s][band][sum M]
    lib = dftu.load()
    L = np.array(s.grid.L)
    # FP64 path: 1e-12 as the other parity tests; complex64 states: the handle sums them in FP32 (2e-6)
    tol = 1e-12 if dtype == torch.complex128 else 2e-6
    moff = 0
    for I, at in enumerate(s.atoms):
        M = 2 * at.l + 1
        idx, img, phi = h.get_sphere(I)
        idx_d = torch.from_numpy(idx).cuda()
        phi_d = torch.from_numpy(np.ascontiguousarray(phi)).cuda()
        for call, (k, sp) in enumerate([(0, 0), (1, 1), (1, 1)]):  # two calls in a row on the same input, too
            ph = np.exp(1j * ((img * L[None, :]) @ s.kpts[k]))
            ph_d = torch.from_numpy(np.ascontiguousarray(ph)).cuda()
            out = torch.full((nb, M), float("nan"), dtype=torch.complex128, device="cuda")
            assert _noalloc(lib, psi[k, sp], idx_d, ph_d, phi_d, M, s.grid.dV, out) == dftu.DFTU_OK
            got = out.cpu().numpy()
            ref = p_ref[k * 2 + sp][:, moff:moff + M]
            assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref)), (I, call)
        moff += M
    h.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib = dftu.load()
    x = torch.zeros((1, 8), dtype=torch.complex128, device="cuda")
    idx = torch.zeros(600 * 512, dtype=torch.int32, device="cuda")
    phi = torch.zeros((600 * 512, 7), dtype=torch.float64, device="cuda")
    out = torch.zeros((200, 7), dtype=torch.complex128, device="cuda")
    big = torch.zeros((200, 8), dtype=torch.complex128, device="cuda")
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    r = lib.dftu_project_sphere_noalloc(C.c_void_p(big.data_ptr()), dftu.C128, 200, 8, C.c_void_p(idx.data_ptr()), None,
                                        C.c_void_p(phi.data_ptr()), idx.numel(), 7, 1.0, C.c_void_p(out.data_ptr()), st)
    assert r == dftu.DFTU_ERR_INVALID_ARG
    assert lib.dftu_project_sphere_noalloc(None, 0, 1, 8, None, None, None, 1, 1, 1.0, None, st) == dftu.DFTU_ERR_INVALID_ARG
    del x
