"""The allocation-free projection entry point (dftu_project_sphere_noalloc), called through the C ABI.

It serves callers that cannot allocate GPU memory (an application that owns the whole device pool, a
real-time loop where allocation is forbidden, plug-in code that only receives pointers); its scratch
is a fixed array in the library's device image.  Its projections must match the oracle's definition
(p = dV sum_j phi_m(j) phase_j psi(idx_j)) and the handle-based dftu_project, on calls in a row that
share the scratch: a large call close to the scratch limit first, then small calls that must not read
its stale partial sums.  A warm call must not change the device's free memory.  This file is
collected last on purpose.
"""
import ctypes as C
from types import SimpleNamespace

import numpy as np
import pytest
import torch

from oracle import dftu_oracle as O
from paper_1711_08935_gb300 import dftu
from tests import _cases

pytestmark = pytest.mark.gpu

SCRATCH_ELEMS = 524288      # complex partial sums the fixed scratch holds (ceil(npts/512) * nbands * M)


def _noalloc(lib, psi_rows, idx_d, ph_d, phi_d, M, dV, out):
    nb, ld = psi_rows.shape
    prec = dftu.C128 if psi_rows.dtype == torch.complex128 else dftu.C64
    st = torch.cuda.current_stream().cuda_stream
    return lib.dftu_project_sphere_noalloc(C.c_void_p(psi_rows.data_ptr()), prec, nb, ld, C.c_void_p(idx_d.data_ptr()),
                                           C.c_void_p(ph_d.data_ptr()) if ph_d is not None else None,
                                           C.c_void_p(phi_d.data_ptr()), idx_d.numel(), M, dV,
                                           C.c_void_p(out.data_ptr()), C.c_void_p(st))


def _oracle_rows(psi_rows_np, idx, T, phi, dV, L, k):
    """oracle.project on one (k, spin) block of rows, with the sphere given as a map dict."""
    sysw = SimpleNamespace(grid=SimpleNamespace(dV=dV, L=L), kpts=np.array([k], dtype=np.float64))
    sm = {"idx": idx, "T": T, "phi": phi}
    return O.project(sysw, [sm], psi_rows_np[None, None])[0][0, 0]


def _large_call(lib):
    """A call that fills the scratch almost to its limit (M = 7, 128 bands, 585 tiles) with non-zero data."""
    rng = np.random.default_rng(5)
    nb, M, npts, ld = 128, 7, 585 * 512, 300_000
    assert -(-npts // 512) * nb * M <= SCRATCH_ELEMS
    psi = (rng.standard_normal((nb, ld)) + 1j * rng.standard_normal((nb, ld))).astype(np.complex128)
    idx = rng.integers(0, ld, npts).astype(np.int32)
    phi = rng.standard_normal((npts, M))
    T = rng.integers(-1, 2, (npts, 3)).astype(np.int32)
    L = np.array([7.0, 8.0, 9.0])
    k = np.array([0.3, -0.2, 0.45])
    ph = np.exp(1j * ((T * L[None, :]) @ k))
    dV = 0.015625
    out = torch.full((nb, M), float("nan"), dtype=torch.complex128, device="cuda")
    psi_d = torch.from_numpy(psi).cuda()
    assert _noalloc(lib, psi_d, torch.from_numpy(idx).cuda(), torch.from_numpy(ph).cuda(),
                    torch.from_numpy(phi).cuda(), M, dV, out) == dftu.DFTU_OK
    ref = _oracle_rows(psi, idx, T, phi, dV, L, k)
    got = out.cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_noalloc_projection_matches_oracle_and_handle(dtype):
    lib = dftu.load()
    _large_call(lib)                       # leaves a nearly full scratch of other partial sums behind
    s = _cases.periodic_two_atoms()
    nb = 9
    psi_np = _cases.states_np(s, nb, seed=17)
    psi = torch.from_numpy(psi_np).cuda().to(dtype)
    psi_seen = psi.to(torch.complex128).cpu().numpy()           # the values the GPU reads, in FP64
    h = dftu.handle_for_system(s, nb)
    h.project(psi)
    p_handle = h.projections(nb)                                 # [k*s][band][sum M]
    st = O.setup_atoms(s)
    p_oracle = O.project(s, st, psi_seen)                        # per atom [k][s][band][M]
    L = np.array(s.grid.L)
    # the entry point sums in FP64 whatever the state precision; the handle sums complex64 states in FP32
    tol_handle = 1e-12 if dtype == torch.complex128 else 2e-6
    moff = 0
    for I, at in enumerate(s.atoms):
        M = 2 * at.l + 1
        idx, img, phi = h.get_sphere(I)
        assert np.array_equal(idx, st[I]["idx"]) and np.array_equal(img, st[I]["T"])
        idx_d = torch.from_numpy(idx).cuda()
        phi_d = torch.from_numpy(np.ascontiguousarray(phi)).cuda()
        for call, (k, sp) in enumerate([(0, 0), (1, 1), (1, 1)]):  # two calls in a row on the same input, too
            ph = np.exp(1j * ((img * L[None, :]) @ s.kpts[k]))
            ph_d = torch.from_numpy(np.ascontiguousarray(ph)).cuda()
            out = torch.full((nb, M), float("nan"), dtype=torch.complex128, device="cuda")
            assert _noalloc(lib, psi[k, sp], idx_d, ph_d, phi_d, M, s.grid.dV, out) == dftu.DFTU_OK
            got = out.cpu().numpy()
            ref = p_oracle[I][k, sp]
            assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref)), (I, call)
            ref_h = p_handle[k * 2 + sp][:, moff:moff + M]
            assert np.max(np.abs(got - ref_h)) <= tol_handle * np.max(np.abs(ref_h)), (I, call)
        moff += M
    h.close()


def test_noalloc_without_phase_at_gamma_and_allocates_nothing():
    """phase = NULL means a factor 1 (a Gamma-point or isolated-box caller); a warm call leaves the
    device's free memory unchanged."""
    lib = dftu.load()
    s = _cases.periodic_two_atoms(k=((0.0, 0.0, 0.0),))
    nb = 7
    psi_np = _cases.states_np(s, nb, seed=23)
    psi = torch.from_numpy(psi_np).cuda()
    st = O.setup_atoms(s)
    p_oracle = O.project(s, st, psi_np)
    for I, at in enumerate(s.atoms):
        M = 2 * at.l + 1
        idx_d = torch.from_numpy(st[I]["idx"].astype(np.int32)).cuda()
        phi_d = torch.from_numpy(np.ascontiguousarray(st[I]["phi"])).cuda()
        out = torch.zeros((nb, M), dtype=torch.complex128, device="cuda")
        out.fill_(float("nan"))                  # warm call, with every kernel the measured loop launches
        assert _noalloc(lib, psi[0, 0], idx_d, None, phi_d, M, s.grid.dV, out) == dftu.DFTU_OK
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        for _ in range(3):
            out.fill_(float("nan"))
            assert _noalloc(lib, psi[0, 0], idx_d, None, phi_d, M, s.grid.dV, out) == dftu.DFTU_OK
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0
        ref = p_oracle[I][0, 0]
        assert np.max(np.abs(out.cpu().numpy() - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_noalloc_rejects_bad_arguments_and_out_of_range_indices():
    lib = dftu.load()
    idx = torch.zeros(600 * 512, dtype=torch.int32, device="cuda")
    phi = torch.zeros((600 * 512, 7), dtype=torch.float64, device="cuda")
    out = torch.zeros((200, 7), dtype=torch.complex128, device="cuda")
    big = torch.zeros((200, 8), dtype=torch.complex128, device="cuda")
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    # 600 tiles x 200 bands x 7 orbitals is beyond the fixed scratch
    r = lib.dftu_project_sphere_noalloc(C.c_void_p(big.data_ptr()), dftu.C128, 200, 8, C.c_void_p(idx.data_ptr()), None,
                                        C.c_void_p(phi.data_ptr()), idx.numel(), 7, 1.0, C.c_void_p(out.data_ptr()), st)
    assert r == dftu.DFTU_ERR_INVALID_ARG
    assert lib.dftu_project_sphere_noalloc(None, 0, 1, 8, None, None, None, 1, 1, 1.0, None, st) == dftu.DFTU_ERR_INVALID_ARG
    # an index outside [0, ld_band) is never read: the projections come out NaN, and the next call is clean
    psi = torch.ones((2, 8), dtype=torch.complex128, device="cuda")
    bad_idx = torch.tensor([0, 3, 8, 1], dtype=torch.int32, device="cuda")
    phi1 = torch.ones((4, 3), dtype=torch.float64, device="cuda")
    o = torch.zeros((2, 3), dtype=torch.complex128, device="cuda")
    assert _noalloc(lib, psi, bad_idx, None, phi1, 3, 1.0, o) == dftu.DFTU_OK
    assert torch.isnan(o.real).all()
    good_idx = torch.tensor([0, 3, 7, 1], dtype=torch.int32, device="cuda")
    assert _noalloc(lib, psi, good_idx, None, phi1, 3, 1.0, o) == dftu.DFTU_OK
    assert torch.allclose(o, torch.full_like(o, 4.0))
