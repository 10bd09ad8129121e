"""States resident in host memory: the kernels read and write them over the host link, so results must
be bit-identical to the same states in device memory.  Pageable host memory is accepted only where the
GPU reads pageable memory, otherwise refused with DFTU_ERR_INVALID_ARG."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_1711_08935_gb300 import dftu
from tests import _cases as Cs

pytestmark = pytest.mark.gpu


def _setup(dtype):
    s = Cs.periodic_two_atoms()
    nb = 9
    psi = Cs.states_np(s, nb, seed=31)
    f = np.linspace(1.0, 0.2, nb)[None, None, :].repeat(s.nk, 0).repeat(2, 1)
    h = dftu.handle_for_system(s, nb)
    for I, (u, j) in enumerate([(0.3, 0.02), (0.25, 0.01)]):
        h.set_u(I, u, j)
    dev = torch.device("cuda:0")
    d = torch.from_numpy(psi).to(dev).to(dtype)
    host = torch.empty(d.shape, dtype=dtype, pin_memory=True)
    host.copy_(d)
    return s, nb, h, d, host, torch.from_numpy(f).to(dev)


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_pinned_host_states_match_device_states(dtype):
    s, nb, h, d, host, fd = _setup(dtype)
    h.project(d)
    p_dev = h.projections(nb)
    h.project(host)
    p_host = h.projections(nb)
    assert np.array_equal(p_dev, p_host)
    h.occupations(fd)
    h.acbn0_uj()
    h.apply(d)
    h.apply(host)
    torch.cuda.synchronize()
    assert torch.equal(d.cpu(), host)
    # a real-time step with host-resident states and work array
    w_dev, w_host = torch.zeros_like(d), torch.zeros_like(host).pin_memory()
    h.taylor_step(d, w_dev, fd, 0.05)
    h.taylor_step(host, w_host, fd, 0.05)
    torch.cuda.synchronize()
    assert torch.equal(d.cpu(), host)
    assert h.sync_status() == 0
    h.close()


def test_pageable_host_states_are_used_or_refused():
    """Ordinary (not page-locked) host memory: used, with the device result, where the GPU reads
    pageable memory; refused with DFTU_ERR_INVALID_ARG and nothing launched elsewhere."""
    s, nb, h, d, host, fd = _setup(torch.complex128)
    h.project(d)
    p_dev = h.projections(nb)
    pageable = np.ascontiguousarray(host.numpy().copy())
    lib = dftu.load()
    torch.cuda.synchronize()
    st = lib.dftu_project(h.h, C.c_void_p(pageable.ctypes.data), dftu.C128, nb, pageable.shape[3],
                          C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st in (dftu.DFTU_OK, dftu.DFTU_ERR_INVALID_ARG)
    if st == dftu.DFTU_OK:
        assert np.array_equal(h.projections(nb), p_dev)
    else:
        assert b"not addressable" in lib.dftu_last_error(h.h)
        assert np.array_equal(h.projections(nb), p_dev)      # the earlier projections are untouched
    torch.cuda.synchronize()
    h.close()


def test_host_occupations_coefficient_and_vector_potential():
    """The occupations f, the apply coefficient and the vector potential A in page-locked host memory
    give the device-memory results bit for bit; pageable f is used or refused like pageable states."""
    s, nb, h, d, host, fd = _setup(torch.complex128)
    c_dev = torch.tensor([0.3 - 0.1j], dtype=torch.complex128, device="cuda")
    A_dev = torch.tensor([0.2, -0.1, 0.3], dtype=torch.float64, device="cuda")
    runs = {}
    for name, f_, c_, A_ in (("device", fd, c_dev, A_dev),
                             ("host", fd.cpu().pin_memory(), c_dev.cpu().pin_memory(), A_dev.cpu().pin_memory())):
        x = d.clone()
        h.set_vector_potential(None)
        h.project(x); h.occupations(f_); h.acbn0_uj(); h.apply(x, c_)
        h.set_vector_potential(A_)
        h.project(x); h.occupations(f_); h.acbn0_uj(); h.apply(x, c_)
        torch.cuda.synchronize()
        runs[name] = (x.cpu(), h.results()["EU"])
    assert torch.equal(runs["device"][0], runs["host"][0])
    assert runs["device"][1] == runs["host"][1]
    assert h.sync_status() == dftu.DFTU_OK
    h.set_vector_potential(None)
    h.project(d)
    fpage = np.ascontiguousarray(fd.cpu().numpy().copy())
    lib = dftu.load()
    torch.cuda.synchronize()
    st = lib.dftu_occupations(h.h, C.c_void_p(fpage.ctypes.data), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st in (dftu.DFTU_OK, dftu.DFTU_ERR_INVALID_ARG)
    if st == dftu.DFTU_ERR_INVALID_ARG:
        assert b"not addressable" in lib.dftu_last_error(h.h)
    torch.cuda.synchronize()
    h.close()
