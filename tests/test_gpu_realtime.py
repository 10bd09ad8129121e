"""Real-time step (Sec. V, Eq. 15) on the GPU: the library's Taylor step against the oracle's on a
10-step prefix, norm conservation per step, the accumulate/assign apply with overlapping spheres, and
replay of the step captured in a CUDA graph."""
import numpy as np
import pytest
import torch

from oracle import dftu_oracle as O
from paper_1711_08935_gb300 import dftu
from tests import _cases as C

pytestmark = pytest.mark.gpu


def _setup(dtype=torch.complex128, nb=6, seed=23):
    s = C.overlapping_three_atoms()
    st = O.setup_atoms(s)
    psi = C.states_np(s, nb, seed=seed)
    f = np.random.default_rng(seed).uniform(0.2, 1.0, (s.nk, 1, nb))
    coul = []
    for sp in range(3):
        coul.append(O.coulomb_integrals(s.grid, s.atoms[sp], st[sp]))
    h = dftu.handle_for_system(s, nb)
    for sp in range(3):
        h.set_coulomb(sp, coul[sp])
    return s, st, psi, f, coul, h


def test_assign_mode_with_overlapping_spheres():
    s, st, psi, f, coul, h = _setup()
    ref = O.hubbard_pass(s, st, psi, f, coulomb=coul, coef=1.0)
    dev = torch.device("cuda:0")
    t = torch.from_numpy(psi).to(dev)
    h.project(t)
    h.occupations(torch.from_numpy(f).to(dev))
    h.acbn0_uj()
    out = torch.full_like(t, complex(3.0, -1.0))          # garbage outside the spheres must survive
    h.apply(out, accumulate=False)
    got = out.cpu().numpy()
    delta = ref["psi_out"] - psi                           # V_U psi (every sphere's contribution)
    mask = np.zeros(s.grid.npts, dtype=bool)
    for sm in st:
        mask[sm["idx"]] = True
    assert np.max(np.abs(got[..., mask] - delta[..., mask])) < 1e-12 * np.max(np.abs(delta))
    assert np.all(got[..., ~mask] == complex(3.0, -1.0))


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_taylor_steps_match_oracle_and_conserve_norm(dtype):
    s, st, psi, f, coul, h = _setup(dtype)
    dt, steps = 0.5, 10
    dev = torch.device("cuda:0")
    t = torch.from_numpy(psi).to(dev).to(dtype)
    work = torch.zeros_like(t)
    fd = torch.from_numpy(f).to(dev)
    ref = psi.copy()
    n0 = s.grid.dV * np.sum(np.abs(psi) ** 2, axis=-1)
    for step in range(steps):
        ref, base = O.taylor_step(s, st, ref, f, dt, coulomb=coul)
        h.taylor_step(t, work, fd, dt, order=4)
        got = t.to(torch.complex128).cpu().numpy()
        rel = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
        assert rel < (1e-11 if dtype == torch.complex128 else 2e-6), (step, rel)
        nrm = s.grid.dV * np.sum(np.abs(got) ** 2, axis=-1)
        if dtype == torch.complex128:
            assert np.max(np.abs(nrm - n0)) < 1e-10 * (step + 1)
    r = h.results()
    assert np.allclose(r["U"], base["U"], rtol=1e-9 if dtype == torch.complex128 else 1e-4)
    assert h.sync_status() == dftu.DFTU_OK


def test_taylor_step_in_cuda_graph_replays_identically():
    s, st, psi, f, coul, h = _setup(nb=5, seed=3)
    dev = torch.device("cuda:0")
    fd = torch.from_numpy(f).to(dev)
    a = torch.from_numpy(psi).to(dev)
    wa = torch.zeros_like(a)
    for _ in range(3):
        h.taylor_step(a, wa, fd, 0.3)
    torch.cuda.synchronize()
    b = torch.from_numpy(psi).to(dev)
    wb = torch.zeros_like(b)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        h.taylor_step(b, wb, fd, 0.3)                        # warm-up outside the capture (1 step)
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        h.taylor_step(b, wb, fd, 0.3)
    g.replay()                                              # steps 2 and 3
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(a, b)
