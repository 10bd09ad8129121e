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


def _oracle_p(s, st, psi):
    return np.concatenate(O.project(s, st, psi), axis=-1)   # [k][s][n][sum_I M_I], atom order


@pytest.mark.parametrize("case", ["overlapping", "disjoint"])
def test_taylor_steps_fused_gather_matches_oracle(case):
    """dftu_taylor_steps on complex64 states: the scatter of each step also projects the values it writes
    (on the tiles no later apply colour touches; the rest are projected after the last colour).  Over 10
    steps the states follow the oracle's steps, the handle's projections afterwards are the oracle's
    projections of the outgoing states, and U follows the last step's incoming states.  'overlapping':
    spheres overlap each other and their own images (tiles of both kinds); 'disjoint': one apply colour,
    every tile final."""
    if case == "overlapping":
        s, st, psi, f, coul, h = _setup(torch.complex64)
    else:
        s = C.periodic_two_atoms(nspin=2)
        st = O.setup_atoms(s)
        psi = C.states_np(s, 6, seed=31)
        f = np.random.default_rng(31).uniform(0.2, 1.0, (s.nk, 2, 6))
        coul = [O.coulomb_integrals(s.grid, s.atoms[sp], st[sp]) for sp in range(2)]
        h = dftu.handle_for_system(s, 6)
        for sp in range(2):
            h.set_coulomb(sp, coul[sp])
    dt, steps = 0.5, 10
    dev = torch.device("cuda:0")
    t = torch.from_numpy(psi).to(dev).to(torch.complex64)
    fd = torch.from_numpy(f).to(dev)
    ref = t.to(torch.complex128).cpu().numpy()             # the oracle starts from the same rounded states
    for _ in range(steps):
        ref, base = O.taylor_step(s, st, ref, f, dt, coulomb=coul)
    h.taylor_steps(t, fd, dt, steps, order=4)
    got = t.to(torch.complex128).cpu().numpy()
    assert np.max(np.abs(got - ref)) < 2e-6 * np.max(np.abs(ref))
    p_ref = _oracle_p(s, st, got).reshape(-1, psi.shape[2], h.lib.dftu_total_orbitals(h.h))
    p = h.projections(psi.shape[2])
    assert np.max(np.abs(p - p_ref)) < 2e-6 * np.max(np.abs(p_ref))
    r = h.results()
    assert np.allclose(r["U"], base["U"], rtol=1e-4)
    assert h.sync_status() == dftu.DFTU_OK


def test_taylor_steps_fused_equals_single_steps_within_fp32():
    """The fused steps and as many dftu_taylor_step calls on the same complex64 states differ only by the
    FP32 summation order of the gathers."""
    s, st, psi, f, coul, h = _setup(torch.complex64, nb=7, seed=5)
    dev = torch.device("cuda:0")
    fd = torch.from_numpy(f).to(dev)
    a = torch.from_numpy(psi).to(dev).to(torch.complex64)
    b = a.clone()
    h.taylor_steps(a, fd, 0.4, 6)
    ua = h.results()["U"]
    for _ in range(6):
        h.taylor_step(b, None, fd, 0.4)
    ub = h.results()["U"]
    assert (a - b).abs().max().item() < 1e-6 * b.abs().max().item()
    assert np.allclose(ua, ub, rtol=1e-5)


def test_taylor_steps_complex128_are_single_steps_in_turn():
    """Without the fused form (complex128) the steps run one projection and one apply at a time: the
    states equal those of successive dftu_taylor_step calls bit for bit."""
    s, st, psi, f, coul, h = _setup(nb=5, seed=8)
    dev = torch.device("cuda:0")
    fd = torch.from_numpy(f).to(dev)
    a = torch.from_numpy(psi).to(dev)
    b = a.clone()
    h.taylor_steps(a, fd, 0.3, 3)
    for _ in range(3):
        h.taylor_step(b, None, fd, 0.3)
    assert torch.equal(a, b)


def test_taylor_steps_in_cuda_graph_replays_identically():
    s, st, psi, f, coul, h = _setup(torch.complex64, nb=5, seed=9)
    dev = torch.device("cuda:0")
    fd = torch.from_numpy(f).to(dev)
    a = torch.from_numpy(psi).to(dev).to(torch.complex64)
    h.taylor_steps(a, fd, 0.3, 3)
    h.taylor_steps(a, fd, 0.3, 3)
    torch.cuda.synchronize()
    b = torch.from_numpy(psi).to(dev).to(torch.complex64)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        h.taylor_steps(b, fd, 0.3, 3)                        # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        h.taylor_steps(b, fd, 0.3, 3)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(a, b)
