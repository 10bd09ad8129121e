"""Gauge-invariant Hubbard operator (Sec. V, Eq. 16) and Hubbard current (Eq. 17) on the GPU against the
oracle, element by element.  Tolerances as for the plain operator: 1e-12 relative to the largest element
for complex128 states (FP32-pair and native FP64), 2e-6 for complex64 states."""
import numpy as np
import pytest
import torch

from oracle import dftu_oracle as O
from paper_1711_08935_gb300 import dftu, synth
from tests import _cases as C
from tests._gpu import split_p

pytestmark = pytest.mark.gpu

A_VEC = np.array([0.41, -0.27, 0.33])   # |A.d| reaches ~2 rad on spheres of radius 3 bohr

SYSTEMS = {
    "periodic_two_atoms": C.periodic_two_atoms,
    "periodic_self_overlap": C.periodic_tiny,
    "overlapping_three_atoms": C.overlapping_three_atoms,
}


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _fixed_u(s):
    return [(0.3 + 0.1 * I, 0.02 * (I + 1)) for I in range(len(s.atoms))]


def _oracle_gauge_pass(s, st, psi, f, U, A, coef=1.0):
    p = O.project_gauge(s, st, psi, A)
    occ = O.occupations(s, p, f)
    V = [np.stack([O.potential(occ[I][0][a], U[I][0] - U[I][1]) for a in range(psi.shape[1])]) for I in range(len(st))]
    return p, occ, V, O.apply_gauge(s, st, psi, p, V, A, coef)


def _gpu_handle(s, nb, U, mode=dftu.F64_PAIR):
    h = dftu.handle_for_system(s, nb)
    h.set_f64_mode(mode)
    for I, (u, j) in enumerate(U):
        h.set_u(I, u, j)
    return h


CASES = [("periodic_two_atoms", torch.complex128, dftu.F64_PAIR), ("periodic_two_atoms", torch.complex128, dftu.F64_NATIVE),
         ("periodic_two_atoms", torch.complex64, dftu.F64_PAIR), ("periodic_self_overlap", torch.complex128, dftu.F64_PAIR),
         ("overlapping_three_atoms", torch.complex128, dftu.F64_PAIR), ("overlapping_three_atoms", torch.complex64, dftu.F64_PAIR),
         ("overlapping_three_atoms", torch.complex128, dftu.F64_NATIVE)]


@pytest.mark.parametrize("name,dtype,mode", CASES)
def test_gauge_pass_matches_oracle(name, dtype, mode):
    """p^A, the occupations and psi + c V_U^A psi against the oracle (overlapping spheres and a sphere that
    overlaps its own images exercise the colour-ordered scatter with the per-point phases)."""
    s = SYSTEMS[name]()
    st = O.setup_atoms(s)
    nb = 37                                      # several band chunks and a ragged last one
    psi = C.states_np(s, nb, seed=11)
    f = np.linspace(1.0, 0.1, nb)[None, None, :].repeat(s.nk, 0).repeat(psi.shape[1], 1)
    U = _fixed_u(s)
    coef = 0.7 - 0.4j
    p_ref, occ_ref, _, out_ref = _oracle_gauge_pass(s, st, psi, f, U, A_VEC, coef)
    h = _gpu_handle(s, nb, U, mode)
    dev = torch.device("cuda:0")
    A = torch.tensor(A_VEC, dtype=torch.float64, device=dev)
    h.set_vector_potential(A)
    t = torch.from_numpy(psi).to(dev).to(dtype)
    h.project(t)
    p = split_p(s, h.projections(nb))
    h.occupations(torch.from_numpy(f).to(dev))
    h.acbn0_uj()
    n = h.occupation_matrices()
    h.apply(t, torch.tensor([coef], dtype=torch.complex128, device=dev))
    got = t.to(torch.complex128).cpu().numpy()
    fp64 = dtype == torch.complex128
    for I in range(len(s.atoms)):
        assert rel(p[I], p_ref[I]) < (1e-12 if fp64 else 2e-6), I
        assert np.max(np.abs(n[I] - O.paper_n(occ_ref[I][0]))) < (1e-12 if fp64 else 1e-6), I
    assert rel(got, out_ref) < (1e-12 if fp64 else 1e-6)
    assert h.sync_status() == 0
    h.close()


def test_zero_vector_potential_is_the_plain_operator():
    """A = 0 gives the plain projections to within the pair arithmetic's error (the gauge path's accumulator
    offset is one power of two larger, so the roundings differ), and clearing A restores the plain path bit
    for bit."""
    s = C.periodic_two_atoms()
    nb = 9
    psi = C.states_np(s, nb, seed=4)
    f = np.full((s.nk, 2, nb), 0.8)
    U = _fixed_u(s)
    dev = torch.device("cuda:0")
    h = _gpu_handle(s, nb, U)
    t0 = torch.from_numpy(psi).to(dev)
    h.project(t0)
    p0 = h.projections(nb)
    h.set_vector_potential(torch.zeros(3, dtype=torch.float64, device=dev))
    h.project(t0)
    pz = h.projections(nb)
    assert rel(pz, p0) < 1e-12
    h.set_vector_potential(torch.tensor(A_VEC, dtype=torch.float64, device=dev))
    h.project(t0)
    assert rel(h.projections(nb), p0) > 1e-3
    h.set_vector_potential(None)
    h.project(t0)
    assert np.array_equal(h.projections(nb), p0)
    h.close()


def test_gauge_taylor_step_matches_oracle():
    """One real-time step with V_U^A (Eq. 15 with Eq. 16), against the Taylor series built from the oracle's
    gauge projection and scatter."""
    s = C.periodic_two_atoms()
    st = O.setup_atoms(s)
    nb, dt, order = 6, 0.4, 4
    psi = C.states_np(s, nb, seed=6)
    f = np.linspace(1.0, 0.4, nb)[None, None, :].repeat(s.nk, 0).repeat(2, 1)
    U = _fixed_u(s)
    _, _, V, _ = _oracle_gauge_pass(s, st, psi, f, U, A_VEC)
    out, term = psi.copy(), psi
    for j in range(1, order + 1):
        pj = O.project_gauge(s, st, term, A_VEC)
        term = (-1j * dt / j) * O.apply_gauge(s, st, np.zeros_like(term), pj, V, A_VEC)
        out = out + term
    dev = torch.device("cuda:0")
    h = _gpu_handle(s, nb, U)
    h.set_vector_potential(torch.tensor(A_VEC, dtype=torch.float64, device=dev))
    t = torch.from_numpy(psi).to(dev)
    w = torch.zeros_like(t)
    h.taylor_step(t, w, torch.from_numpy(f).to(dev), dt, order)
    assert rel(t.cpu().numpy(), out) < 1e-12
    h.close()


@pytest.mark.parametrize("name", ["periodic_self_overlap", "overlapping_three_atoms"])
def test_gauge_taylor_steps_with_overlapping_spheres_match_oracle(name):
    """Three real-time steps with V_U^A where spheres overlap each other or their own images: the step's
    overlap blocks between different atoms and images carry the phases exp(+i A.(d_a - d_b)) and
    exp(+i k.(T_a - T_b) L); against the term-by-term Taylor series of the oracle's gauge operator."""
    s = SYSTEMS[name]()
    st = O.setup_atoms(s)
    nb, dt, order = 5, 0.35, 4
    psi = C.states_np(s, nb, seed=8)
    ns = psi.shape[1]
    f = np.linspace(1.0, 0.3, nb)[None, None, :].repeat(s.nk, 0).repeat(ns, 1)
    U = _fixed_u(s)
    dev = torch.device("cuda:0")
    h = _gpu_handle(s, nb, U)
    h.set_vector_potential(torch.tensor(A_VEC, dtype=torch.float64, device=dev))
    t = torch.from_numpy(psi).to(dev)
    fd = torch.from_numpy(f).to(dev)
    ref = psi.copy()
    for step in range(3):
        _, _, V, _ = _oracle_gauge_pass(s, st, ref, f, U, A_VEC)
        out, term = ref.copy(), ref
        for j in range(1, order + 1):
            pj = O.project_gauge(s, st, term, A_VEC)
            term = (-1j * dt / j) * O.apply_gauge(s, st, np.zeros_like(term), pj, V, A_VEC)
            out = out + term
        ref = out
        h.taylor_step(t, None, fd, dt, order)
        assert rel(t.cpu().numpy(), ref) < 1e-12, step
    h.close()


def test_vector_potential_in_cuda_graph_follows_device_A():
    """A graph that captures dftu_set_vector_potential + dftu_taylor_step reads A from device memory at each
    replay: replays after A changes equal eager steps with the new A."""
    s = C.periodic_two_atoms()
    nb = 5
    psi = C.states_np(s, nb, seed=9)
    f = np.full((s.nk, 2, nb), 0.9)
    U = _fixed_u(s)
    dev = torch.device("cuda:0")
    fd = torch.from_numpy(f).to(dev)
    As = [A_VEC, 0.5 * A_VEC[::-1].copy(), -A_VEC]
    h1 = _gpu_handle(s, nb, U)
    a = torch.from_numpy(psi).to(dev)
    wa = torch.zeros_like(a)
    for Av in As:
        h1.set_vector_potential(torch.tensor(Av, dtype=torch.float64, device=dev))
        h1.taylor_step(a, wa, fd, 0.3)
    torch.cuda.synchronize()
    h2 = _gpu_handle(s, nb, U)
    Adev = torch.tensor(As[0], dtype=torch.float64, device=dev)
    b = torch.from_numpy(psi).to(dev)
    wb = torch.zeros_like(b)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        h2.set_vector_potential(Adev)
        h2.taylor_step(b, wb, fd, 0.3)                     # step 1, outside the capture
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        h2.set_vector_potential(Adev)
        h2.taylor_step(b, wb, fd, 0.3)
    for Av in As[1:]:
        Adev.copy_(torch.tensor(Av, dtype=torch.float64, device=dev))
        g.replay()
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    h1.close()
    h2.close()


@pytest.mark.parametrize("dtype,mode", [(torch.complex128, dftu.F64_PAIR), (torch.complex128, dftu.F64_NATIVE),
                                        (torch.complex64, dftu.F64_PAIR)])
@pytest.mark.parametrize("with_A", [False, True])
def test_hubbard_current_matches_oracle(dtype, mode, with_A):
    """Eq. (17) current (velocity operator -i[r, .]) from projections onto the displaced orbitals."""
    s = C.periodic_two_atoms()
    st = O.setup_atoms(s)
    nb = 7
    psi = C.states_np(s, nb, seed=8)
    f = np.linspace(0.3, 1.0, nb)[None, None, :].repeat(s.nk, 0).repeat(2, 1)
    U = _fixed_u(s)
    Av = A_VEC if with_A else np.zeros(3)
    _, _, V, _ = _oracle_gauge_pass(s, st, psi, f, U, Av)
    Jref = O.hubbard_current(s, st, psi, f, V, Av)
    Jat_ref = np.stack([O.hubbard_current(s, [st[I]], psi, f, [V[I]], Av) for I in range(len(st))])
    dev = torch.device("cuda:0")
    h = _gpu_handle(s, nb, U, mode)
    if with_A:
        h.set_vector_potential(torch.tensor(Av, dtype=torch.float64, device=dev))
    t = torch.from_numpy(psi).to(dev).to(dtype)
    fd = torch.from_numpy(f).to(dev)
    h.project(t)
    h.occupations(fd)
    h.acbn0_uj()
    J, Jat = h.hubbard_current(t, fd, per_atom=True)
    tol = 1e-12 if dtype == torch.complex128 else 2e-6
    assert np.max(np.abs(J - Jref)) < tol * np.max(np.abs(Jref))
    assert np.max(np.abs(Jat - Jat_ref)) < tol * np.max(np.abs(Jat_ref))
    assert np.max(np.abs(Jref)) > 1e-6
    h.close()


def test_gauge_argument_errors():
    """Forces are refused while A is set; a non-collinear handle refuses A and the current; stale results
    after a new A are refused."""
    s = C.periodic_two_atoms()
    nb = 3
    psi = C.states_np(s, nb, seed=1)
    f = np.full((s.nk, 2, nb), 1.0)
    dev = torch.device("cuda:0")
    h = _gpu_handle(s, nb, _fixed_u(s))
    t = torch.from_numpy(psi).to(dev)
    fd = torch.from_numpy(f).to(dev)
    A = torch.tensor(A_VEC, dtype=torch.float64, device=dev)
    h.set_vector_potential(A)
    h.project(t)
    h.occupations(fd)
    h.acbn0_uj()
    with pytest.raises(dftu.DftuError) as e:
        h.forces([t, t, t], fd)
    assert e.value.status == dftu.DFTU_ERR_INVALID_ARG
    h.set_vector_potential(A)                                # marks the projections stale
    with pytest.raises(dftu.DftuError) as e:
        h.hubbard_current(t, fd)
    assert e.value.status == dftu.DFTU_ERR_NOT_READY
    h.project(t); h.occupations(fd); h.acbn0_uj()
    h.set_vector_potential(None)                             # clearing A makes them stale too
    with pytest.raises(dftu.DftuError) as e:
        h.apply(t)
    assert e.value.status == dftu.DFTU_ERR_NOT_READY
    with pytest.raises(ValueError):
        h.set_vector_potential(torch.zeros(3, dtype=torch.float32, device=dev))
    h.close()
    snc = synth.noncollinear_system(n=24, natoms=2)
    hn = dftu.handle_for_system(snc, 2)
    with pytest.raises(dftu.DftuError) as e:
        hn.set_vector_potential(A)
    assert e.value.status == dftu.DFTU_ERR_INVALID_ARG
    hn.close()
