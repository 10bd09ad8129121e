"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU needed).

Each test checks the oracle against something other than itself: brute force, closed forms,
invariants, special cases that reduce to a textbook or library routine.
"""
import math

import numpy as np
import pytest
import scipy.integrate
import scipy.linalg
from sympy.physics.wigner import wigner_3j

from oracle import dftu_oracle as O
from paper_1711_08935_gb300 import synth
from tests import _cases as C


# --------------------------------------------------------------------------- sphere maps, orbitals

def test_sphere_point_count_tiny():
    """R = 4, h = 0.3, atom on a grid point: lattice points in the ball (Sec. II, Fig. 2 bottom
    panel counts these).  Brute-force count over the integer cube, and ~ 4 pi R^3 / 3 h^3."""
    s = synth.tiny_system()
    sm = O.sphere_map(s.grid, s.atoms[0])
    r = np.arange(-14, 15)
    I, J, K = np.meshgrid(r, r, r, indexing="ij")
    brute = int(np.sum((I * I + J * J + K * K) * 0.09 <= 16.0 + 1e-9))
    assert len(sm["idx"]) == brute == 9843
    assert abs(len(sm["idx"]) / (4 * math.pi * 4.0 ** 3 / 3 / 0.3 ** 3) - 1) < 0.01


def test_sphere_map_canonical_order_and_folding():
    s = C.periodic_tiny()
    sm = O.sphere_map(s.grid, s.atoms[0])
    u = sm["u"]
    key = (u[:, 2] * 10 ** 6 + u[:, 1]) * 10 ** 6 + u[:, 0] + 10 ** 12 * 0
    assert np.all(np.diff(key) > 0)                                    # strictly ascending z, y, x
    n = np.array(s.grid.n)
    w = u - sm["T"] * n[None, :]
    assert np.all((w >= 0) & (w < n[None, :]))
    assert np.array_equal(sm["idx"], w[:, 0] + n[0] * (w[:, 1] + n[1] * w[:, 2]))
    assert len(np.unique(sm["idx"])) < len(sm["idx"])                  # R > L/2: self-image overlap
    assert len({tuple(t) for t in sm["T"]}) == 8                        # 2R > L: two cells per axis


def test_sphere_boundary_is_inclusive():
    """Points exactly on the sphere belong to it (the inclusive reading of Sec. II).  With h = 0.5,
    R = 2.5 and the atom on a grid point, every squared distance is exact in binary: the sphere holds
    the integer points with i^2 + j^2 + k^2 <= 25, 30 of them on the boundary (the permutations and
    signs of (5, 0, 0) and (3, 4, 0))."""
    g = synth.Grid((16, 16, 16), (0.5, 0.5, 0.5), periodic=False)
    sm = O.sphere_map(g, synth.Atom((4.0, 4.0, 4.0), 0, 2, 2.5))
    r = np.arange(-5, 6)
    I, J, K = np.meshgrid(r, r, r, indexing="ij")
    q = I * I + J * J + K * K
    assert int(np.sum(q == 25)) == 30
    assert len(sm["idx"]) == int(np.sum(q <= 25)) == 515
    assert int(np.sum(sm["r"] == 2.5)) == 30


def degenerate_shell_systems():
    """Two atoms whose orbitals are linearly dependent on their sphere, and a healthy neighbour case.
    On an h = 0.5 grid a sphere of radius 0.6 around a grid point holds the point and its six axis
    neighbours: xy, yz and xz vanish on all seven (and the 3d radial vanishes at the centre), so three
    of the five d orbitals are zero there.  A radial table of zeros gives S = 0.  The p shell on the
    same seven points has three independent orbitals (x, y, z along the axes)."""
    g = synth.Grid((8, 8, 8), (0.5, 0.5, 0.5), periodic=False)
    one = lambda at, rad: synth.System(g, [at], [rad], np.zeros((1, 3)), np.ones(1), nspin=1)
    d7 = one(synth.Atom((2.0, 2.0, 2.0), 0, 2, 0.6), synth.hydrogenic_radial(3, 2, 4.0))
    zero = one(synth.Atom((2.0, 2.0, 2.0), 0, 1, 1.6), synth.Radial(0.01, np.zeros(600)))
    p7 = one(synth.Atom((2.0, 2.0, 2.0), 0, 1, 0.6), synth.hydrogenic_radial(2, 1, 2.5))
    return d7, zero, p7


def test_lowdin_refuses_linearly_dependent_orbitals():
    """S^{-1/2} (Sec. III's orthonormal basis) does not exist for dependent orbitals: refused."""
    d7, zero, p7 = degenerate_shell_systems()
    assert len(O.sphere_map(d7.grid, d7.atoms[0])["idx"]) == 7
    for s in (d7, zero):
        with pytest.raises(ValueError):
            O.setup_atoms(s)
    st = O.setup_atoms(p7)[0]
    assert len(st["idx"]) == 7
    assert np.allclose(p7.grid.dV * st["phi"].T @ st["phi"], np.eye(3), atol=1e-13)


def test_radial_interpolation_exact_on_cubics_and_converges():
    dr = 0.05
    r = np.arange(200) * dr
    poly = lambda x: 0.3 - 1.2 * x + 0.7 * x ** 2 - 0.05 * x ** 3
    q = np.random.default_rng(1).uniform(0, r[-2], 500)
    assert np.max(np.abs(O.radial_value(dr, poly(r), q) - poly(q))) < 1e-12
    assert np.all(O.radial_value(dr, poly(r), np.array([r[-1], r[-1] + 1.0])) == 0.0)
    rad = synth.hydrogenic_radial(3, 2, 4.0, dr=0.002)
    x = np.linspace(0.01, 6.0, 300)
    exact = synth.hydrogenic_radial(3, 2, 4.0, dr=1e-6, rmax=6.5)
    ref = (8.0 / 3.0) ** 1.5 * math.sqrt(1 / (6 * 120)) * np.exp(-4 * x / 3) * (8 * x / 3) ** 2
    assert np.max(np.abs(O.radial_value(rad.dr, rad.R, x) - ref)) < 1e-9
    del exact


@pytest.mark.parametrize("l", [0, 1, 2, 3])
def test_real_ylm_orthonormal_on_sphere(l):
    """Gauss-Legendre (cos theta) x uniform (phi) quadrature, exact for these polynomials."""
    xg, wg = np.polynomial.legendre.leggauss(16)
    nphi = 32
    ph = np.arange(nphi) * 2 * math.pi / nphi
    CT, PH = np.meshgrid(xg, ph, indexing="ij")
    W = np.outer(wg, np.full(nphi, 2 * math.pi / nphi)).reshape(-1)
    st = np.sqrt(1 - CT ** 2)
    d = np.stack([(st * np.cos(PH)).reshape(-1), (st * np.sin(PH)).reshape(-1), CT.reshape(-1)], 1)
    Y = O.real_ylm(l, 2.5 * d, np.full(len(d), 2.5))
    G = (Y * W[:, None]).T @ Y
    assert np.allclose(G, np.eye(2 * l + 1), atol=1e-12)


def test_lowdin_orthonormal_and_symmetric():
    s = synth.tiny_system()
    sm = O.sphere_map(s.grid, s.atoms[0])
    raw = O.raw_orbitals(s.atoms[0], s.radials[0], sm)
    phi = O.lowdin(raw, s.grid.dV)
    assert np.allclose(s.grid.dV * phi.T @ phi, np.eye(5), atol=1e-13)
    T = np.linalg.lstsq(raw, phi, rcond=None)[0]                       # phi = raw T, T symmetric
    assert np.allclose(T, T.T, atol=1e-10)
    off = T - np.diag(np.diag(T))
    assert np.max(np.abs(off)) < 1e-10                    # atom on a grid point: cubic symmetry keeps S diagonal
    assert np.all(np.abs(np.diag(T) - 1) < 0.1)           # only the truncation loss is renormalised


# --------------------------------------------------------------------------- projections

@pytest.mark.parametrize("case", ["self_overlap", "isolated"])
def test_projection_matches_brute_force(case):
    """Maps + phases + orbitals against a loop over every cell point and lattice image."""
    if case == "self_overlap":
        s = C.periodic_tiny()
    else:
        s = synth.System(synth.Grid((14, 13, 12), (0.4, 0.45, 0.5), (0.1, -0.2, 0.0), periodic=False),
                         [synth.Atom((2.3, 2.9, 3.1), 0, 1, 2.4)], [synth.hydrogenic_radial(2, 1, 2.5)],
                         np.zeros((1, 3)), np.ones(1), nspin=1)
    psi = C.states_np(s, 6, seed=11)
    st = O.setup_atoms(s)
    p = O.project(s, st, psi)[0][0, 0]
    bf = O.brute_force_project(s, s.atoms[0], s.radials[0], psi[0, 0], s.kpts[0])
    assert np.max(np.abs(p - bf)) < 1e-12 * max(1.0, np.max(np.abs(bf)))


def test_states_equal_orbitals_give_identity():
    """Eq. (4) with psi_m = phi_m (orthonormal, f = 1): n = identity."""
    s = synth.tiny_system()
    st = O.setup_atoms(s)
    g = O.bloch_orbitals_on_grid(s, st, s.kpts[0])[0]
    psi = g[None, None]                                                # [k][s][5][npts]
    p = O.project(s, st, psi)
    rho, Pb = O.occupations(s, p, np.ones((1, 1, 5)))[0]
    assert np.allclose(rho[0], np.eye(5), atol=1e-13)
    assert np.allclose(Pb[0], np.eye(5), atol=1e-13)                   # Nbar = 1 for these states


def tiny_config_states(s, st):
    """The tiny workload: the five orbitals first, then 16 seeded random states, Gram-Schmidt."""
    g = O.bloch_orbitals_on_grid(s, st, s.kpts[0])[0]
    rnd = C.states_np(s, 16, seed=0)[0, 0]
    return C.gram_schmidt_after(g, rnd, s.grid.dV)[None, None]


def test_tiny_workload_diagonal_occupations():
    """Orbitals first then Gram-Schmidt: n = diag(f_0..f_4), Pbar = n, Nbar in {0, 1}."""
    s = synth.tiny_system()
    st = O.setup_atoms(s)
    psi = tiny_config_states(s, st)
    f = synth.fermi_occupations(1, 1, 21)
    p = O.project(s, st, psi)
    nb = O.nbar(s, p)[0][0, 0]
    assert np.allclose(nb[:5], 1.0, atol=1e-12) and np.allclose(nb[5:], 0.0, atol=1e-12)
    rho, Pb = O.occupations(s, p, f)[0]
    assert np.allclose(rho[0], np.diag(f[0, 0, :5]), atol=1e-12)
    assert np.allclose(Pb[0], rho[0], atol=1e-12)


def test_occupations_hermitian_bounded_and_nbar_bounds():
    """Orthonormal states and orbitals: n Hermitian with eigenvalues in [0, max f]; 0 <= Nbar <= 1
    (the bound stated in Sec. III)."""
    s = C.periodic_two_atoms()
    st = O.setup_atoms(s)
    psi = C.states_np(s, 24, seed=5)
    f = synth.fermi_occupations(s.nk, 2, 24, kT=0.05, e0=-0.3, de=0.03)
    p = O.project(s, st, psi)
    for sp in O.nbar(s, p):
        assert np.all(sp >= -1e-14) and np.all(sp <= 1 + 1e-12)
    for rho, Pb in O.occupations(s, p, f):
        for a in range(2):
            assert np.allclose(rho[a], rho[a].conj().T, atol=1e-14)
            ev = np.linalg.eigvalsh(rho[a])
            assert ev.min() > -1e-13 and ev.max() < 1 + 1e-12


def _scaled_orbital_states(s, st, a, b=None):
    """psi_n = a_n phi_{0,n,k} (the Bloch orbitals of atom 0 on the cell); with b, spinors
    (a_n phi_{0,n,k}, b_n phi_{0,n,k}).  Returns psi in the system's layout."""
    M = len(a)
    out = np.zeros((s.nk, 2, M, s.grid.npts) if b is None else (s.nk, M, 2, s.grid.npts), dtype=np.complex128)
    for ik in range(s.nk):
        g = O.bloch_orbitals_on_grid(s, st, s.kpts[ik])[0]
        if b is None:
            out[ik, :] = (np.asarray(a)[:, None] * g)[None]
        else:
            out[ik, :, 0] = np.asarray(a)[:, None] * g
            out[ik, :, 1] = np.asarray(b)[:, None] * g
    return out


def test_nbar_closed_form_for_scaled_orbital_states():
    """Eq. (9): Nbar_{nk} sums |p|^2 over the atoms of one species and over m.  The d atom (species 0)
    and the p atom (species 1) have disjoint spheres that do not reach their own images, so the
    states psi_n = a_n phi_{0,n,k} project as p_{0,m,n} = a_n delta_mn and not at all onto the p atom:
    Nbar^0_n = a_n^2 and Nbar^1_n = 0 at every k and spin."""
    s = C.periodic_two_atoms()
    st = O.setup_atoms(s)
    a = np.array([0.9, 0.3, 0.6, 0.8, 0.45])
    p = O.project(s, st, _scaled_orbital_states(s, st, a))
    assert np.allclose(p[0], np.diag(a)[None, None], atol=1e-13)
    nb = O.nbar(s, p)
    assert np.allclose(nb[0], (a * a)[None, None], atol=1e-13)
    assert np.allclose(nb[1], 0.0, atol=1e-13)


def test_nbar_closed_form_for_scaled_orbital_spinors():
    """Eq. (B4): for spinors Nbar also sums over both components, so (a_n phi_n, b_n phi_n) gives
    Nbar^0_n = a_n^2 + b_n^2 and Nbar^1_n = 0."""
    s = C.periodic_two_atoms(nspin=1)
    s.noncollinear = True
    st = O.setup_atoms(s)
    a = np.array([0.9, 0.3, 0.6, 0.8, 0.45])
    b = np.array([0.1, 0.7, 0.5, 0.2, 0.6])
    p = O.project_nc(s, st, _scaled_orbital_states(s, st, a, b))
    nb = O.nbar(s, p, noncollinear=True)
    assert np.allclose(nb[0], (a * a + b * b)[None], atol=1e-13)
    assert np.allclose(nb[1], 0.0, atol=1e-13)


def test_lattice_translation_leaves_occupations_unchanged():
    """Moving an atom by a lattice vector only relabels images: n is unchanged (Sec. II phase)."""
    s = C.periodic_two_atoms()
    psi = C.states_np(s, 8, seed=7)
    f = np.ones((s.nk, 2, 8))
    st = O.setup_atoms(s)
    r0 = O.occupations(s, O.project(s, st, psi), f)
    L = s.grid.L
    s2 = C.periodic_two_atoms()
    a0 = s2.atoms[0]
    s2.atoms[0] = synth.Atom((a0.pos[0] + L[0], a0.pos[1] - L[1], a0.pos[2] + 2 * L[2]), a0.species, a0.l, a0.radius)
    st2 = O.setup_atoms(s2)
    r1 = O.occupations(s2, O.project(s2, st2, psi), f)
    assert np.allclose(r0[0][0], r1[0][0], atol=1e-12)


# --------------------------------------------------------------------------- energy, potential

def test_dudarev_energy_and_potential_closed_forms_diagonal():
    """Eq. (3) and Eq. (6) for diagonal n: E = U/2 sum_s sum_m (f_m - f_m^2), V = U diag(1/2 - f)."""
    f = np.array([[0.9, 0.1, 0.5, 0.3, 1.0], [0.2, 0.6, 0.0, 0.8, 0.4]])
    rho = np.stack([np.diag(f[0]), np.diag(f[1])]).astype(complex)
    U = 0.17
    assert abs(O.hubbard_energy(rho, U, 2) - U / 2 * np.sum(f - f * f)) < 1e-15
    assert abs(O.hubbard_energy(rho[:1], U, 1) - U * np.sum(f[0] - f[0] ** 2)) < 1e-15
    assert np.allclose(O.potential(rho[0], U), U * np.diag(0.5 - f[0]))


def _energy_of(s, st, psi, f, U):
    p = O.project(s, st, psi)
    occ = O.occupations(s, p, f)
    return sum(O.hubbard_energy(occ[I][0], U[I], s.nspin) for I in range(len(st))), p, occ


def test_potential_is_energy_gradient_with_transposition():
    """Finite-difference check of Eq. (5)-(6): dE_U = 2 Re sum w f <delta|V_U psi>.  It holds with
    V = U(1/2 - n^T) and fails with the printed V = U(1/2 - n) when projections are complex."""
    s = C.periodic_two_atoms()
    st = O.setup_atoms(s)
    psi = C.states_np(s, 6, seed=3)
    rng = np.random.default_rng(4)
    delta = rng.normal(size=psi.shape) + 1j * rng.normal(size=psi.shape)
    f = np.linspace(0.2, 1.0, 6)[None, None, :].repeat(s.nk, 0).repeat(2, 1)
    U = [0.3, 0.2]
    E0, p, occ = _energy_of(s, st, psi, f, U)
    eps = 1e-5
    Ep, _, _ = _energy_of(s, st, psi + eps * delta, f, U)
    Em, _, _ = _energy_of(s, st, psi - eps * delta, f, U)
    fd = (Ep - Em) / (2 * eps)
    wf = np.asarray(s.wk)[:, None, None] * f

    def grad(Vs):
        Hpsi = O.apply(s, st, np.zeros_like(psi), p, Vs)
        return 2 * np.real(np.sum(wf[..., None] * np.conj(delta) * Hpsi) * s.grid.dV)

    V_rho = [np.stack([O.potential(occ[I][0][a], U[I]) for a in range(2)]) for I in range(2)]
    V_n = [np.stack([O.potential(O.paper_n(occ[I][0][a]), U[I]) for a in range(2)]) for I in range(2)]
    g_rho, g_n = grad(V_rho), grad(V_n)
    assert abs(fd - g_rho) < 1e-7 * max(1.0, abs(fd))
    assert abs(fd - g_n) > 1e-4 * abs(fd)


def test_apply_matches_dense_operator():
    """Eq. (6): V_U as a dense matrix dV G V G^H built from the Bloch-summed orbitals on the cell."""
    s = C.periodic_tiny()
    st = O.setup_atoms(s)
    psi = C.states_np(s, 4, seed=9)
    p = O.project(s, st, psi)
    rng = np.random.default_rng(2)
    A = rng.normal(size=(5, 5)) + 1j * rng.normal(size=(5, 5))
    V = [(A + A.conj().T)[None]]
    out = O.apply(s, st, psi, p, V, coef=0.7)
    G = O.bloch_orbitals_on_grid(s, st, s.kpts[0])[0].T             # [npts, M]
    H = s.grid.dV * G @ V[0][0] @ G.conj().T
    ref = psi[0, 0] + 0.7 * (H @ psi[0, 0].T).T
    assert np.max(np.abs(out[0, 0] - ref)) < 1e-12 * np.max(np.abs(ref))


def test_taylor_step_matches_exponential_and_conserves_norm():
    """Sec. V real-time step: the fourth-order Taylor step agrees with expm(-i dt H) to the
    truncation error and conserves the norm for the Hermitian Hubbard operator."""
    s = C.periodic_tiny()
    st = O.setup_atoms(s)
    psi = C.states_np(s, 5, seed=12)
    f = np.ones((1, 1, 5))
    U = [(0.4, 0.05)]
    dt = 0.01
    out, base = O.taylor_step(s, st, psi, f, dt, fixed_u=U)
    G = O.bloch_orbitals_on_grid(s, st, s.kpts[0])[0].T
    H = s.grid.dV * G @ base["V"][0][0] @ G.conj().T
    assert np.allclose(H, H.conj().T, atol=1e-14)
    ref = (scipy.linalg.expm(-1j * dt * H) @ psi[0, 0].T).T
    assert np.max(np.abs(out[0, 0] - ref)) < 1e-13
    n0 = s.grid.dV * np.sum(np.abs(psi) ** 2, axis=-1)
    n1 = s.grid.dV * np.sum(np.abs(out) ** 2, axis=-1)
    assert np.max(np.abs(n1 - n0)) < 1e-12


def test_taylor_step_on_eigenstates_is_the_fourth_order_polynomial():
    """Sec. V step on eigenstates of V_U: with psi_m = phi_m and occupations f_m, n = diag(f) and
    V = U_eff diag(1/2 - f) (Eq. 6), so V_U psi_m = lambda_m psi_m with lambda_m = U_eff (1/2 - f_m),
    and one step multiplies psi_m by sum_{j<=4} (-i lambda_m dt)^j / j! exactly.  With |lambda dt|
    up to 0.3 a propagator of another order or sign misses this by far more than rounding."""
    s = synth.tiny_system()
    st = O.setup_atoms(s)
    psi = O.bloch_orbitals_on_grid(s, st, s.kpts[0])[0][None, None].copy()
    f = np.array([[[1.0, 0.8, 0.5, 0.2, 0.0]]])
    U, J, dt = 0.6, 0.1, 1.2
    out, _ = O.taylor_step(s, st, psi, f, dt, fixed_u=[(U, J)])
    lam = (U - J) * (0.5 - f[0, 0])
    for m in range(5):
        x = -1j * lam[m] * dt
        T4 = sum(x ** j / math.factorial(j) for j in range(5))
        assert np.max(np.abs(out[0, 0, m] - T4 * psi[0, 0, m])) < 1e-13 * np.max(np.abs(psi))


# --------------------------------------------------------------------------- ACBN0 U, J

def _random_coulomb(M, seed):
    """A random tensor with the 8-fold symmetry of real-orbital Coulomb integrals."""
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(M, M, M, M))
    V = A + A.transpose(1, 0, 2, 3)
    V = V + V.transpose(0, 1, 3, 2)
    V = V + V.transpose(2, 3, 0, 1)
    return V


def test_acbn0_closed_form_diagonal_unpolarised():
    """Eqs. (10)-(11) with n = Pbar = diag(f) in both spins (F = sum f, Q = sum f^2):
    U = 4 sum f_m f_m'' (mm|m''m'') / (2(F^2-Q) + 2F^2),  J = sum f_m f_m'' (mm''|m''m) / (F^2-Q)."""
    f = np.array([0.9, 0.4, 0.7, 0.15, 0.55])
    V = _random_coulomb(5, 3)
    rho = np.diag(f)[None].astype(complex)
    U, J, fl = O.acbn0_uj(rho, rho, V, nspin=1)
    F, Q = f.sum(), (f * f).sum()
    Uc = 4 * np.einsum("a,c,aacc->", f, f, V) / (2 * (F * F - Q) + 2 * F * F)
    Jc = np.einsum("a,c,acca->", f, f, V) / (F * F - Q)
    assert not fl and abs(U - Uc) < 1e-13 * abs(Uc) and abs(J - Jc) < 1e-13 * abs(Jc)


def test_acbn0_collinear_spin_sums():
    """Spin-polarised diagonal case written out by hand from Eqs. (10)-(11)."""
    fu, fd = np.array([0.9, 0.2, 0.6]), np.array([0.1, 0.8, 0.3])
    pu, pd = np.array([0.5, 0.1, 0.4]), np.array([0.05, 0.6, 0.2])     # Pbar differs from n
    V = _random_coulomb(3, 8)
    rho = np.stack([np.diag(fu), np.diag(fd)]).astype(complex)
    Pb = np.stack([np.diag(pu), np.diag(pd)]).astype(complex)
    U, J, _ = O.acbn0_uj(rho, Pb, V, nspin=2)
    P = [pu, pd]
    N = [fu, fd]
    numU = sum(np.einsum("a,c,aacc->", P[a], P[b], V) for a in range(2) for b in range(2))
    numJ = sum(np.einsum("a,c,acca->", P[a], P[a], V) for a in range(2))
    same = sum(N[a].sum() ** 2 - (N[a] ** 2).sum() for a in range(2))
    opp = 2 * fu.sum() * fd.sum()
    assert abs(U - numU / (same + opp)) < 1e-13 and abs(J - numJ / same) < 1e-13


def test_acbn0_zero_denominator():
    rho = np.zeros((1, 5, 5), dtype=complex)
    assert O.acbn0_uj(rho, rho, _random_coulomb(5, 1), 1) == (0.0, 0.0, True)


def _spin_pure_spinors(s_col, psi_col):
    """Collinear states [k][2][n][npts] -> spinors [k][2n][2][npts], spin-up states first."""
    nk, _, nb, npts = psi_col.shape
    out = np.zeros((nk, 2 * nb, 2, npts), dtype=complex)
    out[:, :nb, 0] = psi_col[:, 0]
    out[:, nb:, 1] = psi_col[:, 1]
    return out


def test_noncollinear_reduces_to_collinear_for_spin_pure_spinors():
    """App. A/B: spin-pure spinors give block-diagonal n, and the same Ubar, Jbar and E_U."""
    s = C.periodic_two_atoms()
    st = O.setup_atoms(s)
    psi = C.states_np(s, 7, seed=21)
    f = np.random.default_rng(3).uniform(0, 1, (s.nk, 2, 7))
    Vc = [_random_coulomb(5, 1) + 40, _random_coulomb(3, 2) + 40]
    col = O.hubbard_pass(s, st, psi, f, coulomb=Vc)
    snc = C.periodic_two_atoms(nspin=1)
    snc.noncollinear = True
    psi_nc = _spin_pure_spinors(s, psi)
    f_nc = np.concatenate([f[:, 0], f[:, 1]], axis=1)
    nc = O.hubbard_pass(snc, st, psi_nc, f_nc, coulomb=Vc)
    for I in range(2):
        M = st[I]["phi"].shape[1]
        rho_nc = nc["occ"][I][0]
        assert np.allclose(rho_nc[:M, :M], col["occ"][I][0][0], atol=1e-14)
        assert np.allclose(rho_nc[M:, M:], col["occ"][I][0][1], atol=1e-14)
        assert np.allclose(rho_nc[:M, M:], 0, atol=1e-14)
    assert np.allclose(nc["U"], col["U"], rtol=1e-12) and np.allclose(nc["J"], col["J"], rtol=1e-12)
    assert abs(nc["E"] - col["E"]) < 1e-13 * max(1.0, abs(col["E"]))
    out_nc = nc["psi_out"]
    assert np.allclose(out_nc[:, :7, 0], col["psi_out"][:, 0], atol=1e-13)
    assert np.allclose(out_nc[:, 7:, 1], col["psi_out"][:, 1], atol=1e-13)


def test_noncollinear_energy_is_spin_rotation_invariant():
    """Eq. (A5) and Eqs. (B5)-(B6) involve full spin traces: a global SU(2) rotation of the
    spinors leaves E_U, Ubar and Jbar unchanged."""
    s = C.periodic_two_atoms(nspin=1)
    s.noncollinear = True
    st = O.setup_atoms(s)
    psi = synth.make_states(s, 6, seed=31, device="cpu").numpy()
    f = np.random.default_rng(1).uniform(0, 1, (s.nk, 6))
    Vc = [_random_coulomb(5, 1) + 40, _random_coulomb(3, 2) + 40]
    a = nc1 = O.hubbard_pass(s, st, psi, f, coulomb=Vc)
    th, ph = 0.7, 1.9
    Ur = np.array([[math.cos(th / 2), -np.exp(-1j * ph) * math.sin(th / 2)],
                   [np.exp(1j * ph) * math.sin(th / 2), math.cos(th / 2)]])
    psi_r = np.einsum("ab,knbp->knap", Ur, psi)
    b = O.hubbard_pass(s, st, psi_r, f, coulomb=Vc)
    assert np.allclose(a["U"], b["U"], rtol=1e-12) and np.allclose(a["J"], b["J"], rtol=1e-12)
    assert abs(a["E"] - b["E"]) < 1e-12
    del nc1


# --------------------------------------------------------------------------- Coulomb integrals

def test_poisson_gaussian_self_energy():
    """Isolated Gaussian charge rho = (a/pi)^{3/2} exp(-a r^2): int int rho rho / r = sqrt(2a/pi)."""
    g = synth.Grid((1, 1, 1), (0.2, 0.2, 0.2))
    Rsup = 3.0
    nb, Rc = O.poisson_box(g, Rsup)
    a = 2.0
    x = (np.arange(nb[0]) - nb[0] // 2) * 0.2
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    r2 = X ** 2 + Y ** 2 + Z ** 2
    rho = (a / math.pi) ** 1.5 * np.exp(-a * r2) * (r2 <= Rsup ** 2)
    K = O.truncated_coulomb_kernel(nb, g.h, Rc)
    v = O.hartree_potential(rho, K)
    E = g.dV * np.sum(rho * v)
    assert abs(E - math.sqrt(2 * a / math.pi)) < 1e-6


def _slater_Fk(radial, Rcut, k):
    """F^k = int int R^2(r1) R^2(r2) r_<^k / r_>^{k+1} r1^2 r2^2, radial truncated at Rcut and
    renormalised (1-D quadrature, independent of the grid)."""
    r = np.linspace(1e-6, Rcut, 6001)
    Rv = np.interp(r, np.arange(len(radial.R)) * radial.dr, radial.R)
    w = Rv ** 2 * r ** 2
    w /= scipy.integrate.simpson(w, x=r)
    inner_lt = scipy.integrate.cumulative_simpson(w * r ** k, x=r, initial=0.0)
    g = w / r ** (k + 1)
    tail = scipy.integrate.simpson(g, x=r) - scipy.integrate.cumulative_simpson(g, x=r, initial=0.0)
    f = w * (inner_lt / r ** (k + 1) + r ** k * tail)
    return scipy.integrate.simpson(f, x=r)


@pytest.mark.parametrize("which", ["d", "p"])
def test_coulomb_integrals_against_slater_integrals(which):
    """Basis-independent contractions of (mm'|m''m''') against radial Slater integrals and 3j symbols:
    sum_{mm'} (mm|m'm') = (2l+1)^2 F^0 and sum_{mm'} (mm'|m'm) = (2l+1)^2 sum_k (l k l;0 0 0)^2 F^k."""
    if which == "d":
        rad, l, R, h = synth.hydrogenic_radial(3, 2, 4.0), 2, 4.0, 0.25
    else:
        rad, l, R, h = synth.hydrogenic_radial(2, 1, 4.55), 1, 3.5, 0.2
    g = synth.Grid((64, 64, 64), (h, h, h), periodic=False)
    at = synth.Atom((32 * h + 0.03, 32 * h - 0.05, 32 * h + 0.02), 0, l, R)
    sm = O.sphere_map(g, at)
    sm["phi"] = O.lowdin(O.raw_orbitals(at, rad, sm), g.dV)
    V = O.coulomb_integrals(g, at, sm)
    M = 2 * l + 1
    assert np.allclose(V, V.transpose(1, 0, 2, 3)) and np.allclose(V, V.transpose(2, 3, 0, 1))
    pair = V.transpose(0, 1, 2, 3).reshape(M * M, M * M)
    assert np.linalg.eigvalsh(0.5 * (pair + pair.T)).min() > -1e-10          # positive semidefinite
    F = {k: _slater_Fk(rad, R, k) for k in range(0, 2 * l + 1, 2)}
    direct = np.einsum("aabb->", V)
    exch = np.einsum("abba->", V)
    ref_exch = M * M * sum(float(wigner_3j(l, k, l, 0, 0, 0)) ** 2 * F[k] for k in F)
    assert abs(direct / (M * M * F[0]) - 1) < 1.5e-2
    assert abs(exch / ref_exch - 1) < 1.5e-2


def test_hubbard_forces_match_finite_difference_of_energy():
    """Sec. IV: the force from projections of the state gradients equals minus the derivative of E_U
    with respect to moving the atom, taken here by translating the (analytic) states the opposite way
    with the sphere map held fixed; fixed U, complex Bloch states, two spin channels."""
    s = C.periodic_two_atoms()
    st = O.setup_atoms(s)
    nb = 5
    f = np.linspace(0.3, 1.0, nb)[None, None, :].repeat(s.nk, 0).repeat(2, 1)
    U = [0.4, 0.3]
    psi, dpsi = synth.analytic_states(s, nb, seed=3)
    p = O.project(s, st, psi)
    occ = O.occupations(s, p, f)
    V = [np.stack([O.potential(occ[I][0][a], U[I]) for a in range(2)]) for I in range(2)]
    F = O.hubbard_forces(s, st, psi, dpsi, f, V)

    def energy_atom(I, shift):
        ps, _ = synth.analytic_states(s, nb, seed=3, shift=shift)
        oc = O.occupations(s, O.project(s, st, ps), f)
        return O.hubbard_energy(oc[I][0], U[I], 2)

    eps = 1e-4
    for I in range(2):
        for i in range(3):
            sp = [0.0, 0.0, 0.0]
            sp[i] = eps
            sm = [0.0, 0.0, 0.0]
            sm[i] = -eps
            dE = (energy_atom(I, sp) - energy_atom(I, sm)) / (2 * eps)   # psi(r + s) = atom moved by +s
            assert abs(F[I, i] + dE) < 1e-7 * max(1.0, abs(dE)), (I, i, F[I, i], -dE)
    assert np.max(np.abs(F)) > 1e-4


def test_gauge_operator_equals_literal_definition_on_isolated_box():
    """Eq. (16) read literally on an isolated box, exp(-i A.r) V_U exp(+i A.r) with r the grid position,
    equals the atom-relative form the oracle uses (the exp(+-i A.R_I) factors cancel)."""
    g = synth.Grid((18, 16, 17), (0.4, 0.4, 0.4), (0.2, -0.1, 0.3), periodic=False)
    s = synth.System(g, [synth.Atom((3.1, 2.9, 3.4), 0, 2, 2.6), synth.Atom((4.3, 3.5, 3.0), 1, 1, 2.4)],
                     [synth.hydrogenic_radial(3, 2, 3.0), synth.hydrogenic_radial(2, 1, 3.5)],
                     np.zeros((1, 3)), np.ones(1), nspin=2)
    st = O.setup_atoms(s)
    psi = C.states_np(s, 4, seed=2)
    f = np.full((1, 2, 4), 0.7)
    A = np.array([0.31, -0.17, 0.22])
    occ = O.occupations(s, O.project_gauge(s, st, psi, A), f)
    V = [np.stack([O.potential(occ[I][0][a], 0.3) for a in range(2)]) for I in range(2)]
    out = O.apply_gauge(s, st, psi, O.project_gauge(s, st, psi, A), V, A)
    xs = [np.arange(g.n[a]) * g.h[a] + g.origin[a] for a in range(3)]
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    r = np.stack([X.reshape(-1), Y.reshape(-1), Z.reshape(-1)], 1)
    U = np.exp(1j * (r @ A))
    lit = psi * 0
    pu = O.project(s, st, psi * U)
    lit = O.apply(s, st, np.zeros_like(psi), pu, V) * np.conj(U)
    assert np.max(np.abs((out - psi) - lit)) < 1e-13 * np.max(np.abs(lit))


def test_hubbard_current_is_energy_derivative_in_A():
    """The Hubbard current (Sec. V, Eq. 17, with the velocity operator's factor i) equals dE_U/dA at
    fixed states, by central differences; periodic complex Bloch states."""
    s = C.periodic_two_atoms()
    st = O.setup_atoms(s)
    psi = C.states_np(s, 5, seed=8)
    f = np.linspace(0.3, 1.0, 5)[None, None, :].repeat(s.nk, 0).repeat(2, 1)
    U = [0.5, 0.35]
    A0 = np.array([0.05, -0.02, 0.03])

    def E(A):
        oc = O.occupations(s, O.project_gauge(s, st, psi, A), f)
        return sum(O.hubbard_energy(oc[I][0], U[I], 2) for I in range(2))

    oc = O.occupations(s, O.project_gauge(s, st, psi, A0), f)
    V = [np.stack([O.potential(oc[I][0][a], U[I]) for a in range(2)]) for I in range(2)]
    J = O.hubbard_current(s, st, psi, f, V, A0)
    eps = 1e-5
    for a in range(3):
        e = np.zeros(3)
        e[a] = eps
        dE = (E(A0 + e) - E(A0 - e)) / (2 * eps)
        assert abs(J[a] - dE) < 1e-8 * max(1.0, abs(dE)), (a, J[a], dE)
    assert np.max(np.abs(J)) > 1e-6


# ---- App. A: fully-localised-limit decomposition, Eq. (A1) minus Eq. (A3)

def _nc_rho_from_paper_n(n4):
    """Stored rho (n^T, combined index s*M + m) from the paper's n[s][s'][m][m']."""
    M = n4.shape[-1]
    n = n4.transpose(0, 2, 1, 3).reshape(2 * M, 2 * M)
    return n.T.copy()


def _spinor(theta, phi):
    return np.array([math.cos(theta / 2), np.exp(1j * phi) * math.sin(theta / 2)])


def test_fll_energy_vanishes_for_integer_occupations():
    """The FLL energy E_ee - E_DC is zero whenever every orbital is either empty or filled with one
    electron of a definite spin (Sec. III / App. A: the functional corrects only fractional occupations):
    collinear subsets, a full shell, and one or two electrons with a spinor of any direction."""
    U, J = 0.31, 0.07
    rng = np.random.default_rng(3)
    M = 5
    for _ in range(6):
        occ = rng.integers(0, 2, size=(2, M)).astype(float)
        rho = np.stack([np.diag(occ[0]), np.diag(occ[1])]).astype(np.complex128)
        e_ee, e_dc = O.fll_energy(rho, U, J, noncollinear=False, nspin=2)
        assert abs(e_ee - e_dc) < 1e-13
    full = np.stack([np.eye(M), np.eye(M)]).astype(np.complex128)
    e_ee, e_dc = O.fll_energy(full, U, J, noncollinear=False, nspin=2)
    assert abs(e_ee - e_dc) < 1e-13 and abs(e_dc) > 1.0
    for theta, phi in [(0.3, 1.1), (1.9, -2.4), (math.pi / 2, 0.0)]:
        chi = _spinor(theta, phi)
        for orbitals in ([2], [0, 3]):                          # one electron; two with the same spinor
            n4 = np.zeros((2, 2, M, M), dtype=np.complex128)
            for m in orbitals:
                n4[:, :, m, m] = np.outer(chi, np.conj(chi))    # n^{ss'}_mm = chi_s conj(chi_s')
            e_ee, e_dc = O.fll_energy(_nc_rho_from_paper_n(n4), U, J, noncollinear=True)
            assert abs(e_ee - e_dc) < 1e-13, (theta, phi, orbitals)
            assert abs(e_ee) > 1e-3 or len(orbitals) == 1


def test_fll_energy_equals_dudarev_for_diagonal_collinear_occupations():
    """For orbital-diagonal collinear n, Eq. (A1) minus Eq. (A3) reduces to the Dudarev energy Eq. (3)
    with U_eff = U - J, for spin-polarised and unpolarised channels."""
    U, J = 0.42, 0.09
    rng = np.random.default_rng(8)
    for nspin in (2, 1):
        for M in (3, 5, 7):
            occ = rng.uniform(0, 1, size=(nspin, M))
            rho = np.stack([np.diag(o) for o in occ]).astype(np.complex128)
            e_ee, e_dc = O.fll_energy(rho, U, J, noncollinear=False, nspin=nspin)
            ref = O.hubbard_energy(rho, U - J, nspin)
            assert abs((e_ee - e_dc) - ref) < 1e-13 * max(1.0, abs(ref)), (nspin, M)
            assert abs(ref) > 1e-3


def test_fll_double_counting_moment_term():
    """E_DC of Eq. (A3) for one orbital with spin density matrix [[a, c], [conj c, b]]: N = a + b and
    m.m = (a - b)^2 + 4|c|^2 (Pauli matrices), and E_DC is unchanged by a global spin rotation."""
    U, J = 0.5, 0.12
    a, b, c = 0.7, 0.2, 0.25 - 0.1j
    M = 3
    n4 = np.zeros((2, 2, M, M), dtype=np.complex128)
    n4[0, 0, 1, 1], n4[1, 1, 1, 1], n4[0, 1, 1, 1], n4[1, 0, 1, 1] = a, b, c, np.conj(c)
    _, e_dc = O.fll_energy(_nc_rho_from_paper_n(n4), U, J, noncollinear=True)
    N, mm = a + b, (a - b) ** 2 + 4 * abs(c) ** 2
    assert abs(e_dc - (0.5 * U * N * (N - 1) - 0.5 * J * N * (0.5 * N - 1) - 0.25 * J * mm)) < 1e-15
    # a general Hermitian n rotated in spin space: E_DC is invariant, E_ee in general is not
    rng = np.random.default_rng(4)
    X = rng.normal(size=(2 * M, 2 * M)) + 1j * rng.normal(size=(2 * M, 2 * M))
    n = 0.1 * (X @ X.conj().T)
    th, ph = 0.8, -1.3
    R2 = np.array([[math.cos(th / 2), -np.exp(-1j * ph) * math.sin(th / 2)],
                   [np.exp(1j * ph) * math.sin(th / 2), math.cos(th / 2)]])
    R = np.kron(R2, np.eye(M))
    n_rot = R @ n @ R.conj().T
    _, d0 = O.fll_energy(n.T.copy(), U, J, noncollinear=True)
    _, d1 = O.fll_energy(n_rot.T.copy(), U, J, noncollinear=True)
    assert abs(d0 - d1) < 1e-12 * abs(d0)
