"""Plain CPU FP64 oracle for the DFT+U (ACBN0) Hubbard projector.

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously-correct statement of what the
GPU library computes.  Only the test-suite, the smoke check and the CPU-baseline leg of the
benchmark may import it; the library itself never does, and this module imports nothing from
the library.  It follows the paper (Tancogne-Dejean, Oliveira, Rubio, "Self-consistent DFT+U
method for real-space time-dependent density functional theory calculations") equation by
equation.  Equation numbers below are those printed in the paper:

  Eq. (3)  Dudarev Hubbard energy E_U                          (Sec. II)
  Eq. (4)  occupation matrices n^{I,sigma}_{mm'}                (Sec. II)
  Eq. (6)  Hubbard potential V_U = sum V_{mm'} |phi_m><phi_m'|  (Sec. II)
  Eq. (8)  renormalised density matrix  Pbar                   (Sec. III)
  Eq. (9)  renormalised occupation      Nbar                   (Sec. III)
  Eq. (10) ACBN0 Ubar,  Eq. (11) ACBN0 Jbar                    (Sec. III)
  Eq. (A1) Hartree-Fock energy of the shell, Eq. (A3) FLL double counting with the m.m term
  Eq. (A2) non-collinear occupations, Eq. (A5) non-collinear E_U        (App. A)
  Eq. (B2) Coulomb integrals, Eqs. (B3)-(B6) non-collinear ACBN0        (App. B)

Readings of points the paper leaves open (each is also recorded in the design notes):
  * Transposition (Eqs. 4-6): with n_{mm'} = sum w f <psi|phi_m><phi_m'|psi>, the gradient
    dE_U/dpsi* equals sum_{mm'} U(delta/2 - n_{m'm}) |phi_m><phi_m'|psi>.  We therefore carry
    rho = n^T (rho_{mm'} = sum w f p_m conj(p_m')) and use V = U_eff (1/2 - rho).  E_U, Ubar and
    Jbar are unchanged by the transpose for real orbitals.
  * Bloch phase (Sec. II, Fig. 1): psi is the full Bloch function on the cell; a sphere point j
    at unfolded position r_u folds to the cell point r_w = r_u - T_j; the gather multiplies by
    exp(+i k.T_j) and the scatter by exp(-i k.T_j).
  * Sphere membership: d^2 = (dx*dx + dy*dy) + dz*dz <= R*R in FP64 round-to-nearest without
    fused multiply-add, dx = (i*h + origin) - X, canonical order z-major then y then x over
    unfolded integer coordinates; isolated boxes drop points outside the box.
  * Per-atom Loewdin orthonormalisation of the truncated orbitals (Sec. III assumes an
    orthogonal basis on each atom).  S^{-1/2} exists only for orbitals that are linearly
    independent on the sphere: an atom whose overlap has lambda_min <= 1e-10 lambda_max (fewer
    useful points than orbitals, a radial function that vanishes there) is refused.
  * Ubar/Jbar numerators use Pbar_{mm'} Pbar_{m''m'''} as in Eq. (7) (the printed m'm'' index
    in Eqs. 10-11 is read as a typo); the denominators use N_m = n_mm literally.
  * Spin-unpolarised runs store one channel whose occupations f are per spin; every spin sum
    counts that channel twice.
  * A denominator below 1e-14 gives U = J = 0 for that atom and raises the zero-denominator flag.
  * Non-collinear orbitals are spin independent; Nbar sums |p|^2 over both spinor components.
  * Eq. (A1) is printed for occupation matrices diagonal in the orbital index; it is evaluated on
    the orbital-diagonal entries n^{ss'}_{mm} as printed, whatever the off-diagonal ones are.
    Eq. (A3) uses N = Tr n and the moment m_i = Tr_s(sigma_i rho_s), rho_s = Tr_l n.  Collinear
    channels are spin-diagonal blocks (an unpolarised channel stands for both spins).
"""
from __future__ import annotations

import math
from typing import Dict, List, Sequence

import numpy as np

ZERO_DENOM = 1e-14
LOWDIN_MIN_RATIO = 1e-10
HARTREE_EV = 27.211386245988


# ------------------------------------------------------------------------------------------------
# Sphere sub-grids (Sec. II, Fig. 1)
# ------------------------------------------------------------------------------------------------

def sphere_map(grid, atom) -> Dict[str, np.ndarray]:
    """Points of the grid (unfolded across periodic images) inside the atom's sphere.

    Returns, in canonical order (z outer, y, x inner, ascending unfolded integer coordinates):
      idx [S]   wrapped linear grid index i + n0*(j + n1*k)
      T   [S,3] periodic image of each point, in cells (unfolded = wrapped + T*L)
      u   [S,3] unfolded integer coordinates
      d   [S,3] displacement from the atom centre (dx, dy, dz), bohr
      r   [S]   |d|
    """
    n, h, o, X, R = grid.n, grid.h, grid.origin, atom.pos, atom.radius
    lo = [math.floor((X[a] - R - o[a]) / h[a]) - 1 for a in range(3)]
    hi = [math.ceil((X[a] + R - o[a]) / h[a]) + 1 for a in range(3)]
    kz, jy, ix = np.meshgrid(np.arange(lo[2], hi[2] + 1), np.arange(lo[1], hi[1] + 1),
                             np.arange(lo[0], hi[0] + 1), indexing="ij")
    ix, jy, kz = ix.reshape(-1), jy.reshape(-1), kz.reshape(-1)
    dx = (ix.astype(np.float64) * h[0] + o[0]) - X[0]
    dy = (jy.astype(np.float64) * h[1] + o[1]) - X[1]
    dz = (kz.astype(np.float64) * h[2] + o[2]) - X[2]
    d2 = (dx * dx + dy * dy) + dz * dz
    keep = d2 <= R * R
    if not grid.periodic:
        keep &= (ix >= 0) & (ix < n[0]) & (jy >= 0) & (jy < n[1]) & (kz >= 0) & (kz < n[2])
    ix, jy, kz, dx, dy, dz, d2 = (a[keep] for a in (ix, jy, kz, dx, dy, dz, d2))
    wx, wy, wz = np.mod(ix, n[0]), np.mod(jy, n[1]), np.mod(kz, n[2])
    T = np.stack([(ix - wx) // n[0], (jy - wy) // n[1], (kz - wz) // n[2]], axis=1)
    idx = wx + n[0] * (wy + n[1] * wz)
    return dict(idx=idx.astype(np.int64), T=T.astype(np.int64), u=np.stack([ix, jy, kz], 1),
                d=np.stack([dx, dy, dz], 1), r=np.sqrt(d2))


# ------------------------------------------------------------------------------------------------
# Localised orbitals: radial x real spherical harmonic, then per-atom Loewdin (Sec. II, Sec. III)
# ------------------------------------------------------------------------------------------------

def radial_value(dr: float, table: np.ndarray, r: np.ndarray) -> np.ndarray:
    """Four-point Lagrange interpolation of a radial table on r_i = i*dr.
    Nodes a..a+3 with a = clamp(floor(r/dr) - 1, 0, nr - 4); zero at and beyond the last node."""
    table = np.asarray(table, dtype=np.float64)
    nr = len(table)
    t = np.asarray(r, dtype=np.float64) / dr
    i = np.floor(t).astype(np.int64)
    a = np.clip(i - 1, 0, nr - 4)
    x = t - a
    w0 = -(x - 1.0) * (x - 2.0) * (x - 3.0) / 6.0
    w1 = x * (x - 2.0) * (x - 3.0) / 2.0
    w2 = -x * (x - 1.0) * (x - 3.0) / 2.0
    w3 = x * (x - 1.0) * (x - 2.0) / 6.0
    val = w0 * table[a] + w1 * table[a + 1] + w2 * table[a + 2] + w3 * table[a + 3]
    return np.where(i < nr - 1, val, 0.0)


def real_ylm(l: int, d: np.ndarray, r: np.ndarray) -> np.ndarray:
    """Real spherical harmonics, m = -l..l, columns in the order
    s: 1 | p: y, z, x | d: xy, yz, 3z^2-r^2, xz, x^2-y^2 |
    f: y(3x^2-y^2), xyz, y(5z^2-r^2), z(5z^2-3r^2), x(5z^2-r^2), z(x^2-y^2), x(x^2-3y^2).
    Zero at r = 0 for l > 0."""
    x, y, z = d[:, 0], d[:, 1], d[:, 2]
    pi = math.pi
    with np.errstate(divide="ignore", invalid="ignore"):
        if l == 0:
            cols = [np.full_like(r, 0.5 / math.sqrt(pi))]
            return np.stack(cols, 1)
        rl = r ** l
        if l == 1:
            c = math.sqrt(3.0 / (4 * pi))
            cols = [c * y, c * z, c * x]
        elif l == 2:
            c1, c2, c3 = math.sqrt(15.0 / (4 * pi)), math.sqrt(5.0 / (16 * pi)), math.sqrt(15.0 / (16 * pi))
            r2 = r * r
            cols = [c1 * x * y, c1 * y * z, c2 * (3 * z * z - r2), c1 * x * z, c3 * (x * x - y * y)]
        elif l == 3:
            r2 = r * r
            cols = [math.sqrt(35.0 / (32 * pi)) * y * (3 * x * x - y * y),
                    math.sqrt(105.0 / (4 * pi)) * x * y * z,
                    math.sqrt(21.0 / (32 * pi)) * y * (5 * z * z - r2),
                    math.sqrt(7.0 / (16 * pi)) * z * (5 * z * z - 3 * r2),
                    math.sqrt(21.0 / (32 * pi)) * x * (5 * z * z - r2),
                    math.sqrt(105.0 / (16 * pi)) * z * (x * x - y * y),
                    math.sqrt(35.0 / (32 * pi)) * x * (x * x - 3 * y * y)]
        else:
            raise ValueError("l must be 0..3")
        Y = np.stack(cols, 1) / rl[:, None]
    Y[r == 0.0, :] = 0.0
    return Y


def radius_from_threshold(dr: float, table: np.ndarray, threshold: float) -> float:
    """Third radius method of Sec. II: the sphere ends where the radial function drops below the
    threshold for good, i.e. at (i + 1) dr for the last node i with |R_i| >= threshold."""
    above = np.nonzero(np.abs(np.asarray(table)) >= threshold)[0]
    return 0.0 if len(above) == 0 else float((above[-1] + 1) * dr)


def radius_from_cell(grid) -> float:
    """Second radius method of Sec. II: the smallest dimension of the cell."""
    return float(min(grid.n[a] * grid.h[a] for a in range(3)))


def raw_orbitals(atom, radial, smap) -> np.ndarray:
    """phi_m(j) = R(|d_j|) Y_lm(d_j) on the sphere points, [S, 2l+1] (pseudo-atomic orbital of Sec. II)."""
    Rv = radial_value(radial.dr, radial.R, smap["r"])
    return Rv[:, None] * real_ylm(atom.l, smap["d"], smap["r"])


def lowdin(phi: np.ndarray, dV: float) -> np.ndarray:
    """Symmetric orthonormalisation phi S^{-1/2}, S_{mm'} = dV sum_j phi_m phi_m' (Sec. III: the
    localised basis on each atom is orthogonal)."""
    S = dV * (phi.T @ phi)
    lam, U = np.linalg.eigh(S)
    if not (np.all(np.isfinite(lam)) and lam[-1] > 0 and lam[0] > LOWDIN_MIN_RATIO * lam[-1]):
        raise ValueError("orbitals are linearly dependent on the sphere: S^{-1/2} does not exist")
    return phi @ (U @ np.diag(lam ** -0.5) @ U.T)


def setup_atoms(system) -> List[Dict[str, np.ndarray]]:
    """Sphere map plus orthonormal orbitals for every atom."""
    out = []
    for at in system.atoms:
        sm = sphere_map(system.grid, at)
        sm["phi"] = lowdin(raw_orbitals(at, system.radials[at.species], sm), system.grid.dV)
        out.append(sm)
    return out


def phases(system, smap, k) -> np.ndarray:
    """exp(+i k.T_j) for every sphere point (Sec. II, phase correction across the cell border)."""
    L = np.array(system.grid.L)
    return np.exp(1j * ((smap["T"] * L[None, :]) @ np.asarray(k)))


def bloch_orbitals_on_grid(system, atoms_setup, k) -> List[np.ndarray]:
    """The cell representation of each Bloch-summed orbital: phi_{I,m,k}(w) =
    sum_{j: idx_j = w} exp(-i k.T_j) phi_{I,m}(j); returns one [M, npts] array per atom."""
    out = []
    for sm in atoms_setup:
        ph = np.conj(phases(system, sm, k))
        g = np.zeros((sm["phi"].shape[1], system.grid.npts), dtype=np.complex128)
        for m in range(sm["phi"].shape[1]):
            np.add.at(g[m], sm["idx"], ph * sm["phi"][:, m])
        out.append(g)
    return out


# ------------------------------------------------------------------------------------------------
# Projections <phi_{I,m,k}|psi_{nk}> (inside Eqs. 4 and 6)
# ------------------------------------------------------------------------------------------------

def project(system, atoms_setup, psi: np.ndarray) -> List[np.ndarray]:
    """Collinear/unpolarised psi[k][s][n][npts] -> per atom p[k][s][n][m]
    p = dV sum_j phi_m(j) exp(+i k.T_j) psi(idx_j)."""
    dV = system.grid.dV
    out = []
    for sm in atoms_setup:
        nk, ns, nb = psi.shape[:3]
        p = np.zeros((nk, ns, nb, sm["phi"].shape[1]), dtype=np.complex128)
        for ik in range(nk):
            ph = phases(system, sm, system.kpts[ik])
            for s in range(ns):
                p[ik, s] = dV * ((psi[ik, s][:, sm["idx"]] * ph[None, :]) @ sm["phi"])
        out.append(p)
    return out


def project_nc(system, atoms_setup, psi: np.ndarray) -> List[np.ndarray]:
    """Non-collinear spinors psi[k][n][c][npts] (c = spinor component) -> p[k][n][c][m] (App. A)."""
    dV = system.grid.dV
    out = []
    for sm in atoms_setup:
        nk, nb = psi.shape[:2]
        p = np.zeros((nk, nb, 2, sm["phi"].shape[1]), dtype=np.complex128)
        for ik in range(nk):
            ph = phases(system, sm, system.kpts[ik])
            for c in range(2):
                p[ik, :, c] = dV * ((psi[ik, :, c][:, sm["idx"]] * ph[None, :]) @ sm["phi"])
        out.append(p)
    return out


def brute_force_project(system, atom, radial, psi_ks: np.ndarray, k, images=2) -> np.ndarray:
    """Independent check of maps, phases and orbitals: loop over every cell point w and every
    lattice image T in [-images, images]^3, keep r_w + T L inside the sphere (same membership
    rule), evaluate the raw orbital there, orthonormalise with the overlap accumulated the same
    brute-force way, and sum dV phi exp(i k.T L) psi(w).  psi_ks: [nbands, npts] for one (k, s)."""
    g = system.grid
    n, h, o = g.n, g.h, g.origin
    X, R = atom.pos, atom.radius
    M = 2 * atom.l + 1
    rng = range(-images, images + 1) if g.periodic else range(0, 1)
    S = np.zeros((M, M))
    acc = np.zeros((psi_ks.shape[0], M), dtype=np.complex128)
    L = np.array(g.L)
    for tz in rng:
        for ty in rng:
            for tx in rng:
                for wz in range(n[2]):
                    for wy in range(n[1]):
                        ix = np.arange(n[0]) + tx * n[0]
                        jy = wy + ty * n[1]
                        kz = wz + tz * n[2]
                        dx = (ix.astype(np.float64) * h[0] + o[0]) - X[0]
                        dy = (float(jy) * h[1] + o[1]) - X[1]
                        dz = (float(kz) * h[2] + o[2]) - X[2]
                        d2 = (dx * dx + dy * dy) + dz * dz
                        sel = np.nonzero(d2 <= R * R)[0]
                        if sel.size == 0:
                            continue
                        d = np.stack([dx[sel], np.full(sel.size, dy), np.full(sel.size, dz)], 1)
                        r = np.sqrt(d2[sel])
                        phi = radial_value(radial.dr, radial.R, r)[:, None] * real_ylm(atom.l, d, r)
                        S += g.dV * phi.T @ phi
                        w = sel + n[0] * (wy + n[1] * wz)
                        ph = np.exp(1j * float(np.dot(np.array([tx, ty, tz]) * L, k)))
                        acc += g.dV * ph * (psi_ks[:, w] @ phi)
    lam, U = np.linalg.eigh(S)
    return acc @ (U @ np.diag(lam ** -0.5) @ U.T)


# ------------------------------------------------------------------------------------------------
# Occupations: Eq. (4); renormalised Eqs. (8)-(9)
# ------------------------------------------------------------------------------------------------

def nbar(system, p_atoms: Sequence[np.ndarray], noncollinear=False) -> List[np.ndarray]:
    """Eq. (9): Nbar for each state, summed over all atoms of the same species (and shell)
    and all m.  Collinear: [nspecies] arrays [k][s][n]; non-collinear (Eq. B4): [k][n], summed
    over both spinor components."""
    nsp = len(system.radials)
    out = []
    for s in range(nsp):
        tot = None
        for I, at in enumerate(system.atoms):
            if at.species != s:
                continue
            ax = (-2, -1) if noncollinear else (-1,)
            term = np.sum(np.abs(p_atoms[I]) ** 2, axis=ax)
            tot = term if tot is None else tot + term
        out.append(tot)
    return out


def occupations(system, p_atoms, f: np.ndarray):
    """Eq. (4) and Eq. (8), collinear/unpolarised.  f[k][s][n].
    Returns per atom (rho [s][M][M], Pbar_rho [s][M][M]) where rho = n^T, i.e.
    rho_{mm'} = sum_{n,k} w_k f p_m conj(p_m'), and Pbar_rho the same with the factor Nbar."""
    nb_s = nbar(system, p_atoms)
    wk = np.asarray(system.wk)
    out = []
    for I, at in enumerate(system.atoms):
        p = p_atoms[I]                                 # [k][s][n][m]
        wf = wk[:, None, None] * f                     # [k][s][n]
        rho = np.einsum("ksn,ksnm,ksnq->smq", wf, p, np.conj(p))
        Pb = np.einsum("ksn,ksnm,ksnq->smq", wf * nb_s[at.species], p, np.conj(p))
        out.append((rho, Pb))
    return out


def occupations_nc(system, p_atoms, f: np.ndarray):
    """Eq. (A2) and Eq. (B3): 2M x 2M spin-block matrices in the combined index c*M + m.
    f[k][n].  Returns per atom (rho, Pbar_rho) with rho = n^T in the combined index."""
    nb_s = nbar(system, p_atoms, noncollinear=True)
    wk = np.asarray(system.wk)
    out = []
    for I, at in enumerate(system.atoms):
        p = p_atoms[I]                                 # [k][n][c][m]
        nk, nb, _, M = p.shape
        q = p.reshape(nk, nb, 2 * M)
        wf = wk[:, None] * f
        rho = np.einsum("kn,kna,knb->ab", wf, q, np.conj(q))
        Pb = np.einsum("kn,kna,knb->ab", wf * nb_s[at.species], q, np.conj(q))
        out.append((rho, Pb))
    return out


def paper_n(rho: np.ndarray) -> np.ndarray:
    """The paper's n_{mm'} (Eq. 4) from the stored rho: n = rho^T over the last two axes."""
    return np.swapaxes(rho, -1, -2)


# ------------------------------------------------------------------------------------------------
# ACBN0 U and J: Eqs. (10)-(11), non-collinear Eqs. (B5)-(B6)
# ------------------------------------------------------------------------------------------------

def acbn0_uj(rho_s: np.ndarray, Pb_rho_s: np.ndarray, V: np.ndarray, nspin: int):
    """Collinear/unpolarised ACBN0 for one atom.  rho_s, Pb_rho_s: [nspin][M][M] (stored, = n^T);
    V: (mm'|m''m''') [M,M,M,M] in Hartree.  Returns (U, J, zero_denominator_flag)."""
    n = paper_n(rho_s)
    P = paper_n(Pb_rho_s)
    if nspin == 1:                                     # one stored channel counted for both spins
        n = np.stack([n[0], n[0]])
        P = np.stack([P[0], P[0]])
    M = n.shape[-1]
    N = np.real(np.einsum("smm->sm", n))               # N_m^alpha = n_mm^alpha
    numU = 0.0
    for a in range(2):
        for b in range(2):
            numU += np.einsum("ab,cd,abcd->", P[a], P[b], V)
    numJ = 0.0
    for a in range(2):
        numJ += np.einsum("ab,cd,adcb->", P[a], P[a], V)
    off = 1.0 - np.eye(M)
    same = sum(np.einsum("m,q,mq->", N[a], N[a], off) for a in range(2))
    opp = sum(np.einsum("m,q->", N[a], N[1 - a]) for a in range(2))
    denU, denJ = same + opp, same
    flag = False
    if abs(denU) < ZERO_DENOM or abs(denJ) < ZERO_DENOM:
        return 0.0, 0.0, True
    return float(np.real(numU) / denU), float(np.real(numJ) / denJ), flag


def acbn0_uj_nc(rho: np.ndarray, Pb_rho: np.ndarray, V: np.ndarray):
    """Non-collinear ACBN0, Eqs. (B5)-(B6), for one atom; rho, Pb_rho: [2M][2M] in the combined
    index (stored, = n^T).  Returns (U, J, zero_denominator_flag)."""
    M = rho.shape[0] // 2
    n = paper_n(rho).reshape(2, M, 2, M).transpose(0, 2, 1, 3)     # n[s][s'][m][m']
    P = paper_n(Pb_rho).reshape(2, M, 2, M).transpose(0, 2, 1, 3)
    Nd = np.einsum("abmm->abm", n)                                  # N^{ab}_m = n^{ab}_mm
    off = 1.0 - np.eye(M)
    numU = sum(np.einsum("ab,cd,abcd->", P[s, s], P[t, t], V) for s in range(2) for t in range(2))
    numJ = sum(np.einsum("ab,cd,adcb->", P[s, t], P[t, s], V) for s in range(2) for t in range(2))
    den_u = 0.0
    den_j = 0.0
    for s in range(2):
        o = 1 - s
        den_u += np.einsum("m,q->", Nd[s, s], Nd[o, o])
        den_u += np.einsum("m,q,mq->", Nd[s, s], Nd[s, s], off)
        den_u -= np.einsum("m,m->", Nd[s, o], Nd[o, s])
        den_j += np.einsum("m,q,mq->", Nd[s, s], Nd[s, s], off)
        den_j += np.einsum("m,q,mq->", Nd[s, o], Nd[o, s], off)
    den_u, den_j = np.real(den_u), np.real(den_j)
    if abs(den_u) < ZERO_DENOM or abs(den_j) < ZERO_DENOM:
        return 0.0, 0.0, True
    return float(np.real(numU) / den_u), float(np.real(numJ) / den_j), False


# ------------------------------------------------------------------------------------------------
# Energy and potential: Eqs. (3), (6), (A5)
# ------------------------------------------------------------------------------------------------

def hubbard_energy_nc(rho: np.ndarray, Ueff: float) -> float:
    """Eq. (A5): (U-J)/2 [sum_{s,m} n^{ss}_mm - sum n^{ss'}_{mm'} n^{s's}_{m'm}], 2M x 2M matrix."""
    n = paper_n(rho)
    return 0.5 * Ueff * float(np.real(np.trace(n) - np.einsum("ab,ba->", n, n)))


# ------------------------------------------------------------------------------------------------
# Fully-localised-limit decomposition (App. A): E_ee of Eq. (A1) and E_DC of Eq. (A3)
# ------------------------------------------------------------------------------------------------

def spin_blocks(rho: np.ndarray, noncollinear: bool, nspin: int) -> np.ndarray:
    """The paper's n as a [2][2][M][M] array n[s][s'][m][m'] = n^{ss'}_{mm'} from the stored rho
    (n^T): non-collinear 2M x 2M in the combined index s*M + m, collinear [ns][M][M]."""
    n = paper_n(rho)
    if noncollinear:
        M = n.shape[-1] // 2
        return n.reshape(2, M, 2, M).transpose(0, 2, 1, 3)
    M = n.shape[-1]
    out = np.zeros((2, 2, M, M), dtype=np.complex128)
    out[0, 0] = n[0]
    out[1, 1] = n[1] if nspin == 2 else n[0]
    return out


def fll_energy(rho: np.ndarray, U: float, J: float, noncollinear: bool, nspin: int = 2):
    """Eq. (A1) and Eq. (A3) for one shell.  Returns (E_ee, E_DC); E_ee - E_DC is the FLL energy.

    E_ee = U/2 sum_s sum_{m,m'} n^{ss}_mm n^{-s-s}_m'm' - U/2 sum_s sum_m n^{s-s}_mm n^{-ss}_mm
           - J/2 sum_s sum_{m != m'} n^{s-s}_mm n^{-ss}_m'm' + (U-J)/2 sum_s sum_{m != m'} n^{ss}_mm n^{ss}_m'm'
    E_DC = U/2 N (N - 1) - J/2 N (N/2 - 1) - J/4 m.m"""
    nb = spin_blocks(rho, noncollinear, nspin)
    d = np.array([[np.diagonal(nb[s, t]) for t in range(2)] for s in range(2)])   # d[s][t][m] = n^{st}_mm
    e_ee = 0.0 + 0.0j
    for s in range(2):
        o = 1 - s
        e_ee += 0.5 * U * np.sum(d[s, s]) * np.sum(d[o, o])
        e_ee -= 0.5 * U * np.sum(d[s, o] * d[o, s])
        e_ee -= 0.5 * J * (np.sum(d[s, o]) * np.sum(d[o, s]) - np.sum(d[s, o] * d[o, s]))
        e_ee += 0.5 * (U - J) * (np.sum(d[s, s]) ** 2 - np.sum(d[s, s] * d[s, s]))
    rho_s = np.array([[np.sum(d[s, t]) for t in range(2)] for s in range(2)])     # Tr_l n, [s][s']
    pauli = [np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]), np.array([[1, 0], [0, -1]])]
    mvec = np.array([np.trace(P @ rho_s) for P in pauli])
    N = np.trace(rho_s)
    e_dc = 0.5 * U * N * (N - 1) - 0.5 * J * N * (0.5 * N - 1) - 0.25 * J * np.sum(mvec * mvec)
    return float(np.real(e_ee)), float(np.real(e_dc))


def potential(rho: np.ndarray, Ueff: float) -> np.ndarray:
    """Eq. (6) with the transposition reading: V = U_eff (1/2 I - rho), rho = n^T."""
    M = rho.shape[-1]
    return Ueff * (0.5 * np.eye(M) - rho)


def apply(system, atoms_setup, psi: np.ndarray, p_atoms, V_atoms, coef=1.0) -> np.ndarray:
    """Eq. (6) applied to every state: psi(idx_j) += coef * exp(-i k.T_j) sum_m phi_m(j) (V p)_m,
    summed over all atoms and sphere points (overlapping points accumulate).
    Collinear psi[k][s][n][npts]; V_atoms[I] is [s][M][M].  Returns a new array."""
    out = psi.copy()
    for I, sm in enumerate(atoms_setup):
        for ik in range(psi.shape[0]):
            ph = np.conj(phases(system, sm, system.kpts[ik]))
            for s in range(psi.shape[1]):
                Vp = p_atoms[I][ik, s] @ V_atoms[I][s].T          # [n][m] = sum_m' V_mm' p_m'
                upd = coef * (Vp @ sm["phi"].T) * ph[None, :]     # [n][S]
                np.add.at(out[ik, s], (slice(None), sm["idx"]), upd)
    return out


def apply_nc(system, atoms_setup, psi: np.ndarray, p_atoms, V_atoms, coef=1.0) -> np.ndarray:
    """Eq. (6) on spinors psi[k][n][c][npts]: V_atoms[I] is [2M][2M] in the combined index."""
    out = psi.copy()
    for I, sm in enumerate(atoms_setup):
        M = sm["phi"].shape[1]
        for ik in range(psi.shape[0]):
            ph = np.conj(phases(system, sm, system.kpts[ik]))
            q = p_atoms[I][ik].reshape(psi.shape[1], 2 * M)
            Vp = (q @ V_atoms[I].T).reshape(psi.shape[1], 2, M)
            for c in range(2):
                upd = coef * (Vp[:, c] @ sm["phi"].T) * ph[None, :]
                np.add.at(out[ik, :, c], (slice(None), sm["idx"]), upd)
    return out


# ------------------------------------------------------------------------------------------------
# Whole pass and the real-time step (Sec. V, Eq. 15: potential rebuilt from the current states)
# ------------------------------------------------------------------------------------------------

def hubbard_pass(system, atoms_setup, psi, f, coulomb=None, fixed_u=None, coef=1.0):
    """project -> occupations -> U/J (ACBN0, or fixed U_eff per atom) -> energy -> apply.
    coulomb: per species [M,M,M,M] Hartree.  Returns a dict of every intermediate."""
    nc = system.noncollinear
    p = project_nc(system, atoms_setup, psi) if nc else project(system, atoms_setup, psi)
    occ = occupations_nc(system, p, f) if nc else occupations(system, p, f)
    U, J, flags, Vs, E = [], [], [], [], 0.0
    for I, at in enumerate(system.atoms):
        rho, Pb = occ[I]
        if fixed_u is not None:
            u, j, fl = fixed_u[I][0], fixed_u[I][1], False
        elif nc:
            u, j, fl = acbn0_uj_nc(rho, Pb, coulomb[at.species])
        else:
            u, j, fl = acbn0_uj(rho, Pb, coulomb[at.species], system.nspin)
        ueff = u - j
        U.append(u); J.append(j); flags.append(fl)
        if nc:
            E += hubbard_energy_nc(rho, ueff)
            Vs.append(potential(rho, ueff))
        else:
            E += hubbard_energy(rho, ueff, system.nspin)
            Vs.append(np.stack([potential(rho[s], ueff) for s in range(rho.shape[0])]))
    psi_out = (apply_nc if nc else apply)(system, atoms_setup, psi, p, Vs, coef)
    return dict(p=p, occ=occ, U=np.array(U), J=np.array(J), flags=flags, V=Vs, E=E, psi_out=psi_out)


def hubbard_energy(rho_s: np.ndarray, Ueff: float, nspin: int) -> float:
    """Eq. (3) for one atom: U_eff/2 sum_sigma (sum_m n_mm - sum_{mm'} n_mm' n_m'm); rho_s is
    [nspin][M][M]; an unpolarised run's single channel counts twice."""
    e = 0.0
    for s in range(rho_s.shape[0]):
        n = paper_n(rho_s[s])
        e += np.real(np.trace(n) - np.einsum("ab,ba->", n, n))
    if nspin == 1:
        e *= 2.0
    return 0.5 * Ueff * float(e)


def taylor_step(system, atoms_setup, psi, f, dt, coulomb=None, fixed_u=None, order=4):
    """One real-time step psi <- sum_{j=0}^{order} (-i dt H)^j / j! psi with H = V_U built from the
    occupations (and ACBN0 U, J) of the incoming psi and held fixed within the step."""
    base = hubbard_pass(system, atoms_setup, psi, f, coulomb, fixed_u, coef=1.0)
    Vs = base["V"]
    nc = system.noncollinear
    proj = project_nc if nc else project
    app = apply_nc if nc else apply
    out = psi.copy()
    term = psi
    for j in range(1, order + 1):
        p = proj(system, atoms_setup, term)
        Hterm = app(system, atoms_setup, np.zeros_like(term), p, Vs, 1.0)
        term = (-1j * dt / j) * Hterm
        out = out + term
    return out, base


# ------------------------------------------------------------------------------------------------
# Gauge-invariant Hubbard operator V_U^A = exp(-i A.r) V_U exp(i A.r) (Sec. V, Eq. 16) and its current
# ------------------------------------------------------------------------------------------------
# Reading: on atom I's sphere r = R_I + d_j; the factor exp(+-i A.R_I) cancels between the gather and
# the scatter of the same projector and in the occupations, so the operator is the plain one with the
# orbitals phi_m(d) exp(-i A.d): the gather multiplies by exp(+i A.d_j), the scatter by exp(-i A.d_j).

def gauge_phases(smap, A) -> np.ndarray:
    """exp(+i A.d_j) for every sphere point (d_j = unfolded position minus the atom centre)."""
    return np.exp(1j * (smap["d"] @ np.asarray(A, dtype=np.float64)))


def project_gauge(system, atoms_setup, psi, A) -> List[np.ndarray]:
    """p^A = <phi_m exp(-i A.d)|psi> = dV sum_j phi_m(j) exp(+i A.d_j) exp(+i k.T_j) psi(idx_j)."""
    dV = system.grid.dV
    out = []
    for sm in atoms_setup:
        nk, ns, nb = psi.shape[:3]
        g = gauge_phases(sm, A)
        p = np.zeros((nk, ns, nb, sm["phi"].shape[1]), dtype=np.complex128)
        for ik in range(nk):
            ph = phases(system, sm, system.kpts[ik]) * g
            for s in range(ns):
                p[ik, s] = dV * ((psi[ik, s][:, sm["idx"]] * ph[None, :]) @ sm["phi"])
        out.append(p)
    return out


def apply_gauge(system, atoms_setup, psi, p_atoms, V_atoms, A, coef=1.0) -> np.ndarray:
    """Eq. (16): psi(idx_j) += coef exp(-i k.T_j) exp(-i A.d_j) sum_m phi_m(j) (V p)_m."""
    out = psi.copy()
    for I, sm in enumerate(atoms_setup):
        g = np.conj(gauge_phases(sm, A))
        for ik in range(psi.shape[0]):
            ph = np.conj(phases(system, sm, system.kpts[ik])) * g
            for s in range(psi.shape[1]):
                Vp = p_atoms[I][ik, s] @ V_atoms[I][s].T
                upd = coef * (Vp @ sm["phi"].T) * ph[None, :]
                np.add.at(out[ik, s], (slice(None), sm["idx"]), upd)
    return out


def hubbard_current(system, atoms_setup, psi, f, V_atoms, A) -> np.ndarray:
    """Hubbard term of the current (Sec. V, Eq. 17), read as J = sum w f <psi| -i [r, V_U^A] |psi>: the
    printed <psi|[r, V]|psi> + c.c. vanishes for a Hermitian V, so the factor i of the velocity operator
    is restored.  With q^{(a)}_m = <phi_m exp(-i A.d)| d_a psi> this is
    J_a = -i sum w f sum_{mm'} V_{mm'} [conj(q_m) p_m' - conj(p_m) q_m'] (real), and equals dE_U/dA at
    fixed states.  Collinear/unpolarised; returns [3]."""
    p = project_gauge(system, atoms_setup, psi, A)
    wf = np.asarray(system.wk)[:, None, None] * f
    mult = 2.0 if system.nspin == 1 else 1.0
    J = np.zeros(3)
    for a in range(3):
        for I, sm in enumerate(atoms_setup):
            sm_d = dict(sm)
            sm_d["phi"] = sm["phi"] * sm["d"][:, a:a + 1]
            q = project_gauge(system, [sm_d], psi, A)[0]
            X = (np.einsum("ksn,ksnm,ksnq,smq->", wf, np.conj(q), p[I], V_atoms[I])
                 - np.einsum("ksn,ksnm,ksnq,smq->", wf, np.conj(p[I]), q, V_atoms[I]))
            J[a] += mult * float(np.real(-1j * X))
    return J


# ------------------------------------------------------------------------------------------------
# Hubbard forces (Sec. IV): F = -dE_U/dR with dn/dR from projections of the state gradients
# ------------------------------------------------------------------------------------------------

def hubbard_forces(system, atoms_setup, psi, dpsi, f, V_atoms):
    """Sec. IV, in the form that differentiates the states instead of the orbitals:
    dn_{ab}/dR_i = sum w f [<d_i psi|phi_a><phi_b|psi> + <psi|phi_a><phi_b|d_i psi>], and
    F_i = -sum_{sigma,a,b} (dE_U/dn_{ab}) dn_{ab}/dR_i with dE_U/dn_{ab} = U_eff/2 (delta_ab - 2 n_ba),
    which is V_ab of Eq. (6) under the transposition reading.  U_eff is held fixed, as in the paper.
    Collinear/unpolarised psi[k][s][n][npts]; dpsi = [d_x psi, d_y psi, d_z psi]; V_atoms[I] is [s][M][M].
    Returns [natoms][3] in Hartree/bohr."""
    p = project(system, atoms_setup, psi)
    pg = [project(system, atoms_setup, d) for d in dpsi]
    wf = np.asarray(system.wk)[:, None, None] * f
    mult = 2.0 if system.nspin == 1 else 1.0
    F = np.zeros((len(atoms_setup), 3))
    for I in range(len(atoms_setup)):
        for i in range(3):
            a, b = p[I], pg[i][I]                                   # [k][s][n][m]
            dn = (np.einsum("ksn,ksnm,ksnq->smq", wf, np.conj(b), a)
                  + np.einsum("ksn,ksnm,ksnq->smq", wf, np.conj(a), b))
            F[I, i] = -mult * float(np.real(np.einsum("smq,smq->", V_atoms[I], dn)))
    return F


# ------------------------------------------------------------------------------------------------
# Coulomb integrals (mm'|m''m''') on the real-space grid (Sec. III; definition Eq. B2)
# ------------------------------------------------------------------------------------------------

def _smooth_size(n: int) -> int:
    """Smallest m >= n whose only prime factors are 2, 3 and 5."""
    m = max(n, 1)
    while True:
        k = m
        for p in (2, 3, 5):
            while k % p == 0:
                k //= p
        if k == 1:
            return m
        m += 1


def poisson_box(grid, radius: float):
    """FFT box and truncation radius for an isolated charge inside a sphere of this radius:
    R_c = 2R + 2 max(h), box edge >= (2R + R_c)/h per axis, rounded up to a 2,3,5-smooth size."""
    Rc = 2.0 * radius + 2.0 * max(grid.h)
    nb = [_smooth_size(int(math.ceil((2.0 * radius + Rc) / grid.h[a]))) for a in range(3)]
    return nb, Rc


def truncated_coulomb_kernel(nb, h, Rc) -> np.ndarray:
    """Fourier transform of theta(Rc - r)/r: 4 pi (1 - cos(G Rc)) / G^2, and 2 pi Rc^2 at G = 0."""
    g = [2.0 * math.pi * np.fft.fftfreq(nb[a], d=h[a]) for a in range(3)]
    GX, GY, GZ = np.meshgrid(g[0], g[1], g[2], indexing="ij")
    G2 = GX ** 2 + GY ** 2 + GZ ** 2
    G = np.sqrt(G2)
    with np.errstate(divide="ignore", invalid="ignore"):
        K = 4.0 * math.pi * (1.0 - np.cos(G * Rc)) / G2
    K[0, 0, 0] = 2.0 * math.pi * Rc * Rc
    return K


def hartree_potential(rho_box: np.ndarray, K: np.ndarray) -> np.ndarray:
    """v = IFFT(K FFT(rho)): the potential of an isolated density on the padded box."""
    return np.real(np.fft.ifftn(K * np.fft.fftn(rho_box)))


def coulomb_integrals(grid, atom, smap: Dict[str, np.ndarray]) -> np.ndarray:
    """(mm'|m''m''') = dV sum_r phi_m phi_m' v_{m''m'''},  v from the truncated-kernel FFT Poisson
    solve of phi_m'' phi_m''' on a zero-padded box around the sphere.  Returns [M,M,M,M] Hartree."""
    phi = smap["phi"]
    M = phi.shape[1]
    nb, Rc = poisson_box(grid, atom.radius)
    K = truncated_coulomb_kernel(nb, grid.h, Rc)
    u = smap["u"] - smap["u"].min(axis=0)[None, :]
    rho = {}
    v = {}
    for a in range(M):
        for b in range(a, M):
            box = np.zeros(nb)
            box[u[:, 0], u[:, 1], u[:, 2]] = phi[:, a] * phi[:, b]
            rho[(a, b)] = box
            v[(a, b)] = hartree_potential(box, K)
    out = np.zeros((M, M, M, M))
    for a in range(M):
        for b in range(M):
            for c in range(M):
                for d in range(M):
                    ab, cd = (min(a, b), max(a, b)), (min(c, d), max(c, d))
                    out[a, b, c, d] = grid.dV * np.sum(rho[ab] * v[cd])
    return out
