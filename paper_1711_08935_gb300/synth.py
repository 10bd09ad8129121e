"""Seeded synthetic inputs for the Hubbard-projector workloads.

This module only *creates inputs*: grids, atoms, radial tables, k-points,
Kohn-Sham-like states and occupations.  It contains none of the method's
arithmetic (no sphere maps, no orbital sampling, no projections), so the
CUDA path and the CPU oracle can both consume what it produces without
sharing any step of the computation.

Shapes follow the workloads of the paper: transition-metal oxides on a
rocksalt-like lattice (Sec. III, Table I), a non-collinear p-shell system
(Sec. III, App. A/B) and real-time propagation (Sec. V).  Radial functions
are hydrogen-like stand-ins for the pseudo-atomic orbitals of Sec. II.

States are built from atom-centred Gaussian-type functions (a functional form
the method never uses), Bloch-summed over neighbouring images with the phase
exp(i k.T), mixed with seeded random coefficients, given full-grid noise and
orthonormalised (Cholesky QR, twice) under the grid inner product.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np
import torch
from scipy.special import genlaguerre


@dataclasses.dataclass
class Grid:
    n: tuple            # points per axis (n0, n1, n2); linear index i + n0*(j + n1*k)
    h: tuple            # spacing per axis, bohr
    origin: tuple = (0.0, 0.0, 0.0)
    periodic: bool = True

    @property
    def npts(self) -> int:
        return self.n[0] * self.n[1] * self.n[2]

    @property
    def dV(self) -> float:
        return self.h[0] * self.h[1] * self.h[2]

    @property
    def L(self) -> tuple:
        return tuple(self.n[a] * self.h[a] for a in range(3))


@dataclasses.dataclass
class Atom:
    pos: tuple          # bohr
    species: int
    l: int
    radius: float       # sphere radius, bohr


@dataclasses.dataclass
class Radial:
    dr: float           # uniform radial grid r_i = i*dr
    R: np.ndarray       # R(r_i), float64, len >= 4


@dataclasses.dataclass
class System:
    grid: Grid
    atoms: List[Atom]
    radials: List[Radial]          # one per species
    kpts: np.ndarray               # [nk,3] cartesian, 1/bohr
    wk: np.ndarray                 # [nk], sums to 1
    nspin: int                     # 1 unpolarised, 2 collinear; NC uses nspin=1 with spinors
    noncollinear: bool = False
    name: str = ""

    @property
    def nk(self) -> int:
        return len(self.kpts)


def hydrogenic_radial(n: int, l: int, Z: float, dr: float = 0.002, rmax: float = 12.0) -> Radial:
    """Normalised hydrogen-like radial function R_nl(r) for effective charge Z,
    tabulated on r_i = i*dr (a stand-in for a pseudo-atomic radial)."""
    nr = int(round(rmax / dr)) + 1
    r = np.arange(nr, dtype=np.float64) * dr
    rho = 2.0 * Z * r / n
    lag = genlaguerre(n - l - 1, 2 * l + 1)(rho)
    norm = math.sqrt((2.0 * Z / n) ** 3 * math.factorial(n - l - 1) / (2.0 * n * math.factorial(n + l)))
    R = norm * np.exp(-rho / 2.0) * rho ** l * lag
    return Radial(dr=dr, R=R.astype(np.float64))


def mp_kpoints(grid: Grid, nkgrid: Sequence[int]) -> tuple:
    """Monkhorst-Pack grid without symmetry reduction; weights 1/nk."""
    ks = []
    for a in range(nkgrid[0]):
        for b in range(nkgrid[1]):
            for c in range(nkgrid[2]):
                frac = [(2 * (a, b, c)[i] - nkgrid[i] + 1) / (2.0 * nkgrid[i]) for i in range(3)]
                ks.append([frac[i] * 2.0 * math.pi / grid.L[i] for i in range(3)])
    ks = np.array(ks, dtype=np.float64)
    return ks, np.full(len(ks), 1.0 / len(ks))


# ----------------------------------------------------------------------------------------------
# workload definitions
# ----------------------------------------------------------------------------------------------

def tiny_system() -> System:
    """One atom, 5 real d orbitals (hydrogenic 3d, Z_eff=4), isolated 32^3 box, spacing 0.3,
    sphere radius 4 bohr, atom on grid point (16,16,16), Gamma only, unpolarised."""
    g = Grid(n=(32, 32, 32), h=(0.3, 0.3, 0.3), periodic=False)
    atoms = [Atom(pos=(16 * 0.3, 16 * 0.3, 16 * 0.3), species=0, l=2, radius=4.0)]
    return System(g, atoms, [hydrogenic_radial(3, 2, 4.0)], np.zeros((1, 3)), np.ones(1), nspin=1,
                  name="tiny: 1 atom d-shell, isolated 32^3, h=0.3, R=4")


def oxide_system(n: int = 96, h: float = 0.25, nk: int = 2) -> System:
    """Rocksalt-like oxide supercell: 8 transition-metal atoms (3d, R=4.5) on a 2x2x2 sublattice
    of spacing L/2 and 8 oxygens (2p, R=3.5) displaced by L/4 along (1,1,1); periodic cube of
    n^3 points at spacing h; nk^3 Monkhorst-Pack k-points; collinear spin."""
    g = Grid(n=(n, n, n), h=(h, h, h), periodic=True)
    L = n * h
    atoms = []
    for k in range(2):
        for j in range(2):
            for i in range(2):
                atoms.append(Atom(pos=(i * L / 2, j * L / 2, k * L / 2), species=0, l=2, radius=4.5))
    for k in range(2):
        for j in range(2):
            for i in range(2):
                atoms.append(Atom(pos=(i * L / 2 + L / 4, j * L / 2 + L / 4, k * L / 2 + L / 4),
                                  species=1, l=1, radius=3.5))
    kp, wk = mp_kpoints(g, (nk, nk, nk))
    return System(g, atoms, [hydrogenic_radial(3, 2, 4.0), hydrogenic_radial(2, 1, 4.55)], kp, wk,
                  nspin=2, name=f"oxide: 8 TM(3d,R4.5)+8 O(2p,R3.5), periodic {n}^3 h={h}, {len(kp)} k, collinear")


def small_oxide_system() -> System:
    """Scaled-down oxide: 2 TM + 2 O in a periodic 40^3 cell at spacing 0.3 (L=12 bohr),
    2 k-points, collinear; spheres cross the cell faces so several periodic images occur."""
    g = Grid(n=(40, 40, 40), h=(0.3, 0.3, 0.3), periodic=True)
    atoms = [Atom((0.0, 0.0, 0.0), 0, 2, 4.5), Atom((6.0, 6.0, 0.0), 0, 2, 4.5),
             Atom((3.0, 3.0, 3.0), 1, 1, 3.5), Atom((9.0, 9.0, 3.0), 1, 1, 3.5)]
    L = g.L[0]
    kp = np.array([[0.25 * 2 * math.pi / L, 0.25 * 2 * math.pi / L, -0.25 * 2 * math.pi / L],
                   [-0.25 * 2 * math.pi / L, 0.0, 0.25 * 2 * math.pi / L]])
    return System(g, atoms, [hydrogenic_radial(3, 2, 4.0), hydrogenic_radial(2, 1, 4.55)], kp,
                  np.array([0.5, 0.5]), nspin=2, name="small oxide: 2 TM + 2 O, periodic 40^3 h=0.3, 2 k")


def noncollinear_system(n: int = 96, h: float = 0.25, natoms: int = 10, seed: int = 3) -> System:
    """Bi-like p shells (hydrogenic 2p, Z_eff=2, R=4.5) at seeded random positions in a periodic
    cube; 6 k-points at +-1/4 of a reciprocal vector along each axis; spinor states."""
    g = Grid(n=(n, n, n), h=(h, h, h), periodic=True)
    rng = np.random.default_rng(seed)
    L = n * h
    atoms = [Atom(tuple(float(x) for x in rng.uniform(0, L, 3)), 0, 1, 4.5) for _ in range(natoms)]
    kp = []
    for a in range(3):
        for s in (1, -1):
            k = [0.0, 0.0, 0.0]
            k[a] = s * 0.25 * 2 * math.pi / L
            kp.append(k)
    kp = np.array(kp)
    return System(g, atoms, [hydrogenic_radial(2, 1, 2.0)], kp, np.full(6, 1 / 6), nspin=1,
                  noncollinear=True, name=f"non-collinear: {natoms} p-shell atoms, periodic {n}^3, 6 k")


def rt_system(n: int = 128, h: float = 0.3, nk: int = 4) -> System:
    """64 atoms of 3 species on a 4x4x4 lattice of spacing L/4 with sphere radii 3.5/4.5/5.0
    (species assigned cyclically), periodic n^3 grid; nk k-points along the cell diagonal."""
    g = Grid(n=(n, n, n), h=(h, h, h), periodic=True)
    L = n * h
    radii = (3.5, 4.5, 5.0)
    ls = (1, 2, 2)
    atoms = []
    c = 0
    for k in range(4):
        for j in range(4):
            for i in range(4):
                s = c % 3
                atoms.append(Atom((i * L / 4 + 0.1, j * L / 4 + 0.2, k * L / 4 + 0.3), s, ls[s], radii[s]))
                c += 1
    rads = [hydrogenic_radial(2, 1, 3.0), hydrogenic_radial(3, 2, 4.0), hydrogenic_radial(3, 2, 3.2)]
    kp = np.array([[(q + 0.5) / nk * 2 * math.pi / L / 2] * 3 for q in range(nk)])
    return System(g, atoms, rads, kp, np.full(nk, 1.0 / nk), nspin=1,
                  name=f"real-time: 64 atoms 3 species, periodic {n}^3 h={h}, {nk} k")


# ----------------------------------------------------------------------------------------------
# states and occupations
# ----------------------------------------------------------------------------------------------

_POLY = 9  # 1, x, y, z, xy, yz, xz, x^2-y^2, 3z^2-r^2


def _gaussian_basis(system: System, k: np.ndarray, alpha: Sequence[float], device, dtype) -> torch.Tensor:
    """[natoms*9, npts] complex: atom-centred polynomial x Gaussian functions, Bloch-summed over
    images T in {-1,0,1}^3 (periodic) with exp(i k.T), or single-image (isolated)."""
    g = system.grid
    rdt = torch.float64 if dtype == torch.complex128 else torch.float32
    xs = [torch.arange(g.n[a], device=device, dtype=torch.float64) * g.h[a] + g.origin[a] for a in range(3)]
    Z, Y, X = torch.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    X, Y, Z = X.reshape(-1), Y.reshape(-1), Z.reshape(-1)
    imgs = [(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)] if g.periodic else [(0, 0, 0)]
    out = torch.zeros(len(system.atoms) * _POLY, g.npts, device=device, dtype=torch.complex128)
    for ia, at in enumerate(system.atoms):
        a = alpha[at.species]
        for T in imgs:
            Tv = [T[i] * g.L[i] for i in range(3)]
            dx = X - (at.pos[0] + Tv[0]); dy = Y - (at.pos[1] + Tv[1]); dz = Z - (at.pos[2] + Tv[2])
            r2 = dx * dx + dy * dy + dz * dz
            env = torch.exp(-a * r2)
            if float(env.max()) < 1e-30:
                continue
            ph = complex(math.cos(float(np.dot(k, Tv))), math.sin(float(np.dot(k, Tv))))
            polys = (torch.ones_like(dx), dx, dy, dz, dx * dy, dy * dz, dx * dz, dx * dx - dy * dy,
                     3 * dz * dz - r2)
            for p, P in enumerate(polys):
                out[ia * _POLY + p] += ph * (P * env)
    return out.to(dtype) if dtype != torch.complex128 else out


def _orthonormalise_rows(A: torch.Tensor, dV: float) -> torch.Tensor:
    """Rows of A made orthonormal under <a|b> = dV sum conj(a) b by Cholesky QR applied twice; the
    small Gram matrices are factorised on the host (numpy), the products run where A lives."""
    for _ in range(2):
        Gm = (A @ A.conj().transpose(0, 1)) * dV
        L = np.linalg.cholesky(Gm.cpu().numpy())
        Linv = np.linalg.inv(L)
        A = torch.from_numpy(Linv).to(A.device) @ A
    return A


def make_states(system: System, nbands: int, seed: int, device="cpu", noise: float = 0.05,
                spin_bias: Optional[Sequence[float]] = None, dtype=torch.complex128) -> torch.Tensor:
    """Orthonormal (grid inner product with dV) states.
    Collinear/unpolarised layout [nk][nspin][nbands][npts]; non-collinear [nk][nbands][2][npts].
    spin_bias[i] in [0,1] weights atom i's basis functions in spin-up states (1-bias for spin-down)."""
    g = system.grid
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    alpha = [0.6, 0.9, 0.5, 0.7]
    ns = 2 if system.noncollinear else system.nspin
    nat = len(system.atoms)
    if system.noncollinear:
        out = torch.empty(system.nk, nbands, 2, g.npts, dtype=torch.complex128, device=device)
    else:
        out = torch.empty(system.nk, ns, nbands, g.npts, dtype=torch.complex128, device=device)
    for ik in range(system.nk):
        G = _gaussian_basis(system, system.kpts[ik], alpha, device, torch.complex128)
        nb = G.shape[0]
        chans = 1 if system.noncollinear else ns
        for s in range(chans):
            ncomp = 2 if system.noncollinear else 1
            cols = []
            for comp in range(ncomp):
                C = torch.complex(torch.randn(nb, nbands, generator=gen, device=device, dtype=torch.float64),
                                  torch.randn(nb, nbands, generator=gen, device=device, dtype=torch.float64))
                if spin_bias is not None:
                    sb = torch.tensor([spin_bias[i] if (s + comp) % 2 == 0 else 1.0 - spin_bias[i]
                                       for i in range(nat) for _ in range(_POLY)], device=device,
                                      dtype=torch.float64)
                    C = C * sb[:, None]
                psi = C.transpose(0, 1) @ G        # [nbands, npts]
                scale = psi.abs().pow(2).mean().sqrt()
                nz = torch.complex(torch.randn(nbands, g.npts, generator=gen, device=device, dtype=torch.float64),
                                   torch.randn(nbands, g.npts, generator=gen, device=device, dtype=torch.float64))
                psi = psi + noise * scale * nz
                cols.append(psi)
            A = torch.cat(cols, dim=1) if ncomp == 2 else cols[0]   # [nbands, ncomp*npts]
            Q = _orthonormalise_rows(A, g.dV)
            if system.noncollinear:
                out[ik] = Q.reshape(nbands, 2, g.npts)
            else:
                out[ik, s] = Q
            del A, Q, cols
        del G
    return out.to(dtype) if dtype != torch.complex128 else out


def fermi_occupations(nk: int, nspin: int, nbands: int, kT: float = 0.01, e0: float = -0.5,
                      de: float = 0.05, mu: float = 0.0) -> np.ndarray:
    """f[k][s][n] = 1/(1+exp((e_n-mu)/kT)) with e_n = e0 + de*n."""
    e = e0 + de * np.arange(nbands)
    f = 1.0 / (1.0 + np.exp(np.clip((e - mu) / kT, -700, 700)))
    return np.broadcast_to(f, (nk, nspin, nbands)).copy()


def step_occupations(nk: int, nspin: int, nbands: int, nocc: int) -> np.ndarray:
    """f = 1 for the lowest nocc bands of every k and spin channel, 0 above."""
    f = np.zeros((nk, nspin, nbands))
    f[:, :, :nocc] = 1.0
    return f


def afm_spin_bias(system: System, strong: float = 0.85) -> List[float]:
    """Antiferromagnetic seed: transition-metal atom i gets majority-up weight `strong` when
    (ix+iy+iz) of its sublattice position is even, else majority-down; other atoms 0.5."""
    L = system.grid.L
    out = []
    for at in system.atoms:
        if at.l == 2:
            par = sum(int(round(at.pos[a] / (L[a] / 2))) for a in range(3)) % 2
            out.append(strong if par == 0 else 1.0 - strong)
        else:
            out.append(0.5)
    return out


def molecule_systems(nsys: int, seed: int = 5, edge=(48, 80), natoms=(1, 8), radius=(4.0, 5.0), nstates=(20, 200),
                     h: float = 0.3) -> List[System]:
    """Independent isolated molecules: cubic boxes with edge drawn uniformly from `edge` (points) at
    spacing h, 1-8 transition-metal d shells (hydrogenic 3d, Z_eff = 4) with radii uniform in `radius`
    and centres uniform in the box shrunk by the radius, Gamma only, collinear spin.  The band count
    of each system is drawn from `nstates` and stored in System.name as 'nb=<n>'."""
    rng = np.random.default_rng(seed)
    rad = hydrogenic_radial(3, 2, 4.0)
    out = []
    for s in range(nsys):
        n = int(rng.integers(edge[0], edge[1] + 1))
        g = Grid((n, n, n), (h, h, h), periodic=False)
        L = n * h
        na = int(rng.integers(natoms[0], natoms[1] + 1))
        atoms = []
        for _ in range(na):
            R = float(rng.uniform(*radius))
            lo, hi = R, max(R, L - R)
            atoms.append(Atom(tuple(float(x) for x in rng.uniform(lo, hi, 3)), 0, 2, R))
        nb = int(rng.integers(nstates[0], nstates[1] + 1))
        out.append(System(g, atoms, [rad], np.zeros((1, 3)), np.ones(1), nspin=2, name=f"nb={nb}"))
    return out


def bands_of(system: System) -> int:
    """Band count stored by molecule_systems."""
    return int(system.name.split("nb=")[1])


def analytic_states(system: System, nbands: int, seed: int, shift=(0.0, 0.0, 0.0)):
    """States built only from the atom-centred Gaussian-type functions (no noise), evaluated at r + shift,
    together with their exact Cartesian gradients.  Returns numpy (psi, [dpsi_x, dpsi_y, dpsi_z]) with the
    collinear layout [nk][nspin][nbands][npts].  The coefficients depend on the seed only, so shifted
    copies describe the same states translated by -shift (used to check forces by finite differences)."""
    g = system.grid
    rng = np.random.default_rng(seed)
    alpha = [0.6, 0.9, 0.5, 0.7]
    xs = [np.arange(g.n[a]) * g.h[a] + g.origin[a] + shift[a] for a in range(3)]
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    X, Y, Z = X.reshape(-1), Y.reshape(-1), Z.reshape(-1)
    imgs = [(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)] if g.periodic else [(0, 0, 0)]
    nat = len(system.atoms)
    out = np.zeros((system.nk, system.nspin, nbands, g.npts), dtype=np.complex128)
    dout = [np.zeros_like(out) for _ in range(3)]
    for ik in range(system.nk):
        G = np.zeros((nat * 4, g.npts), dtype=np.complex128)
        dG = [np.zeros_like(G) for _ in range(3)]
        for ia, at in enumerate(system.atoms):
            a = alpha[at.species]
            for T in imgs:
                Tv = [T[i] * g.L[i] for i in range(3)]
                d = [X - (at.pos[0] + Tv[0]), Y - (at.pos[1] + Tv[1]), Z - (at.pos[2] + Tv[2])]
                env = np.exp(-a * (d[0] ** 2 + d[1] ** 2 + d[2] ** 2))
                ph = np.exp(1j * float(np.dot(system.kpts[ik], Tv)))
                polys = [np.ones_like(d[0]), d[0], d[1], d[0] * d[2]]
                dpolys = [[0 * d[0], 0 * d[0], 0 * d[0]], [np.ones_like(d[0]), 0 * d[0], 0 * d[0]],
                          [0 * d[0], np.ones_like(d[0]), 0 * d[0]], [d[2], 0 * d[0], d[0]]]
                for p in range(4):
                    G[ia * 4 + p] += ph * polys[p] * env
                    for c in range(3):
                        dG[c][ia * 4 + p] += ph * (dpolys[p][c] - 2 * a * d[c] * polys[p]) * env
        for s in range(system.nspin):
            C = rng.normal(size=(nat * 4, nbands)) + 1j * rng.normal(size=(nat * 4, nbands))
            out[ik, s] = C.T @ G
            for c in range(3):
                dout[c][ik, s] = C.T @ dG[c]
    return out, dout
