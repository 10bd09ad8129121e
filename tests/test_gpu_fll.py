"""Fully-localised-limit decomposition of App. A (E_ee of Eq. A1, E_DC of Eq. A3 with the m.m term) on
the GPU against the oracle, per atom: collinear, unpolarised and non-collinear handles, fixed U and
ACBN0 U.  The values are small FP64 contractions of the occupation matrices, which agree with the
oracle to 1e-12 relative (complex128 states), so E_ee and E_DC are held to 1e-11 Hartree."""
import numpy as np
import pytest
import torch

from oracle import dftu_oracle as O
from paper_1711_08935_gb300 import synth
from tests import _cases as C
from tests._gpu import run_pass

pytestmark = pytest.mark.gpu


def _coulombs(s, st):
    out = []
    for sp in range(len(s.radials)):
        I = [a.species for a in s.atoms].index(sp)
        out.append(O.coulomb_integrals(s.grid, s.atoms[I], st[I]))
    return out


def _check(s, psi, f, fixed=None, acbn0=False):
    st = O.setup_atoms(s)
    V = _coulombs(s, st) if acbn0 else None
    ref = O.hubbard_pass(s, st, psi, f, coulomb=V, fixed_u=fixed)
    out = run_pass(s, psi, f, coulomb=V, fixed_u=fixed)
    ee, dc = out["handle"].fll_energy()
    for I in range(len(s.atoms)):
        r_ee, r_dc = O.fll_energy(ref["occ"][I][0], ref["U"][I], ref["J"][I], s.noncollinear, s.nspin)
        assert abs(ee[I] - r_ee) < 1e-11, (I, ee[I], r_ee)
        assert abs(dc[I] - r_dc) < 1e-11, (I, dc[I], r_dc)
    assert np.max(np.abs(dc)) > 1e-3
    out["handle"].close()


@pytest.mark.parametrize("nspin", [2, 1])
def test_fll_energy_collinear(nspin):
    s = C.periodic_two_atoms(nspin=nspin)
    nb = 9
    psi = C.states_np(s, nb, seed=21)
    f = np.random.default_rng(5).uniform(0, 1, (s.nk, nspin, nb))
    _check(s, psi, f, fixed=[(0.35, 0.05), (0.22, 0.02)])
    _check(s, psi, f, acbn0=True)


def test_fll_energy_noncollinear():
    s = C.periodic_two_atoms(nspin=1)
    s.noncollinear = True
    nb = 10
    psi = synth.make_states(s, nb, seed=43, device="cpu").numpy()
    f = np.random.default_rng(6).uniform(0, 1, (s.nk, nb))
    _check(s, psi, f, fixed=[(0.3, 0.04), (0.27, 0.01)])
    _check(s, psi, f, acbn0=True)
