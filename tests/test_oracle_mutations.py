"""Planted mistakes in the CPU oracle must each fail at least one of its pins.

Every case replaces one oracle function by a plausibly wrong version of it (a flipped sign, a dropped
term or factor, a transposed operand, a wrong index) for the length of one pin, on the CPU, and checks
that the pin named beside it fails.  This is what makes the pins worth trusting: a pin set that
passes a wrong oracle would also pass a wrong GPU path that agrees with it.
"""
import contextlib

import numpy as np
import pytest

from oracle import dftu_oracle as O
from tests import test_oracle_pins as P

ORIG = {name: getattr(O, name) for name in dir(O) if callable(getattr(O, name))}


@contextlib.contextmanager
def planted(**repl):
    saved = {k: getattr(O, k) for k in repl}
    try:
        for k, fn in repl.items():
            setattr(O, k, fn)
        yield
    finally:
        for k, fn in saved.items():
            setattr(O, k, fn)


def _acbn0_variant(numJ_idx="adcb", denom_from_P=False, numU_pairs="ab,cd"):
    """The collinear ACBN0 ratio (Eqs. 10-11) with one term written wrongly (see the cases below)."""
    def acbn0(rho_s, Pb_rho_s, V, nspin):
        n, Pm = O.paper_n(rho_s), O.paper_n(Pb_rho_s)
        if nspin == 1:
            n, Pm = np.stack([n[0], n[0]]), np.stack([Pm[0], Pm[0]])
        M = n.shape[-1]
        D = Pm if denom_from_P else n
        N = np.real(np.einsum("smm->sm", D))
        numU = sum(np.einsum(numU_pairs + ",abcd->", Pm[a], Pm[b], V) for a in range(2) for b in range(2))
        numJ = sum(np.einsum("ab,cd," + numJ_idx + "->", Pm[a], Pm[a], V) for a in range(2))
        off = 1.0 - np.eye(M)
        same = sum(np.einsum("m,q,mq->", N[a], N[a], off) for a in range(2))
        opp = sum(np.einsum("m,q->", N[a], N[1 - a]) for a in range(2))
        if abs(same + opp) < O.ZERO_DENOM or abs(same) < O.ZERO_DENOM:
            return 0.0, 0.0, True
        return float(np.real(numU) / (same + opp)), float(np.real(numJ) / same), False
    return acbn0


def _smap_variant(fn):
    def sphere_map(grid, atom):
        return fn(ORIG["sphere_map"](grid, atom))
    return sphere_map


def _neg_T(sm):
    sm = dict(sm)
    sm["T"] = -sm["T"]
    return sm


def _shift_idx(sm):   # gather from the neighbouring grid point along x
    sm = dict(sm)
    sm["idx"] = np.where(sm["idx"] < sm["idx"].max(), sm["idx"] + 1, sm["idx"])
    return sm


def _nbar_all_atoms(system, p_atoms, noncollinear=False):
    ax = (-2, -1) if noncollinear else (-1,)
    tot = sum(np.sum(np.abs(p) ** 2, axis=ax) for p in p_atoms)
    return [tot for _ in system.radials]


def _occupations_variant(transpose=False, drop_wk=False):
    def occupations(system, p_atoms, f):
        nb_s = O.nbar(system, p_atoms)
        wk = np.ones(len(system.wk)) if drop_wk else np.asarray(system.wk)
        out = []
        for I, at in enumerate(system.atoms):
            p = p_atoms[I]
            wf = wk[:, None, None] * f
            spec = "ksn,ksnq,ksnm->smq" if transpose else "ksn,ksnm,ksnq->smq"
            out.append((np.einsum(spec, wf, p, np.conj(p)),
                        np.einsum(spec, wf * nb_s[at.species], p, np.conj(p))))
        return out
    return occupations


def _ylm_scaled(l, d, r):
    Y = ORIG["real_ylm"](l, d, r)
    if l == 2:
        Y = Y.copy()
        Y[:, 2] *= 1.05   # a wrong normalisation constant for 3z^2 - r^2
    return Y


def _radial_linear(dr, table, r):
    return np.interp(r, dr * np.arange(len(table)), table, right=0.0)


def _kernel_no_g0(nb, h, Rc):
    K = ORIG["truncated_coulomb_kernel"](nb, h, Rc).copy()
    K.flat[0] = 0.0
    return K


def _fll_without_mm(rho, U, J, noncollinear, nspin=2):
    ee, dc = ORIG["fll_energy"](rho, U, J, noncollinear, nspin)
    nb = O.spin_blocks(rho, noncollinear, nspin)
    tr = np.array([[np.trace(nb[s, t]) for t in range(2)] for s in range(2)])
    mz = np.real(tr[0, 0] - tr[1, 1])
    mx = np.real(tr[0, 1] + tr[1, 0])
    my = np.real(1j * (tr[0, 1] - tr[1, 0]))
    return ee, dc + 0.25 * J * (mx * mx + my * my + mz * mz)


def _strict_boundary(grid, atom):
    sm = ORIG["sphere_map"](grid, atom)
    keep = sm["r"] < atom.radius
    return {k: v[keep] for k, v in sm.items()}


def _occupations_nc_m_major(system, p_atoms, f):
    """Spin-block matrices with the combined index m*2 + c instead of c*M + m."""
    swapped = [p.transpose(0, 1, 3, 2)[..., None, :, :].reshape(p.shape) for p in p_atoms]
    return ORIG["occupations_nc"](system, swapped, f)


def _acbn0_nc_without_spin_flip(rho, Pb_rho, V):
    """Eqs. (B5)-(B6) with the spin-flip products N^{s,-s} N^{-s,s} left out of both denominators."""
    M = rho.shape[0] // 2
    n = O.paper_n(rho).reshape(2, M, 2, M).transpose(0, 2, 1, 3)
    Pm = O.paper_n(Pb_rho).reshape(2, M, 2, M).transpose(0, 2, 1, 3)
    Nd = np.einsum("abmm->abm", n)
    off = 1.0 - np.eye(M)
    numU = sum(np.einsum("ab,cd,abcd->", Pm[s, s], Pm[t, t], V) for s in range(2) for t in range(2))
    numJ = sum(np.einsum("ab,cd,adcb->", Pm[s, t], Pm[t, s], V) for s in range(2) for t in range(2))
    den_u = sum(np.einsum("m,q->", Nd[s, s], Nd[1 - s, 1 - s]) + np.einsum("m,q,mq->", Nd[s, s], Nd[s, s], off)
                for s in range(2))
    den_j = sum(np.einsum("m,q,mq->", Nd[s, s], Nd[s, s], off) for s in range(2))
    return float(np.real(numU) / np.real(den_u)), float(np.real(numJ) / np.real(den_j)), False


def _fll_without_spin_flip_exchange(rho, U, J, noncollinear, nspin=2):
    """E_ee of Eq. (A1) with the -J/2 spin-flip (off-diagonal spin block) term left out."""
    ee, dc = ORIG["fll_energy"](rho, U, J, noncollinear, nspin)
    nb = O.spin_blocks(rho, noncollinear, nspin)
    d = np.array([[np.diagonal(nb[s, t]) for t in range(2)] for s in range(2)])
    flip = sum(-0.5 * J * (np.sum(d[s, 1 - s]) * np.sum(d[1 - s, s]) - np.sum(d[s, 1 - s] * d[1 - s, s])) for s in range(2))
    return ee - float(np.real(flip)), dc


# name -> (replacements, pin that must fail, its arguments)
CASES = {
    "Bloch phase with the wrong sign": (
        dict(phases=lambda system, smap, k: np.conj(ORIG["phases"](system, smap, k))),
        P.test_projection_matches_brute_force, ("self_overlap",)),
    "Bloch phase dropped": (
        dict(phases=lambda system, smap, k: np.ones(len(smap["idx"]), dtype=np.complex128)),
        P.test_projection_matches_brute_force, ("self_overlap",)),
    "lattice image with the wrong sign": (
        dict(sphere_map=_smap_variant(_neg_T)),
        P.test_sphere_map_canonical_order_and_folding, ()),
    "gather from the neighbouring grid point": (
        dict(sphere_map=_smap_variant(_shift_idx)),
        P.test_projection_matches_brute_force, ("isolated",)),
    "sphere boundary taken as strict": (
        dict(sphere_map=_strict_boundary),
        P.test_sphere_boundary_is_inclusive, ()),
    "orbitals not orthonormalised": (
        dict(lowdin=lambda phi, dV: phi),
        P.test_lowdin_orthonormal_and_symmetric, ()),
    "S^-1 in place of S^-1/2": (
        dict(lowdin=lambda phi, dV: phi @ np.linalg.inv(dV * (phi.T @ phi))),
        P.test_lowdin_orthonormal_and_symmetric, ()),
    "wrong normalisation of one real harmonic": (
        dict(real_ylm=_ylm_scaled),
        P.test_real_ylm_orthonormal_on_sphere, (2,)),
    "linear in place of cubic radial interpolation": (
        dict(radial_value=_radial_linear),
        P.test_radial_interpolation_exact_on_cubics_and_converges, ()),
    "projection conjugated": (
        dict(project=lambda system, st, psi: [np.conj(p) for p in ORIG["project"](system, st, psi)]),
        P.test_projection_matches_brute_force, ("self_overlap",)),
    "volume element dropped from the projection": (
        dict(project=lambda system, st, psi: [p / system.grid.dV for p in ORIG["project"](system, st, psi)]),
        P.test_states_equal_orbitals_give_identity, ()),
    "Nbar summed over every species": (
        dict(nbar=_nbar_all_atoms),
        P.test_nbar_closed_form_for_scaled_orbital_states, ()),
    "Nbar from |p| instead of |p|^2": (
        dict(nbar=lambda system, p_atoms, noncollinear=False: [
            np.sqrt(x) for x in ORIG["nbar"](system, p_atoms, noncollinear)]),
        P.test_nbar_closed_form_for_scaled_orbital_states, ()),
    "spinor Nbar from one component": (
        dict(nbar=lambda system, p_atoms, noncollinear=False: ORIG["nbar"](
            system, [p[..., :1, :] for p in p_atoms] if noncollinear else p_atoms, noncollinear)),
        P.test_nbar_closed_form_for_scaled_orbital_spinors, ()),
    "occupations without the k-point weights": (
        dict(occupations=_occupations_variant(drop_wk=True)),
        P.test_occupations_hermitian_bounded_and_nbar_bounds, ()),
    "occupations stored untransposed": (
        dict(occupations=_occupations_variant(transpose=True)),
        P.test_potential_is_energy_gradient_with_transposition, ()),
    "spinor matrices in the m-major combined index": (
        dict(occupations_nc=_occupations_nc_m_major),
        P.test_noncollinear_reduces_to_collinear_for_spin_pure_spinors, ()),
    "non-collinear denominators without the spin-flip products": (
        dict(acbn0_uj_nc=_acbn0_nc_without_spin_flip),
        P.test_noncollinear_energy_is_spin_rotation_invariant, ()),
    "non-collinear energy with n n^T in place of n n": (
        dict(hubbard_energy_nc=lambda rho, U: 0.5 * U * float(np.real(
            np.trace(O.paper_n(rho)) - np.einsum("ab,ab->", O.paper_n(rho), O.paper_n(rho))))),
        P.test_noncollinear_energy_is_spin_rotation_invariant, ()),
    "exchange numerator with the Hartree index order": (
        dict(acbn0_uj=_acbn0_variant(numJ_idx="abcd")),
        P.test_acbn0_closed_form_diagonal_unpolarised, ()),
    "printed index typo in the U numerator": (
        dict(acbn0_uj=_acbn0_variant(numU_pairs="ab,bc")),
        P.test_acbn0_closed_form_diagonal_unpolarised, ()),
    "denominators from Pbar instead of n": (
        dict(acbn0_uj=_acbn0_variant(denom_from_P=True)),
        P.test_acbn0_collinear_spin_sums, ()),
    "potential with the printed, untransposed n": (
        dict(potential=lambda rho, U: ORIG["potential"](np.swapaxes(rho, -1, -2), U)),
        P.test_potential_is_energy_gradient_with_transposition, ()),
    "potential with the wrong sign": (
        dict(potential=lambda rho, U: -ORIG["potential"](rho, U)),
        P.test_dudarev_energy_and_potential_closed_forms_diagonal, ()),
    "energy without the quadratic term": (
        dict(hubbard_energy=lambda rho_s, U, nspin: ORIG["hubbard_energy"](rho_s, U, nspin)
             + 0.5 * U * (2 // nspin) * float(np.real(np.einsum("smq,sqm->", rho_s, rho_s)))),
        P.test_dudarev_energy_and_potential_closed_forms_diagonal, ()),
    "apply with V transposed": (
        dict(apply=lambda system, st, psi, p, V, coef=1.0: ORIG["apply"](
            system, st, psi, p, [np.swapaxes(v, -1, -2) for v in V], coef)),
        P.test_apply_matches_dense_operator, ()),
    "third-order propagator": (
        dict(taylor_step=lambda *a, **k: ORIG["taylor_step"](*a, **{**k, "order": 3})),
        P.test_taylor_step_on_eigenstates_is_the_fourth_order_polynomial, ()),
    "propagator with the wrong sign of the time step": (
        dict(taylor_step=lambda system, st, psi, f, dt, **k: ORIG["taylor_step"](system, st, psi, f, -dt, **k)),
        P.test_taylor_step_matches_exponential_and_conserves_norm, ()),
    "Coulomb kernel without its G = 0 term": (
        dict(truncated_coulomb_kernel=_kernel_no_g0),
        P.test_poisson_gaussian_self_energy, ()),
    "Coulomb integrals with two indices exchanged": (
        dict(coulomb_integrals=lambda grid, atom, smap: np.transpose(
            ORIG["coulomb_integrals"](grid, atom, smap), (0, 2, 1, 3))),
        P.test_coulomb_integrals_against_slater_integrals, ("p",)),
    "gauge phase missing from the projection": (
        dict(project_gauge=lambda system, st, psi, A: ORIG["project"](system, st, psi)),
        P.test_gauge_operator_equals_literal_definition_on_isolated_box, ()),
    "gauge scatter with the gather's phase": (
        dict(apply_gauge=lambda system, st, psi, p, V, A, coef=1.0: ORIG["apply_gauge"](
            system, st, psi, p, V, -np.asarray(A, dtype=np.float64), coef)),
        P.test_gauge_operator_equals_literal_definition_on_isolated_box, ()),
    "current components on the wrong axes": (
        dict(hubbard_current=lambda *a: ORIG["hubbard_current"](*a)[[1, 2, 0]]),
        P.test_hubbard_current_is_energy_derivative_in_A, ()),
    "forces from the gradients of the wrong axes": (
        dict(hubbard_forces=lambda system, st, psi, dpsi, f, V: ORIG["hubbard_forces"](
            system, st, psi, [dpsi[1], dpsi[2], dpsi[0]], f, V)),
        P.test_hubbard_forces_match_finite_difference_of_energy, ()),
    "Coulomb truncation radius too short": (
        dict(poisson_box=lambda grid, radius: (ORIG["poisson_box"](grid, radius)[0], 1.0 * radius)),
        P.test_coulomb_integrals_against_slater_integrals, ("d",)),
    "unpolarised channel counted once in the energy": (
        dict(hubbard_energy=lambda rho_s, U, nspin: ORIG["hubbard_energy"](rho_s, U, nspin) / (2 if nspin == 1 else 1)),
        P.test_dudarev_energy_and_potential_closed_forms_diagonal, ()),
    "spinor occupations without the k-point weights": (
        dict(occupations_nc=lambda system, p_atoms, f: ORIG["occupations_nc"](
            system, p_atoms, f * len(system.wk) * np.asarray(system.wk)[:, None] ** 0)),
        P.test_noncollinear_reduces_to_collinear_for_spin_pure_spinors, ()),
    "FLL E_ee without the spin-flip exchange": (
        dict(fll_energy=_fll_without_spin_flip_exchange),
        P.test_fll_energy_vanishes_for_integer_occupations, ()),
    "FLL double counting without the m.m term": (
        dict(fll_energy=_fll_without_mm),
        P.test_fll_double_counting_moment_term, ()),
    "forces with the wrong sign": (
        dict(hubbard_forces=lambda *a: -ORIG["hubbard_forces"](*a)),
        P.test_hubbard_forces_match_finite_difference_of_energy, ()),
    "gauge phase with the wrong sign": (
        dict(gauge_phases=lambda smap, A: np.conj(ORIG["gauge_phases"](smap, A))),
        P.test_gauge_operator_equals_literal_definition_on_isolated_box, ()),
    "Hubbard current with the wrong sign": (
        dict(hubbard_current=lambda *a: -ORIG["hubbard_current"](*a)),
        P.test_hubbard_current_is_energy_derivative_in_A, ()),
}


def test_every_pin_passes_on_the_unmodified_oracle():
    for _, (_, pin, args) in CASES.items():
        pin(*args)


@pytest.mark.parametrize("name", list(CASES))
def test_planted_mistake_fails_its_pin(name):
    repl, pin, args = CASES[name]
    with planted(**repl):
        with pytest.raises(AssertionError):
            pin(*args)
