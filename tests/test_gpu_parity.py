"""GPU library vs the CPU FP64 oracle, element by element, on seeded small systems.

Tolerances (from the arithmetic of each path):
  complex128 states (FP32-pair or native FP64): projections, n, Pbar, Nbar and the applied states to
  1e-12 relative to the largest element; U and J to 1e-10 eV.
  complex64 states: |dn| <= 1e-6, U and J to 1e-4 eV (the states themselves carry 2^-24 rounding).
Sphere maps (grid index and lattice image of every point, canonical order) are compared bit for bit.
"""
import math

import numpy as np
import pytest
import torch

from oracle import dftu_oracle as O
from paper_1711_08935_gb300 import dftu, synth
from tests import _cases as C
from tests._gpu import run_pass, split_p

pytestmark = pytest.mark.gpu
EV = O.HARTREE_EV


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def isolated_aniso():
    g = synth.Grid((14, 13, 12), (0.4, 0.45, 0.5), (0.1, -0.2, 0.0), periodic=False)
    return synth.System(g, [synth.Atom((2.3, 2.9, 3.1), 0, 1, 2.4), synth.Atom((3.6, 2.2, 2.9), 1, 3, 2.2)],
                        [synth.hydrogenic_radial(2, 1, 2.5), synth.hydrogenic_radial(4, 3, 5.0)],
                        np.zeros((1, 3)), np.ones(1), nspin=1, name="isolated anisotropic, p + f")


SYSTEMS = {
    "tiny": synth.tiny_system,
    "periodic_self_overlap": C.periodic_tiny,
    "periodic_two_atoms": C.periodic_two_atoms,
    "isolated_aniso": isolated_aniso,
    "small_oxide": synth.small_oxide_system,
}


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_sphere_maps_bit_exact_and_orbitals(name):
    s = SYSTEMS[name]()
    h = dftu.handle_for_system(s, 4)
    st = O.setup_atoms(s)
    for I in range(len(s.atoms)):
        idx, img, phi = h.get_sphere(I)
        assert np.array_equal(idx.astype(np.int64), st[I]["idx"])
        assert np.array_equal(img.astype(np.int64), st[I]["T"])
        assert rel(phi, st[I]["phi"]) < 1e-13
    h.close()


def _collinear_case(name, nb=12, seed=5):
    s = SYSTEMS[name]()
    psi = C.states_np(s, nb, seed=seed)
    rng = np.random.default_rng(seed)
    f = rng.uniform(0.0, 1.0, (s.nk, s.nspin, nb))
    return s, psi, f


def _coulombs(s, st):
    out = []
    for sp in range(len(s.radials)):
        I = [a.species for a in s.atoms].index(sp)
        out.append(O.coulomb_integrals(s.grid, s.atoms[I], st[I]))
    return out


@pytest.mark.parametrize("name", ["periodic_self_overlap", "periodic_two_atoms", "small_oxide", "isolated_aniso"])
@pytest.mark.parametrize("mode", ["pair", "native", "c64"])
def test_full_pass_collinear(name, mode):
    s, psi, f = _collinear_case(name)
    st = O.setup_atoms(s)
    V = _coulombs(s, st)
    ref = O.hubbard_pass(s, st, psi, f, coulomb=V, coef=1.0)
    dtype = torch.complex64 if mode == "c64" else torch.complex128
    md = dftu.F64_NATIVE if mode == "native" else dftu.F64_PAIR
    out = run_pass(s, psi, f, coulomb=V, dtype=dtype, mode=md)
    p = split_p(s, out["p"])
    fp64 = mode != "c64"
    tol_p = 1e-12 if fp64 else 2e-6
    for I in range(len(s.atoms)):
        assert rel(p[I], ref["p"][I]) < tol_p, (I, rel(p[I], ref["p"][I]))
        n_ref = O.paper_n(ref["occ"][I][0])
        Pb_ref = O.paper_n(ref["occ"][I][1])
        if fp64:
            assert rel(out["n"][I], n_ref) < 1e-12
            assert rel(out["Pbar"][I], Pb_ref) < 1e-12
        else:
            assert np.max(np.abs(out["n"][I] - n_ref)) < 1e-6
            assert np.max(np.abs(out["Pbar"][I] - Pb_ref)) < 1e-6
    for sp, nb_ref in enumerate(O.nbar(s, ref["p"])):
        got = out["Nbar"][:, :, sp].reshape(nb_ref.shape)
        assert np.max(np.abs(got - nb_ref)) < (1e-12 if fp64 else 2e-6)
    tol_uj = 1e-10 if fp64 else 1e-4
    assert np.max(np.abs(out["U"] - ref["U"])) * EV < tol_uj
    assert np.max(np.abs(out["J"] - ref["J"])) * EV < tol_uj
    assert abs(out["EU"] - ref["E"]) * EV < (1e-10 if fp64 else 1e-4)
    assert rel(out["psi_out"], ref["psi_out"]) < (1e-12 if fp64 else 1e-6)
    assert out["status"] == dftu.DFTU_OK


def test_tiny_workload_closed_forms_on_gpu():
    """Orbitals first then Gram-Schmidt (the tiny workload): n = Pbar = diag(f_0..f_4) on the GPU too."""
    from tests.test_oracle_pins import tiny_config_states
    s = synth.tiny_system()
    st = O.setup_atoms(s)
    psi = tiny_config_states(s, st)
    f = synth.fermi_occupations(1, 1, 21)
    out = run_pass(s, psi, f, gpu_coulomb=True)
    assert np.allclose(out["n"][0][0], np.diag(f[0, 0, :5]), atol=1e-12)
    assert np.allclose(out["Pbar"][0][0], out["n"][0][0], atol=1e-12)
    Vref = _coulombs(s, st)[0]
    F, Q = f[0, 0, :5].sum(), (f[0, 0, :5] ** 2).sum()
    fm = f[0, 0, :5]
    Vg = out["handle"].coulomb_integrals(0)
    Uc = 4 * np.einsum("a,c,aacc->", fm, fm, Vg) / (2 * (F * F - Q) + 2 * F * F)
    Jc = np.einsum("a,c,acca->", fm, fm, Vg) / (F * F - Q)
    assert abs(out["U"][0] - Uc) * EV < 1e-10 and abs(out["J"][0] - Jc) * EV < 1e-10
    assert rel(Vg, Vref) < 1e-10


@pytest.mark.parametrize("name", ["tiny", "small_oxide"])
def test_coulomb_integrals_match_oracle(name):
    s = SYSTEMS[name]()
    st = O.setup_atoms(s)
    h = dftu.handle_for_system(s, 2)
    for sp, Vref in enumerate(_coulombs(s, st)):
        assert rel(h.coulomb_integrals(sp), Vref) < 1e-10
    h.close()


@pytest.mark.parametrize("mode", ["pair", "c64"])
def test_full_pass_noncollinear(mode):
    s = C.periodic_two_atoms(nspin=1)
    s.noncollinear = True
    nb = 10
    psi = synth.make_states(s, nb, seed=41, device="cpu").numpy()
    f = np.random.default_rng(2).uniform(0, 1, (s.nk, nb))
    st = O.setup_atoms(s)
    V = _coulombs(s, st)
    ref = O.hubbard_pass(s, st, psi, f, coulomb=V)
    dtype = torch.complex64 if mode == "c64" else torch.complex128
    out = run_pass(s, psi, f, coulomb=V, dtype=dtype)
    fp64 = mode == "pair"
    p = split_p(s, out["p"])
    for I in range(2):
        assert rel(p[I], ref["p"][I]) < (1e-12 if fp64 else 2e-6)
        n_ref = O.paper_n(ref["occ"][I][0])
        assert np.max(np.abs(out["n"][I][0] - n_ref)) < (1e-12 if fp64 else 1e-6)
    assert np.max(np.abs(out["U"] - ref["U"])) * EV < (1e-10 if fp64 else 1e-4)
    assert np.max(np.abs(out["J"] - ref["J"])) * EV < (1e-10 if fp64 else 1e-4)
    assert abs(out["EU"] - ref["E"]) * EV < (1e-10 if fp64 else 1e-4)
    assert rel(out["psi_out"], ref["psi_out"]) < (1e-12 if fp64 else 1e-6)


def test_fixed_u_and_complex_coefficient():
    """Fixed-U DFT+U (Sec. II) and a complex apply coefficient (the Taylor-step use)."""
    s, psi, f = _collinear_case("periodic_two_atoms", nb=7, seed=9)
    st = O.setup_atoms(s)
    fixed = [(0.25, 0.03), (0.4, 0.0)]
    coef = complex(0.0, -0.01)
    ref = O.hubbard_pass(s, st, psi, f, fixed_u=fixed, coef=coef)
    out = run_pass(s, psi, f, fixed_u=fixed, coef=coef)
    assert np.allclose(out["U"], [0.25, 0.4]) and np.allclose(out["J"], [0.03, 0.0])
    assert abs(out["EU"] - ref["E"]) < 1e-13
    assert rel(out["psi_out"], ref["psi_out"]) < 1e-12


def test_edge_cases_bands_padding_zero_states():
    """nbands = 1 and an odd band count, ld_band > npts (padded rows), an all-zero state."""
    s, psi, f = _collinear_case("periodic_two_atoms", nb=3, seed=3)
    psi[:, :, 1] = 0.0
    st = O.setup_atoms(s)
    ref = O.hubbard_pass(s, st, psi, f, fixed_u=[(0.3, 0.05), (0.2, 0.01)])
    pad = np.zeros(psi.shape[:3] + (psi.shape[3] + 37,), dtype=complex)
    pad[..., :psi.shape[3]] = psi
    h = dftu.handle_for_system(s, 5)
    dev = torch.device("cuda:0")
    tp = torch.from_numpy(pad).to(dev)
    h.set_u(0, 0.3, 0.05)
    h.set_u(1, 0.2, 0.01)
    h.project(tp)
    p = split_p(s, h.projections(3))
    for I in range(2):
        assert rel(p[I], ref["p"][I]) < 1e-12
        assert np.all(p[I][:, :, 1] == 0)
    h.occupations(torch.from_numpy(f).to(dev))
    h.acbn0_uj()
    h.apply(tp)
    got = tp.cpu().numpy()
    assert rel(got[..., :psi.shape[3]], ref["psi_out"]) < 1e-12
    assert np.all(got[..., psi.shape[3]:] == 0)
    # one band only
    out1 = run_pass(s, psi[:, :, :1].copy(), f[:, :, :1].copy(), fixed_u=[(0.3, 0.05), (0.2, 0.01)])
    ref1 = O.hubbard_pass(s, st, psi[:, :, :1].copy(), f[:, :, :1].copy(), fixed_u=[(0.3, 0.05), (0.2, 0.01)])
    assert rel(out1["psi_out"], ref1["psi_out"]) < 1e-12


def test_device_status_nonfinite_and_zero_denominator():
    s, psi, f = _collinear_case("periodic_two_atoms", nb=4, seed=1)
    st = O.setup_atoms(s)
    V = _coulombs(s, st)
    out = run_pass(s, psi, np.zeros_like(f), coulomb=V)    # empty shells: ACBN0 denominators vanish
    assert out["status"] == dftu.DFTU_ERR_ZERO_DENOM
    assert np.all(out["U"] == 0) and np.all(out["J"] == 0)
    bad = psi.copy()
    bad[0, 0, 2, st[0]["idx"][5]] = np.nan
    h = dftu.handle_for_system(s, 4)
    h.project(torch.from_numpy(bad).cuda())
    assert h.sync_status() == dftu.DFTU_ERR_NONFINITE
    assert h.sync_status() == dftu.DFTU_OK                  # the status word is cleared by reading it


def test_argument_and_order_errors():
    s, psi, f = _collinear_case("periodic_two_atoms", nb=2, seed=1)
    h = dftu.handle_for_system(s, 2)
    t = torch.from_numpy(psi).cuda()
    with pytest.raises(dftu.DftuError) as e:
        h.acbn0_uj()
    assert e.value.status == dftu.DFTU_ERR_NOT_READY
    h.project(t)
    h.occupations(torch.from_numpy(f).cuda())
    with pytest.raises(dftu.DftuError) as e:
        h.acbn0_uj()                                        # no Coulomb integrals, no fixed U
    assert e.value.status == dftu.DFTU_ERR_NOT_READY
    big = torch.zeros((s.nk, 2, 3, s.grid.npts), dtype=torch.complex128, device="cuda")
    with pytest.raises(dftu.DftuError) as e:
        h.project(big)                                      # more bands than max_bands
    assert e.value.status == dftu.DFTU_ERR_INVALID_ARG
    with pytest.raises(dftu.DftuError):
        h.set_u(0, float("nan"), 0.1)
    bad = synth.System(s.grid, [synth.Atom((0.0, 0.0, 0.0), 0, 2, 30.0)], s.radials[:1], s.kpts, s.wk, nspin=2)
    with pytest.raises(dftu.DftuError) as e:
        dftu.handle_for_system(bad, 2)                      # sphere beyond two periodic images
    assert e.value.status == dftu.DFTU_ERR_INVALID_ARG


def test_linearly_dependent_orbitals_are_refused():
    """Orbitals that are linearly dependent on their sphere have no S^{-1/2}: the library refuses them
    at set-up, like the oracle, and accepts the independent p shell on the same seven points."""
    from tests.test_oracle_pins import degenerate_shell_systems
    d7, zero, p7 = degenerate_shell_systems()
    for s in (d7, zero):
        with pytest.raises(dftu.DftuError) as e:
            dftu.handle_for_system(s, 2)
        assert e.value.status == dftu.DFTU_ERR_INVALID_ARG
        assert "linearly dependent" in str(e.value)
    h = dftu.handle_for_system(p7, 2)
    idx, img, phi = h.get_sphere(0)
    st = O.setup_atoms(p7)[0]
    assert np.array_equal(idx.astype(np.int64), st["idx"])
    assert rel(phi, st["phi"]) < 1e-13
    h.close()


def test_allocation_failure_is_reported_and_harmless():
    """A handle sized for 2^30 bands asks for 550 GB in its first band-sized buffer, more than the device
    holds: the set-up returns DFTU_ERR_ALLOC (a failed allocation, nothing launched), and the next
    handle on the same device works normally."""
    s = C.periodic_two_atoms()
    with pytest.raises(dftu.DftuError) as e:
        dftu.handle_for_system(s, 1 << 30)
    assert e.value.status == dftu.DFTU_ERR_ALLOC
    nb = 4
    psi = C.states_np(s, nb, seed=3)
    f = np.full((s.nk, 2, nb), 0.5)
    st = O.setup_atoms(s)
    fixed = [(0.3, 0.02), (0.25, 0.01)]
    ref = O.hubbard_pass(s, st, psi, f, fixed_u=fixed)
    out = run_pass(s, psi, f, fixed_u=fixed)
    assert rel(out["psi_out"], ref["psi_out"]) < 1e-12
    assert out["status"] == dftu.DFTU_OK


NBV = 150


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_every_kernel_variant_matches_oracle(dtype):
    """The autotuner may pick any shape variant: each must give the oracle's projections and applied states.
    150 bands fill more than two band groups of every shape (64 bands per group at 4 lanes per band)
    and leave a ragged last group."""
    s, psi, f = _collinear_case("small_oxide", nb=NBV, seed=13)
    st = O.setup_atoms(s)
    fixed = [(0.3, 0.02), (0.25, 0.01), (0.4, 0.05), (0.2, 0.0)]
    ref = O.hubbard_pass(s, st, psi, f, fixed_u=fixed)
    fp64 = dtype == torch.complex128
    lib = dftu.load()
    nvar = lib.dftu_kernel_variants(0)
    for var in range(nvar):
        h = dftu.handle_for_system(s, NBV)
        for I, (u, j) in enumerate(fixed):
            h.set_u(I, u, j)
        h.set_kernel_variant(0 if fp64 else 1, var)
        h.set_kernel_variant(2 if fp64 else 3, var)
        t = torch.from_numpy(psi).cuda().to(dtype)
        h.project(t)
        p = split_p(s, h.projections(NBV))
        for I in range(len(s.atoms)):
            assert rel(p[I], ref["p"][I]) < (1e-12 if fp64 else 2e-6), (var, I)
        h.occupations(torch.from_numpy(f).cuda())
        h.acbn0_uj()
        h.apply(t)
        got = t.to(torch.complex128).cpu().numpy()
        assert rel(got, ref["psi_out"]) < (1e-12 if fp64 else 1e-6), var
        h.close()


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_hubbard_forces_match_oracle(dtype):
    """Sec. IV forces from the projections of the state gradients (fixed U), against the oracle."""
    s = C.periodic_two_atoms()
    st = O.setup_atoms(s)
    nb = 6
    psi, dpsi = synth.analytic_states(s, nb, seed=5)
    f = np.linspace(0.2, 1.0, nb)[None, None, :].repeat(s.nk, 0).repeat(2, 1)
    U = [(0.4, 0.05), (0.3, 0.02)]
    occ = O.occupations(s, O.project(s, st, psi), f)
    V = [np.stack([O.potential(occ[I][0][a], U[I][0] - U[I][1]) for a in range(2)]) for I in range(2)]
    Fref = O.hubbard_forces(s, st, psi, dpsi, f, V)
    h = dftu.handle_for_system(s, nb)
    for I, (u, j) in enumerate(U):
        h.set_u(I, u, j)
    t = torch.from_numpy(psi).cuda().to(dtype)
    g = [torch.from_numpy(d).cuda().to(dtype) for d in dpsi]
    fd = torch.from_numpy(f).cuda()
    h.project(t); h.occupations(fd); h.acbn0_uj()
    F = h.forces(g, fd)
    assert np.max(np.abs(F - Fref)) < (1e-12 if dtype == torch.complex128 else 2e-6) * np.max(np.abs(Fref))
    assert np.max(np.abs(Fref)) > 1e-5


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_access_ceiling_pass_leaves_states_unchanged(dtype):
    """dftu_access_ceiling reads (and in its read-modify-write form writes back) every sphere point of the
    states without changing any value, for collinear and non-collinear layouts."""
    for s, nb in ((C.periodic_two_atoms(), 9), (synth.small_oxide_system(), 70)):
        psi = torch.from_numpy(C.states_np(s, nb, seed=3)).cuda().to(dtype)
        ref = psi.clone()
        h = dftu.handle_for_system(s, nb)
        h.access_ceiling(psi, rmw=False)
        h.access_ceiling(psi, rmw=True)
        torch.cuda.synchronize()
        assert torch.equal(psi, ref)
        assert h.sync_status() == dftu.DFTU_OK
        h.close()
    h = dftu.handle_for_system(C.periodic_two_atoms(), 4)
    assert h.lib.dftu_access_ceiling(h.h, None, 0, 4, 8000, 0, None) == dftu.DFTU_ERR_INVALID_ARG
    h.close()


def _periodic_p_shell():
    g = synth.Grid((18, 18, 18), (0.45, 0.45, 0.45), (0.0, 0.0, 0.0), periodic=True)
    return synth.System(g, [synth.Atom((4.0, 4.1, 3.9), 0, 1, 3.2)], [synth.hydrogenic_radial(2, 1, 2.5)],
                        np.zeros((1, 3)), np.ones(1), nspin=2, name="periodic p shell")


def test_projection_tilings_across_shell_sizes():
    """The complex128 projection's default runs on 1024-point tiles, whose staged orbital rows need more
    shared memory for larger shells. Systems with different largest shells projected in turn in one
    process (d, p only, p + f, d again) must each launch with their own size; the p + f system, whose
    CTAs no longer fit two per SM, falls back to the 512-point tiling. Each against the oracle."""
    nb = 40
    for make in (synth.small_oxide_system, _periodic_p_shell, isolated_aniso, synth.small_oxide_system):
        s = make()
        psi = C.states_np(s, nb, seed=21)
        ref = O.project(s, O.setup_atoms(s), psi)
        h = dftu.handle_for_system(s, nb)
        h.project(torch.from_numpy(psi).cuda())
        p = split_p(s, h.projections(nb))
        for I in range(len(s.atoms)):
            assert rel(p[I], ref[I]) < 1e-12, (s.name, I)
        assert h.sync_status() == dftu.DFTU_OK
        h.close()
