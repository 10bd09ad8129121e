"""Batches of independent molecules (persistent launches over all members) against the same members
run one by one through the single-system calls (bitwise: same arithmetic, same order, same tiling), and
every member against the CPU oracle."""
import numpy as np
import pytest
import torch

from oracle import dftu_oracle as O
from paper_1711_08935_gb300 import dftu, synth

pytestmark = pytest.mark.gpu


def _members(dtype):
    systems = synth.molecule_systems(5, seed=7, edge=(20, 28), natoms=(1, 3), radius=(2.0, 2.6), nstates=(3, 11))
    dev = torch.device("cuda:0")
    out = []
    for i, s in enumerate(systems):
        nb = synth.bands_of(s)
        psi = synth.make_states(s, nb, seed=100 + i, device="cpu").to(dtype)
        f = torch.from_numpy(synth.fermi_occupations(1, 2, nb, kT=0.05, e0=-0.2, de=0.04)).to(dev)
        out.append((s, nb, psi, f))
    return out


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_batch_matches_single_system_calls_bitwise(dtype):
    dev = torch.device("cuda:0")
    mem = _members(dtype)
    hs_a, hs_b, psis_a, psis_b, fs = [], [], [], [], []
    for s, nb, psi, f in mem:
        for hs, ps in ((hs_a, psis_a), (hs_b, psis_b)):
            h = dftu.handle_for_system(s, nb)
            h.coulomb_integrals(0)
            hs.append(h)
            ps.append(psi.to(dev).clone())
        fs.append(f)
    for h, p, f in zip(hs_a, psis_a, fs):                 # one by one
        # batched launches use the 512-point tiling; complex128 projection variant 1 is the batched
        # default shape on that tiling (the single-system default runs on 1024-point tiles, which sums
        # the same products in another order)
        h.set_kernel_variant(0, 1)
        h.project(p); h.occupations(f); h.acbn0_uj(); h.apply(p)
    batch = dftu.Batch(hs_b)
    batch.bind(psis_b, fs)
    batch.project(); batch.occupations(); batch.acbn0_uj(); batch.apply()
    torch.cuda.synchronize()
    for i, (ha, hb) in enumerate(zip(hs_a, hs_b)):
        ra, rb = ha.results(), hb.results()
        for na, nb_ in zip(ra["n"], rb["n"]):
            assert np.array_equal(na, nb_), i
        assert np.array_equal(ra["U"], rb["U"]) and np.array_equal(ra["J"], rb["J"]) and ra["EU"] == rb["EU"]
        assert torch.equal(psis_a[i], psis_b[i]), i
        assert hb.sync_status() in (dftu.DFTU_OK, dftu.DFTU_ERR_ZERO_DENOM)
    batch.close()


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_every_batch_member_matches_oracle(dtype):
    """Every member of a batch against the oracle on the states the GPU holds (complex64 states are
    compared with the oracle run on their FP64 promotion): n, U, J and the applied states, at the
    tolerances of the single-system tests."""
    dev = torch.device("cuda:0")
    mem = _members(dtype)
    hs, ps, fs, refs = [], [], [], []
    for s, nb, psi, f in mem:
        st = O.setup_atoms(s)
        coul = [O.coulomb_integrals(s.grid, s.atoms[0], st[0])]
        h = dftu.handle_for_system(s, nb)
        h.set_coulomb(0, coul[0])
        hs.append(h)
        ps.append(psi.to(dev).clone())
        fs.append(f)
        seen = psi.to(torch.complex128).numpy()
        refs.append(O.hubbard_pass(s, st, seen, f.cpu().numpy(), coulomb=coul))
    batch = dftu.Batch(hs)
    batch.bind(ps, fs)
    batch.project(); batch.occupations(); batch.acbn0_uj(); batch.apply()
    torch.cuda.synchronize()
    fp64 = dtype == torch.complex128
    tol_n, tol_uj, tol_psi = (1e-12, 1e-10, 1e-12) if fp64 else (1e-6, 1e-4, 1e-6)
    for i, ((s, nb, psi, f), h, ref) in enumerate(zip(mem, hs, refs)):
        r = h.results()
        for I in range(len(s.atoms)):
            nref = O.paper_n(ref["occ"][I][0])
            assert np.max(np.abs(r["n"][I] - nref)) < tol_n * max(1.0, np.max(np.abs(nref))), (i, I)
        assert np.max(np.abs(r["U"] - ref["U"])) * O.HARTREE_EV < tol_uj, i
        assert np.max(np.abs(r["J"] - ref["J"])) * O.HARTREE_EV < tol_uj, i
        got = ps[i].to(torch.complex128).cpu().numpy()
        assert np.max(np.abs(got - ref["psi_out"])) < tol_psi * np.max(np.abs(ref["psi_out"])), i
    batch.close()
    for h in hs:
        h.close()


def test_batch_refuses_members_it_cannot_run_uniformly():
    """The batched kernels run one FP64 mode and no gauge phases for all members: a member with a
    vector potential or another FP64 mode is refused (DFTU_ERR_INVALID_ARG), as is an apply before bind."""
    dev = torch.device("cuda:0")
    mem = _members(torch.complex128)[:2]
    hs, ps, fs = [], [], []
    for s, nb, psi, f in mem:
        h = dftu.handle_for_system(s, nb)
        h.coulomb_integrals(0)
        hs.append(h)
        ps.append(psi.to(dev).clone())
        fs.append(f)
    batch = dftu.Batch(hs)
    with pytest.raises(dftu.DftuError) as e:
        batch.apply()
    assert e.value.status == dftu.DFTU_ERR_NOT_READY
    batch.bind(ps, fs)
    hs[1].set_vector_potential(torch.tensor([0.1, 0.0, 0.0], dtype=torch.float64, device=dev))
    with pytest.raises(dftu.DftuError) as e:
        batch.project()
    assert e.value.status == dftu.DFTU_ERR_INVALID_ARG
    hs[1].set_vector_potential(None)
    hs[1].set_f64_mode(dftu.F64_NATIVE)
    with pytest.raises(dftu.DftuError) as e:
        batch.project()
    assert e.value.status == dftu.DFTU_ERR_INVALID_ARG
    hs[1].set_f64_mode(dftu.F64_PAIR)
    batch.project(); batch.occupations(); batch.acbn0_uj(); batch.apply()
    torch.cuda.synchronize()
    batch.close()
    for h in hs:
        h.close()
