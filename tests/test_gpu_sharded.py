"""Sharded occupation sums through the C ABI: handles that each hold a disjoint part of the (k, band) set
(one k-point each with its weight in the full set, or one band range each) export their partial rho and
Pbar (Eqs. 4, 8), the sums are added as an allreduce would, written back, and dftu_acbn0_uj then gives every
handle the U, J, E_U and n of the single handle that holds everything; each handle's apply of its own
states matches the single handle's apply of the same states.  Both "ranks" run on one GPU, one after the
other (no kernel waits for another)."""
import numpy as np
import pytest
import torch

from paper_1711_08935_gb300 import dftu
from paper_1711_08935_gb300.synth import System
from tests import _cases

pytestmark = pytest.mark.gpu


def _full(s, psi, f, nb, dtype):
    h = dftu.handle_for_system(s, nb)
    coul = [h.coulomb_integrals(sp) for sp in range(len(s.radials))]
    x = torch.from_numpy(psi).cuda().to(dtype)
    h.project(x)
    h.occupations(torch.from_numpy(f).cuda())
    h.acbn0_uj()
    r = h.results()
    h.apply(x)
    out = x.to(torch.complex128).cpu().numpy()
    h.close()
    return coul, r, out


def _shard_run(parts, coul, dtype):
    """parts: list of (System, psi part, f part).  Returns per-part (results, applied states)."""
    hs, xs = [], []
    for sub, ps, fs in parts:
        h = dftu.handle_for_system(sub, ps.shape[2])
        for sp, V in enumerate(coul):
            h.set_coulomb(sp, V)
        x = torch.from_numpy(np.ascontiguousarray(ps)).cuda().to(dtype)
        h.project(x)
        h.occupations(torch.from_numpy(np.ascontiguousarray(fs)).cuda())
        hs.append(h)
        xs.append(x)
    total = None
    for h in hs:
        part = h.occupation_sums()
        total = part.clone() if total is None else total + part
    out = []
    for h, x in zip(hs, xs):
        h.set_occupation_sums(total)
        h.acbn0_uj()
        r = h.results()
        h.apply(x)
        out.append((r, x.to(torch.complex128).cpu().numpy()))
        h.close()
    return out


def _check(r, ref, tol_n):
    for a, b in zip(r["n"], ref["n"]):
        assert np.max(np.abs(a - b)) <= tol_n * max(1e-300, np.max(np.abs(b)))
    assert np.max(np.abs(r["U"] - ref["U"])) * dftu.HARTREE_EV < 1e-10
    assert np.max(np.abs(r["J"] - ref["J"])) * dftu.HARTREE_EV < 1e-10
    assert abs(r["EU"] - ref["EU"]) * dftu.HARTREE_EV < 1e-10


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_k_point_shards_with_summed_occupations_match_one_handle(dtype):
    s = _cases.periodic_two_atoms()
    nb = 10
    psi = _cases.states_np(s, nb, seed=41)
    f = np.random.default_rng(6).uniform(0.0, 1.0, (s.nk, 2, nb))
    coul, ref, ref_out = _full(s, psi, f, nb, dtype)
    wk = np.asarray(s.wk)
    parts = [(System(s.grid, s.atoms, s.radials, s.kpts[k:k + 1], wk[k:k + 1], nspin=s.nspin), psi[k:k + 1], f[k:k + 1])
             for k in range(s.nk)]
    tol_psi = 1e-12 if dtype == torch.complex128 else 1e-6
    for k, (r, out) in enumerate(_shard_run(parts, coul, dtype)):
        _check(r, ref, 1e-12)
        assert np.max(np.abs(out - ref_out[k:k + 1])) <= tol_psi * np.max(np.abs(ref_out))


def test_band_shards_with_summed_occupations_match_one_handle():
    s = _cases.periodic_two_atoms()
    nb = 12
    psi = _cases.states_np(s, nb, seed=43)
    f = np.random.default_rng(7).uniform(0.0, 1.0, (s.nk, 2, nb))
    coul, ref, ref_out = _full(s, psi, f, nb, torch.complex128)
    cuts = [(0, 5), (5, nb)]                          # uneven band ranges
    parts = [(s, psi[:, :, a:b], f[:, :, a:b]) for a, b in cuts]
    for (a, b), (r, out) in zip(cuts, _shard_run(parts, coul, torch.complex128)):
        _check(r, ref, 1e-12)
        assert np.max(np.abs(out - ref_out[:, :, a:b])) <= 1e-12 * np.max(np.abs(ref_out))


def test_occupation_sums_round_trip_and_bad_sizes():
    s = _cases.periodic_two_atoms()
    nb = 4
    h = dftu.handle_for_system(s, nb)
    n = int(h.lib.dftu_occupation_elems(h.h))
    MT2 = sum((2 * a.l + 1) ** 2 for a in s.atoms)
    assert n == 2 * 2 * 2 * MT2                       # (rho, Pbar) x 2 spins x complex
    x = torch.from_numpy(_cases.states_np(s, nb, seed=2)).cuda()
    h.project(x)
    h.occupations(torch.full((s.nk, 2, nb), 0.5, dtype=torch.float64, device="cuda"))
    a = h.occupation_sums()
    h.set_occupation_sums(2.0 * a)
    assert torch.equal(h.occupation_sums(), 2.0 * a)
    with pytest.raises(ValueError):
        h.set_occupation_sums(a[:-1].contiguous())
    h.close()
