"""Sharding the Hubbard pass over ranks (host logic, no GPU): the occupation sums of Eqs. (4) and (8) are
additive over disjoint parts of the (k, band) set, so ranks that each hold a part -- whole k-points with
their weights in the full set, or a band range of a k-point -- can form partial rho and Pbar, add them
with one allreduce, and obtain the U, J and E_U of the whole set (Eqs. 10, 11, 3).  Two gloo ranks on the
CPU, each running the oracle on its own part, against the oracle on everything in one process."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

ATOL_U_EV = 1e-10


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _problem():
    from tests import _cases
    s = _cases.periodic_two_atoms()                    # 2 k-points (weights 1/2), collinear spin
    nb = 8
    psi = _cases.states_np(s, nb, seed=31)
    f = np.random.default_rng(4).uniform(0.0, 1.0, (s.nk, 2, nb))
    rng = np.random.default_rng(9)
    coul = []
    for sp in range(len(s.radials)):
        M = 2 * [a.l for a in s.atoms if a.species == sp][0] + 1
        A = rng.standard_normal((M * M, M * M))
        W = (A @ A.T) / (M * M)                        # positive definite pair matrix
        V = W.reshape(M, M, M, M)
        V = 0.5 * (V + V.transpose(1, 0, 2, 3))         # (mm'|..) = (m'm|..)
        V = 0.5 * (V + V.transpose(0, 1, 3, 2))
        V = 0.5 * (V + V.transpose(2, 3, 0, 1))
        coul.append(V)
    return s, nb, psi, f, coul


def _parts(s, psi, f, rank):
    """Rank 0: k-point 0 (all bands) and the first half of k-point 1's bands; rank 1: the rest."""
    from paper_1711_08935_gb300.synth import System
    nb = psi.shape[2]
    h = nb // 2
    spans = [(0, 0, nb), (1, 0, h)] if rank == 0 else [(1, h, nb)]
    out = []
    for k, b0, b1 in spans:
        sub = System(s.grid, s.atoms, s.radials, s.kpts[k:k + 1], np.asarray(s.wk)[k:k + 1], nspin=s.nspin)
        out.append((sub, psi[k:k + 1, :, b0:b1], f[k:k + 1, :, b0:b1]))
    return out


def _partial_sums(rank):
    from oracle import dftu_oracle as O
    s, nb, psi, f, coul = _problem()
    st = O.setup_atoms(s)
    tot = None
    for sub, ps, fs in _parts(s, psi, f, rank):
        occ = O.occupations(sub, O.project(sub, st, ps), fs)
        flat = np.concatenate([np.concatenate([r.ravel(), P.ravel()]) for r, P in occ])
        tot = flat if tot is None else tot + flat
    return tot


def _finish(flat):
    """U, J and E_U of every atom from summed (rho, Pbar)."""
    from oracle import dftu_oracle as O
    s, nb, psi, f, coul = _problem()
    U, J, E, o = [], [], 0.0, 0
    for at in s.atoms:
        M = 2 * at.l + 1
        n = 2 * M * M
        rho = flat[o:o + n].reshape(2, M, M)
        Pb = flat[o + n:o + 2 * n].reshape(2, M, M)
        o += 2 * n
        u, j, _ = O.acbn0_uj(rho, Pb, coul[at.species], 2)
        U.append(u)
        J.append(j)
        E += O.hubbard_energy(rho, u - j, 2)
    return np.array(U), np.array(J), E


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    part = _partial_sums(rank)
    t = torch.from_numpy(np.stack([part.real, part.imag]))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    total = t[0].numpy() + 1j * t[1].numpy()
    U, J, E = _finish(total)
    out[rank] = (total, U, J, E)
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_occupations_over_two_gloo_ranks_equal_the_single_process_pass():
    from oracle import dftu_oracle as O
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    s, nb, psi, f, coul = _problem()
    st = O.setup_atoms(s)
    ref = O.hubbard_pass(s, st, psi, f, coulomb=coul)
    ref_flat = np.concatenate([np.concatenate([r.ravel(), P.ravel()]) for r, P in ref["occ"]])
    for r in range(2):
        total, U, J, E = out[r]
        assert np.max(np.abs(total - ref_flat)) <= 1e-13 * np.max(np.abs(ref_flat))
        assert np.max(np.abs(U - ref["U"])) * O.HARTREE_EV < ATOL_U_EV
        assert np.max(np.abs(J - ref["J"])) * O.HARTREE_EV < ATOL_U_EV
        assert abs(E - ref["E"]) * O.HARTREE_EV < ATOL_U_EV
    # each rank's share alone is not the answer (the exchange step matters)
    half = _partial_sums(1)
    assert np.max(np.abs(half - ref_flat)) > 1e-3 * np.max(np.abs(ref_flat))
