"""Helpers for the GPU parity tests: run the library on a System and collect every output."""
import numpy as np
import torch

from paper_1711_08935_gb300 import dftu


def run_pass(system, psi_np, f_np, coulomb=None, fixed_u=None, dtype=torch.complex128, mode=dftu.F64_PAIR,
             coef=None, max_bands=None, gpu_coulomb=False):
    """project -> occupations -> U/J -> apply through the C ABI; returns a dict of host arrays."""
    nb = psi_np.shape[1] if system.noncollinear else psi_np.shape[2]
    h = dftu.handle_for_system(system, max_bands or nb)
    h.set_f64_mode(mode)
    dev = torch.device("cuda:0")
    psi = torch.from_numpy(np.ascontiguousarray(psi_np)).to(dev).to(dtype)
    f = torch.from_numpy(np.ascontiguousarray(f_np, dtype=np.float64)).to(dev)
    for sp in range(len(system.radials)):
        if gpu_coulomb:
            h.coulomb_integrals(sp)
        elif coulomb is not None:
            h.set_coulomb(sp, coulomb[sp])
    if fixed_u is not None:
        for I, (u, j) in enumerate(fixed_u):
            h.set_u(I, u, j)
    h.project(psi)
    p = h.projections(nb)
    h.occupations(f)
    h.acbn0_uj()
    res = h.results()
    Pb, Nb = h.renormalized(nb)
    c = None
    if coef is not None:
        c = torch.tensor([coef], dtype=torch.complex128, device=dev)
    h.apply(psi, c)
    torch.cuda.synchronize()
    status = h.sync_status()
    out = dict(p=p, Pbar=Pb, Nbar=Nb, psi_out=psi.to(torch.complex128).cpu().numpy(), status=status, handle=h, **res)
    return out


def split_p(system, p_flat):
    """[rows][nb][MT] -> per-atom arrays shaped like the oracle's projections."""
    out, o = [], 0
    nk = system.nk
    for at in system.atoms:
        M = 2 * at.l + 1
        blk = p_flat[:, :, o:o + M]
        if system.noncollinear:
            nb = blk.shape[1]
            out.append(blk.reshape(nk, 2, nb, M).transpose(0, 2, 1, 3))
        else:
            out.append(blk.reshape(nk, -1, blk.shape[1], M))
        o += M
    return out
