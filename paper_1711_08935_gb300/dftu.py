"""Thin Python binding of libdftu.so (C ABI in include/dftu.h).

Argument marshalling only: every step of the Hubbard-projector path runs in the library's CUDA
kernels.  Device arrays are torch tensors (PyTorch supplies memory and streams); host-side inputs
and outputs are numpy arrays.  The library must have been built (paper_1711_08935_gb300.build_lib);
importing this module without it raises, there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libdftu.so")

DFTU_OK, DFTU_ERR_INVALID_ARG, DFTU_ERR_NOT_READY, DFTU_ERR_ALLOC, DFTU_ERR_CUDA, DFTU_ERR_NONFINITE, \
    DFTU_ERR_ZERO_DENOM, DFTU_ERR_TIMEOUT = range(8)
STATUS_NAMES = ["OK", "INVALID_ARG", "NOT_READY", "ALLOC", "CUDA", "NONFINITE", "ZERO_DENOM", "TIMEOUT"]
C128, C64 = 0, 1
COLLINEAR, UNPOLARIZED, NONCOLLINEAR = 0, 1, 2
F64_PAIR, F64_NATIVE = 0, 1
HARTREE_EV = 27.211386245988

# Every symbol include/dftu.h declares (checked by the CPU tests).
EXPORTED = ["dftu_create", "dftu_setup_atoms", "dftu_get_sphere", "dftu_coulomb_integrals", "dftu_set_coulomb",
            "dftu_set_u", "dftu_set_f64_mode", "dftu_project", "dftu_occupations", "dftu_acbn0_uj", "dftu_apply",
            "dftu_get_results", "dftu_get_renormalized", "dftu_get_projections", "dftu_total_orbitals",
            "dftu_atom_points", "dftu_sync_status", "dftu_last_error", "dftu_destroy",
            "dftu_set_kernel_variant", "dftu_kernel_variants", "dftu_project_sphere_noalloc",
            "dftu_taylor_step", "dftu_taylor_steps", "dftu_batch_create", "dftu_batch_bind", "dftu_batch_project",
            "dftu_batch_occupations", "dftu_batch_acbn0_uj", "dftu_batch_apply", "dftu_batch_last_error",
            "dftu_batch_destroy", "dftu_forces", "dftu_radius_cell", "dftu_radius_threshold",
            "dftu_set_vector_potential", "dftu_hubbard_current", "dftu_fll_energy", "dftu_occupation_elems",
            "dftu_export_occupations", "dftu_import_occupations", "dftu_access_ceiling"]


class DftuGrid(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("h", C.c_double * 3), ("origin", C.c_double * 3), ("periodic", C.c_int)]


class DftuAtom(C.Structure):
    _fields_ = [("pos", C.c_double * 3), ("species", C.c_int), ("l", C.c_int), ("radius", C.c_double)]


class DftuRadial(C.Structure):
    _fields_ = [("nr", C.c_int), ("dr", C.c_double), ("R", C.POINTER(C.c_double))]


class DftuError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"dftu {STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


_lib: Optional[C.CDLL] = None


def load() -> C.CDLL:
    """Load libdftu.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1711_08935_gb300.build_lib`")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, d, dp, ip = C.c_void_p, C.c_int, C.c_int64, C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_int)
    sig = {
        "dftu_create": [C.POINTER(vp), C.POINTER(DftuGrid), i32, dp, dp, i32, i32, i32],
        "dftu_setup_atoms": [vp, i32, C.POINTER(DftuAtom), i32, C.POINTER(DftuRadial), ip],
        "dftu_get_sphere": [vp, i32, C.POINTER(C.c_int32), C.POINTER(C.c_int32), dp],
        "dftu_coulomb_integrals": [vp, i32, dp],
        "dftu_set_coulomb": [vp, i32, dp],
        "dftu_set_u": [vp, i32, d, d],
        "dftu_set_f64_mode": [vp, i32],
        "dftu_project": [vp, vp, i32, i32, i64, vp],
        "dftu_occupations": [vp, vp, vp],
        "dftu_acbn0_uj": [vp, vp],
        "dftu_apply": [vp, vp, i32, i32, i64, vp, i32, vp],
        "dftu_taylor_step": [vp, vp, vp, i32, i32, i64, vp, d, i32, vp],
        "dftu_taylor_steps": [vp, vp, i32, i32, i64, vp, d, i32, i32, vp],
        "dftu_batch_create": [C.POINTER(vp), i32, C.POINTER(vp)],
        "dftu_batch_bind": [vp, C.POINTER(vp), i32, C.POINTER(C.c_int), C.POINTER(C.c_int64), C.POINTER(vp)],
        "dftu_batch_project": [vp, vp],
        "dftu_batch_occupations": [vp, vp],
        "dftu_batch_acbn0_uj": [vp, vp],
        "dftu_batch_apply": [vp, vp, i32, vp],
        "dftu_batch_last_error": [vp],
        "dftu_batch_destroy": [vp],
        "dftu_forces": [vp, C.POINTER(vp), i32, i32, i64, vp, dp, vp],
        "dftu_set_vector_potential": [vp, vp, vp],
        "dftu_hubbard_current": [vp, vp, i32, i32, i64, vp, dp, dp, vp],
        "dftu_fll_energy": [vp, dp, dp, vp],
        "dftu_radius_cell": [C.POINTER(DftuGrid)],
        "dftu_radius_threshold": [C.POINTER(DftuRadial), d],
        "dftu_get_results": [vp, dp, dp, dp, dp, dp, vp],
        "dftu_get_renormalized": [vp, dp, dp, vp],
        "dftu_get_projections": [vp, dp, vp],
        "dftu_total_orbitals": [vp],
        "dftu_atom_points": [vp, i32],
        "dftu_sync_status": [vp],
        "dftu_last_error": [vp],
        "dftu_destroy": [vp],
        "dftu_set_kernel_variant": [vp, i32, i32],
        "dftu_kernel_variants": [i32],
        "dftu_project_sphere_noalloc": [vp, i32, i32, i64, vp, vp, vp, i32, i32, d, vp, vp],
        "dftu_occupation_elems": [vp],
        "dftu_export_occupations": [vp, vp, vp],
        "dftu_import_occupations": [vp, vp, vp],
        "dftu_access_ceiling": [vp, vp, i32, i32, i64, i32, vp],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = C.c_int
    L.dftu_last_error.restype = C.c_char_p
    L.dftu_occupation_elems.restype = C.c_int64
    L.dftu_destroy.restype = None
    L.dftu_batch_last_error.restype = C.c_char_p
    L.dftu_radius_cell.restype = C.c_double
    L.dftu_radius_threshold.restype = C.c_double
    L.dftu_batch_destroy.restype = None
    _lib = L
    return L


def _dp(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _stream_ptr(stream, device) -> C.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream(device)
    return C.c_void_p(s.cuda_stream)


class Handle:
    """One DFT+U context on one GPU: geometry, orbitals, work buffers.  Calls map 1:1 to the C ABI."""

    def __init__(self, grid, kpts, wk, spin: int, max_bands: int, device: int = 0):
        self.lib = load()
        self.device = device
        self.spin = spin
        self.nk = len(kpts)
        self.ns = 1 if spin == UNPOLARIZED else 2
        self.max_bands = max_bands
        self.npts_grid = int(np.prod(grid.n))
        g = DftuGrid((C.c_int * 3)(*grid.n), (C.c_double * 3)(*grid.h), (C.c_double * 3)(*grid.origin),
                     1 if grid.periodic else 0)
        kv = np.ascontiguousarray(np.asarray(kpts, dtype=np.float64).reshape(-1, 3))
        w = np.ascontiguousarray(np.asarray(wk, dtype=np.float64))
        h = C.c_void_p()
        self._check(self.lib.dftu_create(C.byref(h), C.byref(g), self.nk, _dp(kv), _dp(w), spin, max_bands, device), None)
        self.h = h
        self.M = []
        self.species = []
        self.natoms = 0
        self._variants = [0, 0, 0, 0]

    # ------------------------------------------------------------------ plumbing
    def _check(self, status: int, h=-1):
        if status != DFTU_OK:
            hh = self.h if h == -1 else h
            msg = self.lib.dftu_last_error(hh).decode() if hh else ""
            raise DftuError(status, msg)

    def close(self):
        if getattr(self, "h", None):
            self.lib.dftu_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ set-up
    def setup_atoms(self, atoms: Sequence, radials: Sequence) -> np.ndarray:
        arr = (DftuAtom * len(atoms))()
        for i, a in enumerate(atoms):
            arr[i] = DftuAtom((C.c_double * 3)(*a.pos), a.species, a.l, a.radius)
        self._radial_keep = [np.ascontiguousarray(r.R, dtype=np.float64) for r in radials]
        rr = (DftuRadial * len(radials))()
        for i, r in enumerate(radials):
            rr[i] = DftuRadial(len(self._radial_keep[i]), r.dr, _dp(self._radial_keep[i]))
        npts = (C.c_int * len(atoms))()
        self._check(self.lib.dftu_setup_atoms(self.h, len(atoms), arr, len(radials), rr, npts))
        self.M = [2 * a.l + 1 for a in atoms]
        self.species = [a.species for a in atoms]
        self.natoms = len(atoms)
        return np.array(list(npts))

    def get_sphere(self, atom: int):
        n = self.lib.dftu_atom_points(self.h, atom)
        idx = np.zeros(n, dtype=np.int32)
        img = np.zeros((n, 3), dtype=np.int32)
        phi = np.zeros((n, self.M[atom]), dtype=np.float64)
        self._check(self.lib.dftu_get_sphere(self.h, atom, idx.ctypes.data_as(C.POINTER(C.c_int32)),
                                             img.ctypes.data_as(C.POINTER(C.c_int32)), _dp(phi)))
        return idx, img, phi

    def coulomb_integrals(self, species: int) -> np.ndarray:
        M = self.M[self.species.index(species)]
        V = np.zeros((M, M, M, M))
        self._check(self.lib.dftu_coulomb_integrals(self.h, species, _dp(V)))
        return V

    def set_coulomb(self, species: int, V: np.ndarray):
        self._check(self.lib.dftu_set_coulomb(self.h, species, _dp(np.ascontiguousarray(V, dtype=np.float64))))

    def set_u(self, atom: int, U: float, J: float):
        self._check(self.lib.dftu_set_u(self.h, atom, float(U), float(J)))

    def set_f64_mode(self, mode: int):
        self._check(self.lib.dftu_set_f64_mode(self.h, mode))

    def set_kernel_variant(self, which: int, variant: int):
        self._check(self.lib.dftu_set_kernel_variant(self.h, which, variant))
        self._variants[which] = variant

    def variants_now(self):
        """Kernel variants in use: (project c128, project c64, apply c128, apply c64)."""
        return tuple(self._variants)

    # ------------------------------------------------------------------ hot path
    def _psi_args(self, psi: torch.Tensor):
        if psi.dtype == torch.complex128:
            prec = C128
        elif psi.dtype == torch.complex64:
            prec = C64
        else:
            raise TypeError("psi must be complex128 or complex64")
        if not psi.is_contiguous() or not (psi.is_cuda or psi.is_pinned()):
            raise ValueError("psi must be a contiguous CUDA tensor or a contiguous pinned host tensor")
        if self.spin == NONCOLLINEAR:
            if psi.dim() != 4 or psi.shape[0] != self.nk or psi.shape[2] != 2:
                raise ValueError("non-collinear psi must be [nk][nbands][2][npts]")
            nb = psi.shape[1]
        else:
            if psi.dim() != 4 or psi.shape[0] != self.nk or psi.shape[1] != self.ns:
                raise ValueError("psi must be [nk][nspin][nbands][npts]")
            nb = psi.shape[2]
        if psi.shape[3] < self.npts_grid:
            raise ValueError("psi's last dimension is shorter than the grid")
        return prec, nb, psi.shape[3]

    @staticmethod
    def _f_arg(f: torch.Tensor) -> C.c_void_p:
        if f.dtype != torch.float64 or not f.is_contiguous() or not (f.is_cuda or f.is_pinned()):
            raise ValueError("f must be a contiguous float64 CUDA tensor or pinned host tensor")
        return C.c_void_p(f.data_ptr())

    def project(self, psi: torch.Tensor, stream=None):
        prec, nb, ld = self._psi_args(psi)
        self._check(self.lib.dftu_project(self.h, C.c_void_p(psi.data_ptr()), prec, nb, ld, _stream_ptr(stream, self.device)))

    def occupations(self, f: torch.Tensor, stream=None):
        self._check(self.lib.dftu_occupations(self.h, self._f_arg(f), _stream_ptr(stream, self.device)))

    def access_ceiling(self, psi: torch.Tensor, rmw: bool = False, stream=None):
        """One pass of the access pattern alone (dftu_access_ceiling): read every sphere point of psi, or
        read and write each back unchanged; time it to bound the projection (read) and the apply (rmw)."""
        prec, nb, ld = self._psi_args(psi)
        self._check(self.lib.dftu_access_ceiling(self.h, C.c_void_p(psi.data_ptr()), prec, nb, ld, 1 if rmw else 0,
                                                 _stream_ptr(stream, self.device)))

    def occupation_sums(self, out: torch.Tensor = None, stream=None) -> torch.Tensor:
        """This handle's occupation sums (rho, Pbar) of the last occupations, as a float64 tensor on the
        handle's device (written into `out` when given) -- the part a rank adds up with the others."""
        n = int(self.lib.dftu_occupation_elems(self.h))
        if out is None:
            out = torch.empty(n, dtype=torch.float64, device=torch.device("cuda", self.device))
        if out.dtype != torch.float64 or out.numel() != n or not out.is_contiguous():
            raise ValueError(f"out must be a contiguous float64 tensor of {n} elements")
        self._check(self.lib.dftu_export_occupations(self.h, C.c_void_p(out.data_ptr()), _stream_ptr(stream, self.device)))
        return out

    def set_occupation_sums(self, sums: torch.Tensor, stream=None):
        """Overwrite the occupation sums (e.g. with their total over ranks) before acbn0_uj."""
        n = int(self.lib.dftu_occupation_elems(self.h))
        if sums.dtype != torch.float64 or sums.numel() != n or not sums.is_contiguous():
            raise ValueError(f"sums must be a contiguous float64 tensor of {n} elements")
        self._check(self.lib.dftu_import_occupations(self.h, C.c_void_p(sums.data_ptr()), _stream_ptr(stream, self.device)))

    def acbn0_uj(self, stream=None):
        self._check(self.lib.dftu_acbn0_uj(self.h, _stream_ptr(stream, self.device)))

    def apply(self, psi: torch.Tensor, coef: Optional[torch.Tensor] = None, accumulate: bool = True, stream=None):
        prec, nb, ld = self._psi_args(psi)
        cp = None
        if coef is not None:
            if coef.dtype != torch.complex128 or not (coef.is_cuda or coef.is_pinned()):
                raise ValueError("coef must be a complex128 CUDA tensor or pinned host tensor")
            cp = C.c_void_p(coef.data_ptr())
        self._check(self.lib.dftu_apply(self.h, C.c_void_p(psi.data_ptr()), prec, nb, ld, cp, 1 if accumulate else 0,
                                        _stream_ptr(stream, self.device)))

    def forces(self, dpsi: Sequence[torch.Tensor], f: torch.Tensor, stream=None) -> np.ndarray:
        """Hubbard forces [natoms][3] (Hartree/bohr) from the gradients of the last projected states."""
        prec, nb, ld = self._psi_args(dpsi[0])
        for d in dpsi:
            if d.shape != dpsi[0].shape or d.dtype != dpsi[0].dtype or not d.is_contiguous():
                raise ValueError("the three gradients must share shape, dtype and layout")
        arr = (C.c_void_p * 3)(*[d.data_ptr() for d in dpsi])
        F = np.zeros((self.natoms, 3))
        self._check(self.lib.dftu_forces(self.h, arr, prec, nb, ld, self._f_arg(f), _dp(F),
                                         _stream_ptr(stream, self.device)))
        return F

    def set_vector_potential(self, A: Optional[torch.Tensor], stream=None):
        """Uniform vector potential of the gauge-invariant operator (Sec. V): a float64 tensor of 3 on the GPU
        or in pinned host memory, or None."""
        if A is not None and (A.dtype != torch.float64 or not (A.is_cuda or A.is_pinned()) or A.numel() != 3
                              or not A.is_contiguous()):
            raise ValueError("A must be a contiguous float64 CUDA or pinned host tensor of 3 elements")
        self._A = A   # keep it alive: the phase kernel reads it when it runs
        ptr = C.c_void_p(A.data_ptr()) if A is not None else None
        self._check(self.lib.dftu_set_vector_potential(self.h, ptr, _stream_ptr(stream, self.device)))

    def hubbard_current(self, psi: torch.Tensor, f: torch.Tensor, per_atom: bool = False, stream=None):
        """Hubbard current J [3] (Sec. V, Eq. 17) of the last projected states; with per_atom also [natoms][3]."""
        prec, nb, ld = self._psi_args(psi)
        J = np.zeros(3)
        Jat = np.zeros((self.natoms, 3))
        self._check(self.lib.dftu_hubbard_current(self.h, C.c_void_p(psi.data_ptr()), prec, nb, ld, self._f_arg(f),
                                                  _dp(J), _dp(Jat), _stream_ptr(stream, self.device)))
        return (J, Jat) if per_atom else J

    def fll_energy(self, stream=None):
        """(E_ee, E_DC) per atom (Hartree), App. A Eqs. (A1) and (A3), with the current U and J."""
        ee, dc = np.zeros(self.natoms), np.zeros(self.natoms)
        self._check(self.lib.dftu_fll_energy(self.h, _dp(ee), _dp(dc), _stream_ptr(stream, self.device)))
        return ee, dc

    def taylor_step(self, psi: torch.Tensor, work: Optional[torch.Tensor], f: torch.Tensor, dt: float, order: int = 4,
                    stream=None):
        """One real-time step (dftu_taylor_step); `work` is not needed and may be None."""
        prec, nb, ld = self._psi_args(psi)
        if work is not None and (work.shape != psi.shape or work.dtype != psi.dtype or not work.is_contiguous()):
            raise ValueError("work must match psi")
        wp = C.c_void_p(work.data_ptr()) if work is not None else None
        self._check(self.lib.dftu_taylor_step(self.h, C.c_void_p(psi.data_ptr()), wp, prec, nb, ld,
                                              self._f_arg(f), float(dt), int(order), _stream_ptr(stream, self.device)))

    def taylor_steps(self, psi: torch.Tensor, f: torch.Tensor, dt: float, nsteps: int, order: int = 4, stream=None):
        """nsteps real-time steps (dftu_taylor_steps): for complex64 collinear states the scatter of each
        step also gathers the updated states for the next one."""
        prec, nb, ld = self._psi_args(psi)
        self._check(self.lib.dftu_taylor_steps(self.h, C.c_void_p(psi.data_ptr()), prec, nb, ld, self._f_arg(f),
                                               float(dt), int(order), int(nsteps), _stream_ptr(stream, self.device)))

    # ------------------------------------------------------------------ results
    def _mat_sizes(self):
        if self.spin == NONCOLLINEAR:
            return [(1, 2 * M) for M in self.M]
        return [(self.ns, M) for M in self.M]

    def _unpack_mats(self, flat: np.ndarray):
        out, o = [], 0
        for nb, D in self._mat_sizes():
            n = nb * D * D
            out.append((flat[2 * o:2 * (o + n):2] + 1j * flat[2 * o + 1:2 * (o + n):2]).reshape(nb, D, D))
            o += n
        return out

    def results(self, stream=None) -> dict:
        tot = sum(nb * D * D for nb, D in self._mat_sizes())
        n = np.zeros(2 * tot)
        U, J, E = np.zeros(self.natoms), np.zeros(self.natoms), np.zeros(self.natoms)
        Et = np.zeros(1)
        self._check(self.lib.dftu_get_results(self.h, _dp(n), _dp(U), _dp(J), _dp(E), _dp(Et), _stream_ptr(stream, self.device)))
        return dict(n=self._unpack_mats(n), U=U, J=J, EU_atom=E, EU=float(Et[0]))

    def occupation_matrices(self, stream=None):
        tot = sum(nb * D * D for nb, D in self._mat_sizes())
        n = np.zeros(2 * tot)
        self._check(self.lib.dftu_get_results(self.h, _dp(n), None, None, None, None, _stream_ptr(stream, self.device)))
        return self._unpack_mats(n)

    def renormalized(self, nbands: int, stream=None):
        tot = sum(nb * D * D for nb, D in self._mat_sizes())
        P = np.zeros(2 * tot)
        rows = self.nk if self.spin == NONCOLLINEAR else self.nk * self.ns
        nsp = max(self.species) + 1
        Nb = np.zeros(rows * nbands * nsp)
        self._check(self.lib.dftu_get_renormalized(self.h, _dp(P), _dp(Nb), _stream_ptr(stream, self.device)))
        return self._unpack_mats(P), Nb.reshape(rows, nbands, nsp)

    def projections(self, nbands: int, stream=None) -> np.ndarray:
        MT = self.lib.dftu_total_orbitals(self.h)
        rows = self.nk * self.ns if self.spin != NONCOLLINEAR else self.nk * 2
        p = np.zeros(2 * rows * nbands * MT)
        self._check(self.lib.dftu_get_projections(self.h, _dp(p), _stream_ptr(stream, self.device)))
        return (p[0::2] + 1j * p[1::2]).reshape(rows, nbands, MT)

    def sync_status(self) -> int:
        return self.lib.dftu_sync_status(self.h)


class Batch:
    """Many set-up handles processed by persistent launches (dftu_batch_*).  Keeps references to the
    member handles and the bound tensors so they outlive the batch."""

    def __init__(self, handles: Sequence[Handle]):
        self.lib = load()
        self.handles = list(handles)
        arr = (C.c_void_p * len(handles))(*[h.h.value for h in handles])
        b = C.c_void_p()
        st = self.lib.dftu_batch_create(C.byref(b), len(handles), arr)
        if st != DFTU_OK:
            raise DftuError(st, "batch_create")
        self.b = b
        self.device = handles[0].device

    def _check(self, st):
        if st != DFTU_OK:
            raise DftuError(st, self.lib.dftu_batch_last_error(self.b).decode())

    def bind(self, psis: Sequence[torch.Tensor], fs: Sequence[torch.Tensor]):
        n = len(self.handles)
        prec = C128 if psis[0].dtype == torch.complex128 else C64
        nb, ld = [], []
        for h, p, f in zip(self.handles, psis, fs):
            pr, nbi, ldi = h._psi_args(p)
            if pr != prec:
                raise ValueError("one precision for the whole batch")
            if f.dtype != torch.float64 or not f.is_cuda or not f.is_contiguous():
                raise ValueError("f must be contiguous float64 CUDA tensors")
            nb.append(nbi)
            ld.append(ldi)
        self._keep = (list(psis), list(fs))
        pa = (C.c_void_p * n)(*[p.data_ptr() for p in psis])
        fa = (C.c_void_p * n)(*[f.data_ptr() for f in fs])
        self._check(self.lib.dftu_batch_bind(self.b, pa, prec, (C.c_int * n)(*nb), (C.c_int64 * n)(*ld), fa))

    def project(self, stream=None):
        self._check(self.lib.dftu_batch_project(self.b, _stream_ptr(stream, self.device)))

    def occupations(self, stream=None):
        self._check(self.lib.dftu_batch_occupations(self.b, _stream_ptr(stream, self.device)))

    def access_ceiling(self, psi: torch.Tensor, rmw: bool = False, stream=None):
        """One pass of the access pattern alone (dftu_access_ceiling): read every sphere point of psi, or
        read and write each back unchanged; time it to bound the projection (read) and the apply (rmw)."""
        prec, nb, ld = self._psi_args(psi)
        self._check(self.lib.dftu_access_ceiling(self.h, C.c_void_p(psi.data_ptr()), prec, nb, ld, 1 if rmw else 0,
                                                 _stream_ptr(stream, self.device)))

    def occupation_sums(self, out: torch.Tensor = None, stream=None) -> torch.Tensor:
        """This handle's occupation sums (rho, Pbar) of the last occupations, as a float64 tensor on the
        handle's device (written into `out` when given) -- the part a rank adds up with the others."""
        n = int(self.lib.dftu_occupation_elems(self.h))
        if out is None:
            out = torch.empty(n, dtype=torch.float64, device=torch.device("cuda", self.device))
        if out.dtype != torch.float64 or out.numel() != n or not out.is_contiguous():
            raise ValueError(f"out must be a contiguous float64 tensor of {n} elements")
        self._check(self.lib.dftu_export_occupations(self.h, C.c_void_p(out.data_ptr()), _stream_ptr(stream, self.device)))
        return out

    def set_occupation_sums(self, sums: torch.Tensor, stream=None):
        """Overwrite the occupation sums (e.g. with their total over ranks) before acbn0_uj."""
        n = int(self.lib.dftu_occupation_elems(self.h))
        if sums.dtype != torch.float64 or sums.numel() != n or not sums.is_contiguous():
            raise ValueError(f"sums must be a contiguous float64 tensor of {n} elements")
        self._check(self.lib.dftu_import_occupations(self.h, C.c_void_p(sums.data_ptr()), _stream_ptr(stream, self.device)))

    def acbn0_uj(self, stream=None):
        self._check(self.lib.dftu_batch_acbn0_uj(self.b, _stream_ptr(stream, self.device)))

    def apply(self, coef: Optional[torch.Tensor] = None, accumulate: bool = True, stream=None):
        cp = C.c_void_p(coef.data_ptr()) if coef is not None else None
        self._check(self.lib.dftu_batch_apply(self.b, cp, 1 if accumulate else 0, _stream_ptr(stream, self.device)))

    def close(self):
        if getattr(self, "b", None):
            self.lib.dftu_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def radius_cell(grid) -> float:
    """Second method of Sec. II: the smallest cell edge."""
    g = DftuGrid((C.c_int * 3)(*grid.n), (C.c_double * 3)(*grid.h), (C.c_double * 3)(*grid.origin), 1 if grid.periodic else 0)
    return load().dftu_radius_cell(C.byref(g))


def radius_threshold(radial, threshold: float) -> float:
    """Third method of Sec. II: where the radial function falls below `threshold` for good."""
    R = np.ascontiguousarray(radial.R, dtype=np.float64)
    r = DftuRadial(len(R), radial.dr, _dp(R))
    return load().dftu_radius_threshold(C.byref(r), float(threshold))


def handle_for_system(system, max_bands: int, device: int = 0) -> Handle:
    """Create a handle for a synthetic System (see synth.py) and set up its atoms."""
    spin = NONCOLLINEAR if system.noncollinear else (UNPOLARIZED if system.nspin == 1 else COLLINEAR)
    h = Handle(system.grid, system.kpts, system.wk, spin, max_bands, device)
    h.setup_atoms(system.atoms, system.radials)
    return h
