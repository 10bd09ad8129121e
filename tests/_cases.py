"""Small seeded systems shared by the oracle pins and the GPU parity tests."""
import math

import numpy as np
import torch

from paper_1711_08935_gb300 import synth
from paper_1711_08935_gb300.synth import Atom, Grid, System


def periodic_tiny(R=3.5, n=12, h=0.5, k=(0.3, -0.2, 0.1)):
    """Periodic 12^3 cell of edge 6 bohr with one d atom whose sphere (R > L/2) overlaps its own
    periodic images; one general k-point so projections are complex."""
    g = Grid(n=(n, n, n), h=(h, h, h), periodic=True)
    at = [Atom((1.1, 2.3, 5.7), 0, 2, R)]
    return System(g, at, [synth.hydrogenic_radial(3, 2, 2.0)], np.array([k]), np.ones(1), nspin=1,
                  name="periodic tiny, self-overlapping sphere")


def periodic_two_atoms(nspin=2, k=((0.21, -0.13, 0.07), (-0.1, 0.05, 0.3))):
    """Periodic 20^3 cell (h=0.4, L=8) with a d atom and a p atom near opposite corners, two k-points."""
    g = Grid(n=(20, 20, 20), h=(0.4, 0.4, 0.4), periodic=True)
    at = [Atom((0.3, 7.6, 0.5), 0, 2, 3.0), Atom((4.2, 3.9, 4.4), 1, 1, 2.6)]
    kp = np.array(k)
    return System(g, at, [synth.hydrogenic_radial(3, 2, 3.0), synth.hydrogenic_radial(2, 1, 3.5)], kp,
                  np.full(len(kp), 1.0 / len(kp)), nspin=nspin, name="periodic 20^3, d + p atom, 2 k")


def states_np(system, nbands, seed, **kw):
    return synth.make_states(system, nbands, seed, device="cpu", **kw).numpy()


def gram_schmidt_after(first: np.ndarray, rest: np.ndarray, dV: float) -> np.ndarray:
    """Modified Gram-Schmidt (grid inner product) of the rows of [first; rest], first rows kept
    as they are when they are already orthonormal."""
    A = np.concatenate([first, rest], 0).astype(np.complex128)
    for i in range(A.shape[0]):
        for j in range(i):
            A[i] -= dV * np.vdot(A[j], A[i]) * A[j]
        A[i] /= math.sqrt(dV * np.vdot(A[i], A[i]).real)
    return A


def overlapping_three_atoms():
    """Periodic 24^3 cell (h = 0.4, L = 9.6) with three atoms of three species whose spheres overlap
    each other (and one reaches its own periodic image): the apply must add every contribution."""
    g = Grid(n=(24, 24, 24), h=(0.4, 0.4, 0.4), periodic=True)
    at = [Atom((1.0, 1.2, 0.8), 0, 2, 3.2), Atom((3.1, 2.0, 1.5), 1, 1, 2.8), Atom((2.0, 3.6, 2.9), 2, 2, 5.0)]
    kp = np.array([[0.11, -0.05, 0.2], [-0.2, 0.13, 0.04]])
    return System(g, at, [synth.hydrogenic_radial(3, 2, 3.0), synth.hydrogenic_radial(2, 1, 3.5),
                          synth.hydrogenic_radial(3, 2, 2.5)], kp, np.array([0.5, 0.5]), nspin=1,
                  name="overlapping spheres, three species, 2 k")
