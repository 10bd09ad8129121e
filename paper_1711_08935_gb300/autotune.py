"""Autotuner for the streaming kernels: times every shape variant of the projection and apply
kernels (dftu_set_kernel_variant) on the caller's own states with CUDA events and keeps the fastest.
The apply variants accumulate into `out` (the caller's H psi buffer), or into psi itself when no
buffer is given."""
from __future__ import annotations

import torch

from . import dftu

WHICH = {("project", torch.complex128): 0, ("project", torch.complex64): 1,
         ("apply", torch.complex128): 2, ("apply", torch.complex64): 3}


def _time(fn, reps, stream):
    fn()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def autotune(h: dftu.Handle, psi: torch.Tensor, reps: int = 3, out: torch.Tensor = None) -> dict:
    """Pick the fastest projection and apply variants for psi's precision; returns the timings (ms).
    The handle must already hold a potential (dftu_acbn0_uj) for the apply to run."""
    target = psi if out is None else out
    stream = torch.cuda.current_stream(psi.device)
    out = {}
    for kind in ("project", "apply"):
        which = WHICH[(kind, psi.dtype)]
        n = h.lib.dftu_kernel_variants(which)
        times = []
        for v in range(n):
            h.set_kernel_variant(which, v)
            fn = (lambda: h.project(psi)) if kind == "project" else (lambda: h.apply(target))
            times.append(_time(fn, reps, stream))
        best = min(range(n), key=lambda i: times[i])
        h.set_kernel_variant(which, best)
        out[kind] = {"variant": best, "ms": [round(t, 4) for t in times]}
    h.project(psi)      # leave fresh projections of the current states in the handle
    return out


def autotune_batch(batch: dftu.Batch, dtype: torch.dtype, coef: torch.Tensor = None, reps: int = 3) -> dict:
    """The same for a batch: its persistent launches use the shapes set on its first member, so every
    shape is timed on the batch's own launches.  The batch must hold potentials (batch acbn0_uj) for
    the apply to run; its applies change the bound states, with `coef` as the coefficient."""
    h0 = batch.handles[0]
    stream = torch.cuda.current_stream(torch.device("cuda", batch.device))
    out = {}
    for kind in ("project", "apply"):
        which = WHICH[(kind, dtype)]
        n = h0.lib.dftu_kernel_variants(which)
        times = []
        for v in range(n):
            h0.set_kernel_variant(which, v)
            fn = batch.project if kind == "project" else (lambda: batch.apply(coef))
            times.append(_time(fn, reps, stream))
        best = min(range(n), key=lambda i: times[i])
        h0.set_kernel_variant(which, best)
        out[kind] = {"variant": best, "ms": [round(t, 4) for t in times]}
    batch.project()
    return out
