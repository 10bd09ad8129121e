"""Autotuner for the streaming kernels: times every shape variant of the projection and apply
kernels (dftu_set_kernel_variant) on the caller's own states with CUDA events (median of single-launch
timings after warm-up), re-times the two fastest, and keeps the faster.
The apply variants accumulate into `out` (the caller's H psi buffer), or into psi itself when no
buffer is given."""
from __future__ import annotations

import statistics

import torch

from . import dftu

WHICH = {("project", torch.complex128): 0, ("project", torch.complex64): 1,
         ("apply", torch.complex128): 2, ("apply", torch.complex64): 3}


def _time(fn, reps, stream, warmup=2):
    """Median of `reps` single-launch CUDA-event timings after `warmup` untimed launches (ms)."""
    for _ in range(warmup):
        fn()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a, b in ev:
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return statistics.median(a.elapsed_time(b) for a, b in ev)


def _pick(set_variant, n, fn, reps, stream):
    """Time every variant, then time the two fastest again (alternating, more repetitions) and keep the
    faster of those, so that one noisy repetition cannot decide the shape."""
    times = []
    for v in range(n):
        set_variant(v)
        times.append(_time(fn, reps, stream))
    order = sorted(range(n), key=lambda i: times[i])[:2]
    final = {v: [] for v in order}
    for _ in range(3):
        for v in order:
            set_variant(v)
            final[v].append(_time(fn, reps, stream, warmup=1))
    best = min(order, key=lambda v: statistics.median(final[v]))
    set_variant(best)
    return best, times, {v: round(statistics.median(t), 4) for v, t in final.items()}


def autotune(h: dftu.Handle, psi: torch.Tensor, reps: int = 5, out: torch.Tensor = None) -> dict:
    """Pick the fastest projection and apply variants for psi's precision; returns the timings (ms).
    The handle must already hold a potential (dftu_acbn0_uj) for the apply to run."""
    target = psi if out is None else out
    stream = torch.cuda.current_stream(psi.device)
    out = {}
    for kind in ("project", "apply"):
        which = WHICH[(kind, psi.dtype)]
        n = h.lib.dftu_kernel_variants(which)
        fn = (lambda: h.project(psi)) if kind == "project" else (lambda: h.apply(target))
        best, times, final = _pick(lambda v: h.set_kernel_variant(which, v), n, fn, reps, stream)
        out[kind] = {"variant": best, "ms": [round(t, 4) for t in times], "retimed": final}
    h.project(psi)      # leave fresh projections of the current states in the handle
    return out


def autotune_batch(batch: dftu.Batch, dtype: torch.dtype, coef: torch.Tensor = None, reps: int = 5) -> dict:
    """The same for a batch: its persistent launches use the shapes set on its first member, so every
    shape is timed on the batch's own launches.  The batch must hold potentials (batch acbn0_uj) for
    the apply to run; its applies change the bound states, with `coef` as the coefficient."""
    h0 = batch.handles[0]
    stream = torch.cuda.current_stream(torch.device("cuda", batch.device))
    out = {}
    for kind in ("project", "apply"):
        which = WHICH[(kind, dtype)]
        n = h0.lib.dftu_kernel_variants(which)
        fn = batch.project if kind == "project" else (lambda: batch.apply(coef))
        best, times, final = _pick(lambda v: h0.set_kernel_variant(which, v), n, fn, reps, stream)
        out[kind] = {"variant": best, "ms": [round(t, 4) for t in times], "retimed": final}
    batch.project()
    return out
