"""Benchmark of the DFT+U (ACBN0) Hubbard-projector pass on GB300.

One step = one pass of the whole hot path over the oxide supercell (periodic 96^3 grid at 0.25 bohr,
8 transition-metal d shells + 8 oxygen p shells, 256 bands, 8 k-points, collinear spin):
    project -> occupations (n, Nbar, Pbar) -> ACBN0 U, J, E_U, V -> apply (H psi += V_U psi)
through the C ABI, the apply accumulating into a separate H psi buffer so that every step sees the
same states.  The metric is algorithmic GB/s of that pass: every sphere point of every state is read
by the projection and read + written by the apply (complex128: 16 B per point).

Prints ONE JSON line (rank 0).  --impl reference times the CPU FP64 oracle on a bounded sample of the
same workload instead.  Under torchrun every rank runs an independent replica (the pass has no
cross-GPU exchange), timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DFT+U projector GB/s & %HBM peak; FP32-state vs FP64 speedup at |dn|<=1e-6"
UNIT = "GB/s"
WORKLOAD = "oxide supercell 96^3 h=0.25, 8 TM(3d,R4.5)+8 O(2p,R3.5), 256 bands, 8 k, collinear, FP64 states"

# DRAM bytes per state (one band of one k-point and spin) measured by ncu (dram__bytes_read.sum +
# dram__bytes_write.sum) on the 64-band oxide case for the kernel variants named here; see
# profiles/project_apply_oxide_small.md.  Valid only while that variant is the one timed.
NCU_TRAFFIC_PER_STATE = {("project", 0): (802.03e6 + 5.63e6) / 128,
                         ("apply", 0): (800.74e6 + 566.71e6) / 128}
# The same for the fixed complex128 shapes of the gauge-invariant path; see
# profiles/gauge_project_apply_current_oxide_small.md.
# Both kernels changed after that capture (the projection's split and shape, the apply's precomputed
# coefficients), so neither figure is reported.
NCU_TRAFFIC_PER_STATE_GAUGE = {"project": None, "apply": None}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            return float(d.get("hbm_gbs")), "measured (MEASURED_PEAKS.json)"
        except Exception:
            pass
    return 6800.0, "fallback (6.8 TB/s, profiling recipe)"


def smi_gpu_id(ordinal: int, uuid=None, visible=None) -> str:
    """The nvidia-smi -i argument that names CUDA device `ordinal`.  nvidia-smi numbers GPUs by its own
    (PCI) enumeration and ignores CUDA_VISIBLE_DEVICES, so a CUDA ordinal is not an nvidia-smi index when
    only some GPUs are visible.  The device's UUID names it unambiguously; without one, the ordinal's
    entry of CUDA_VISIBLE_DEVICES (an index or a UUID) is used, and the ordinal itself only when that
    variable is unset."""
    if uuid:
        u = str(uuid).strip()
        return u if u.startswith(("GPU-", "MIG-")) else "GPU-" + u
    if visible:
        entries = [x.strip() for x in visible.split(",") if x.strip()]
        if 0 <= ordinal < len(entries):
            return entries[ordinal]
    return str(ordinal)


def resolve_smi_id(ordinal: int) -> str:
    uuid = None
    try:
        import torch
        uuid = str(torch.cuda.get_device_properties(ordinal).uuid)
    except Exception:
        uuid = None
    visible = os.environ.get("CUDA_VISIBLE_DEVICES")
    for cand in (smi_gpu_id(ordinal, uuid, visible), smi_gpu_id(ordinal, None, visible)):
        try:
            r = subprocess.run(["nvidia-smi", "-i", cand, "--query-gpu=uuid", "--format=csv,noheader"],
                               capture_output=True, text=True, timeout=20)
            if r.returncode == 0 and r.stdout.strip():
                return cand
        except Exception:
            pass
    return smi_gpu_id(ordinal, uuid, visible)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region.  Sampling starts before the region
    (nvidia-smi takes a moment to start) and every sample carries nvidia-smi's own timestamp; mark() records
    the region's wall-clock bounds, and only the samples inside them are summarised (all of them when no
    region was marked, with the count of those inside reported either way)."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 25

    def __init__(self, device_ordinal: int):
        self.gpu = resolve_smi_id(device_ordinal)
        self.rows = []
        self.proc = None
        self.marks = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.gpu, f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", str(self.PERIOD_MS)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.5)   # let nvidia-smi start sampling before the region begins
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def mark(self):
        """Call right after a device synchronisation at the start and at the end of the timed region."""
        self.marks.append(time.time())

    @staticmethod
    def summarize(rows, t0=None, t1=None):
        """Median SM clock, maximum clock and the throttle reasons seen, over the samples whose timestamp
        lies in [t0, t1].  Without a region, or when no sample carries a readable timestamp, all samples
        count; when none falls inside the region, those within 0.1 s of it count, and a note says so."""
        import datetime
        parsed = []
        for r in rows:
            if len(r) < 10 or not r[2].replace(".", "").isdigit():
                continue
            try:
                ts = datetime.datetime.strptime(r[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                ts = None
            parsed.append((ts, r))
        note = None
        use = [r for _, r in parsed]
        if t0 is not None:
            if not any(ts is not None for ts, _ in parsed):
                note = "nvidia-smi timestamps unreadable: all samples used"
            else:
                inside = [r for ts, r in parsed if ts is not None and t0 <= ts <= t1]
                near = [r for ts, r in parsed if ts is not None and t0 - 0.1 <= ts <= t1 + 0.1]
                if inside:
                    use = inside
                elif near:
                    use, note = near, "no sample inside the timed region: samples within 0.1 s of it used"
                else:
                    note = "no sample near the timed region: all samples used"
        sm = [float(r[2]) for r in use]
        mx = [float(r[3]) for r in use if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in use:
            for n, val in zip(names, r[6:10]):
                if val.lower().startswith("active"):
                    reasons.add(n)
        out = {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
               "reasons": sorted(reasons), "samples": len(sm), "sample_period_ms": ClockSampler.PERIOD_MS}
        if t0 is not None:
            out["region_s"] = round(t1 - t0, 3)
        if note:
            out["note"] = note
        return out

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        out = self.summarize(self.rows, self.marks[0], self.marks[-1]) if len(self.marks) >= 2 else self.summarize(self.rows)
        out["gpu"] = self.gpu
        return out


def max_over_ranks(values, device):
    """Element-wise maximum of a list of floats over all ranks of the default process group (any
    backend); the identity without torch.distributed initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return list(values)
    t = torch.tensor(values, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_system(s, rank, ws):
    """The k-point shard of `rank` out of `ws`: each rank holds its own copy of the base k-point set shifted
    by rank * (1/97, 1/89, 1/83) of the reciprocal lattice vectors, with the weights divided by ws, so the
    ranks together hold one k-point set of ws times the base size (per-GPU work fixed: weak scaling)."""
    if ws <= 1:
        return s
    import dataclasses
    L = np.array(s.grid.L, dtype=np.float64)
    shift = rank * (2.0 * math.pi / L) * np.array([1.0 / 97, 1.0 / 89, 1.0 / 83])
    return dataclasses.replace(s, kpts=np.asarray(s.kpts) + shift[None, :], wk=np.asarray(s.wk) / ws)


def algorithmic_bytes(handle_npts, nbands, nk, ns, bytes_per_point, orbitals_bytes):
    """(projection bytes, apply bytes) of one pass: every sphere point of every state once for the
    projection (plus the orbital table once), twice (read + write) for the apply."""
    pts = int(sum(handle_npts))
    states = pts * bytes_per_point * nbands * nk * ns
    return states + orbitals_bytes, 2 * states + orbitals_bytes


def run_ours(args):
    import torch
    from paper_1711_08935_gb300 import dftu, synth

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    s = rank_system(synth.oxide_system(n=args.grid, nk=args.nkgrid), rank, ws)
    nb = args.nbands
    nocc = nb // 2
    t0 = time.time()
    psi = synth.make_states(s, nb, seed=2, device=dev, spin_bias=synth.afm_spin_bias(s))
    gen_s = time.time() - t0
    f = torch.from_numpy(synth.step_occupations(s.nk, 2, nb, nocc)).to(dev)
    h = dftu.handle_for_system(s, nb, device=local)
    for sp in range(len(s.radials)):
        h.coulomb_integrals(sp)
    npts = [h.lib.dftu_atom_points(h.h, i) for i in range(len(s.atoms))]
    MT = h.lib.dftu_total_orbitals(h.h)
    orb_bytes = sum(n * (2 * a.l + 1) * 8 for n, a in zip(npts, s.atoms))
    stream = torch.cuda.current_stream(dev)

    # ---- precision check on identical inputs before any apply: FP32-state vs FP64 occupations
    psi32 = psi.to(torch.complex64)
    h.project(psi); h.occupations(f); h.acbn0_uj()
    r64 = h.results()
    h.project(psi32); h.occupations(f); h.acbn0_uj()
    r32 = h.results()
    max_dn = max(float(np.max(np.abs(a - b))) for a, b in zip(r64["n"], r32["n"]))
    dU = float(np.max(np.abs(r64["U"] - r32["U"]))) * dftu.HARTREE_EV
    dJ = float(np.max(np.abs(r64["J"] - r32["J"]))) * dftu.HARTREE_EV
    dE = abs(r64["EU"] - r32["EU"]) * dftu.HARTREE_EV

    # Under torchrun every rank holds its own k-points of one k-point set (weights in the whole set): the
    # occupation sums of Eqs. (4) and (8) are added over the ranks (one allreduce per pass) before ACBN0.
    sums = torch.empty(int(h.lib.dftu_occupation_elems(h.h)), dtype=torch.float64, device=dev)

    def exchange():
        if ws > 1:
            h.occupation_sums(sums)
            torch.distributed.all_reduce(sums)
            h.set_occupation_sums(sums)

    # H psi accumulates V_U psi (Eq. 6) in its own buffer, as in a Hamiltonian application: every step
    # then works on the same states, and the apply reads and writes as many bytes as an in-place one.
    def step(x, out):
        h.project(x)
        h.occupations(f)
        exchange()
        h.acbn0_uj()
        h.apply(out)

    def timed(x, out, steps, warmup, sampler=None):
        for _ in range(warmup):
            step(x, out)
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
               torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
               torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        if sampler is not None:
            sampler.mark()
        start.record(stream)
        for i in range(steps):
            e0, e1, e2, e3, e4 = ev[i]
            e0.record(stream)
            h.project(x)
            e1.record(stream)
            h.occupations(f)
            exchange()
            h.acbn0_uj()
            e2.record(stream)
            e3.record(stream)
            h.apply(out)
            e4.record(stream)
        end.record(stream)
        torch.cuda.synchronize()
        if sampler is not None:
            sampler.mark()
        total = start.elapsed_time(end)
        proj = [e[0].elapsed_time(e[1]) for e in ev]
        small = [e[1].elapsed_time(e[2]) for e in ev]
        app = [e[3].elapsed_time(e[4]) for e in ev]
        return total / steps, statistics.mean(proj), statistics.mean(small), statistics.mean(app)

    tuned = {}
    if args.variants:
        for which, var in enumerate(int(x) for x in args.variants.split(",")):
            h.set_kernel_variant(which, var)
        tuned["fixed"] = args.variants
    hpsi = torch.zeros_like(psi)
    if not args.variants and not args.no_tune:
        from paper_1711_08935_gb300.autotune import autotune
        tuned["c128"] = autotune(h, psi, out=hpsi)
        hpsi32 = torch.zeros_like(psi32)
        tuned["c64"] = autotune(h, psi32, out=hpsi32)
        del hpsi32
        h.project(psi); h.occupations(f); h.acbn0_uj()
    clocks = ClockSampler(local)
    clocks.start()
    ms64, proj64, small64, app64 = timed(psi, hpsi, args.steps, args.warmup, sampler=clocks)
    clk = clocks.stop()
    # the access pattern's own ceiling on these buffers: gather (projection) and read-modify-write (apply)
    def ceiling_ms(x, rmw, reps=5):
        for _ in range(2):
            h.access_ceiling(x, rmw)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for e0, e1 in evs:
            e0.record(stream)
            h.access_ceiling(x, rmw)
            e1.record(stream)
        torch.cuda.synchronize()
        return statistics.median(e0.elapsed_time(e1) for e0, e1 in evs)

    ceil = {"c128_gather_ms": ceiling_ms(psi, False), "c128_rmw_ms": ceiling_ms(hpsi, True)}
    # the same pass with plain FP64 fused multiply-adds (DFTU_F64_NATIVE), same states and buffers
    msn = projn = appn = None
    if not args.no_extra:
        h.set_f64_mode(dftu.F64_NATIVE)
        msn, projn, _, appn = timed(psi, hpsi, max(2, min(args.steps, 5)), 2)
        h.set_f64_mode(dftu.F64_PAIR)
    del psi, hpsi
    torch.cuda.empty_cache()
    hpsi32 = torch.zeros_like(psi32)
    ms32, proj32, small32, app32 = timed(psi32, hpsi32, args.steps, args.warmup)
    ceil["c64_gather_ms"] = ceiling_ms(psi32, False)
    ceil["c64_rmw_ms"] = ceiling_ms(hpsi32, True)
    del hpsi32
    status = h.sync_status()

    pb64, ab64 = algorithmic_bytes(npts, nb, s.nk, 2, 16, orb_bytes)
    pb32, ab32 = algorithmic_bytes(npts, nb, s.nk, 2, 8, orb_bytes)
    step_bytes64 = pb64 + ab64
    ms64, ms32 = max_over_ranks([ms64, ms32], dev)
    if msn is not None:
        msn = max_over_ranks([msn], dev)[0]
    value = ws * step_bytes64 / (ms64 * 1e-3) / 1e9
    peak, peak_src = measured_peaks()
    # dominant kernel by time: the apply (read + write of every sphere point)
    dom = "apply" if app64 >= proj64 else "project"
    dom_ms = app64 if dom == "apply" else proj64
    dom_bytes = ab64 if dom == "apply" else pb64
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9
    chosen = {"project": h.variants_now()[0], "apply": h.variants_now()[2]}
    tkey = (dom, chosen[dom])
    traffic = NCU_TRAFFIC_PER_STATE[tkey] * nb * s.nk * 2 if tkey in NCU_TRAFFIC_PER_STATE else None

    # ---- end to end through the public API with host (pinned) states
    e2e = None
    if not args.no_e2e:
        # every rank pins its own host copy of the states: skip the leg if the copies would not fit
        host_ram = os.sysconf("SC_PHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
        need = 2 * ws * host_bytes(s, nb)              # psi and H psi, pinned, per rank
        if need > 0.75 * host_ram:
            e2e = {"skipped": f"{ws} ranks x {2 * host_bytes(s, nb) / 1e9:.0f} GB of pinned host states exceed "
                              f"0.75 of the host's {host_ram / 1e9:.0f} GB"}
        else:
            e2e = run_e2e(args, h, s, nb, f, dev, step_bytes64, ws, exchange)

    line = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms64, 4), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c128 states; FP32-pair arithmetic (~2^-44) for products, FP64 occupations/U/J",
        "data": "synthetic (seeded Gaussian-type Bloch states, orthonormalised; hydrogenic radial orbitals)",
        "config": {"workload": WORKLOAD, "global_batch": nb * s.nk * 2 * ws, "seq_len": int(sum(npts)),
                   "parallelism": (f"k-point shards x{ws}: one allreduce of the occupation sums per pass" if ws > 1
                                   else "single GPU"),
                   "l2": "inputs (58 GB of states) far larger than L2; no flush needed",
                   "sphere_points": int(sum(npts)), "bands": nb, "kpoints": s.nk, "spins": 2},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "peak_source": peak_src,
                     "frac_of_nominal_7900": round(achieved / 7900.0, 4),
                     "traffic": round(traffic) if traffic else None,
                     "bytes_per_launch": dom_bytes},
        "kernels_ms": {"project": round(proj64, 4), "occupations+acbn0": round(small64, 4), "apply": round(app64, 4),
                       "project_GBps": round(pb64 / (proj64 * 1e-3) / 1e9, 1),
                       "apply_GBps": round(ab64 / (app64 * 1e-3) / 1e9, 1)},
        "fp32_state": {"ms_per_step": round(ms32, 4), "GBps": round((pb32 + ab32) / (ms32 * 1e-3) / 1e9, 2),
                       "speedup_vs_fp64": round(ms64 / ms32, 3),
                       "speedup_vs_fp64_native": round(msn / ms32, 3) if msn else None,
                       "max_abs_dn": max_dn, "max_dU_eV": dU, "max_dJ_eV": dJ, "dEU_eV": dE,
                       "differences_against": "the complex128 pass on the same states (itself held to 1e-12 of the "
                                              "oracle at full size by the GPU tests)",
                       "project_ms": round(proj32, 4), "apply_ms": round(app32, 4)},
        "access_ceiling": {
            "what": "one pass of the access pattern alone (dftu_access_ceiling): every sphere point read once, or read "
                    "and written back unchanged, same tiles, no arithmetic",
            "c128_gather_GBps": round((pb64 - orb_bytes) / (ceil["c128_gather_ms"] * 1e-3) / 1e9, 1),
            "c128_rmw_GBps": round((ab64 - orb_bytes) / (ceil["c128_rmw_ms"] * 1e-3) / 1e9, 1),
            "c64_gather_GBps": round((pb32 - orb_bytes) / (ceil["c64_gather_ms"] * 1e-3) / 1e9, 1),
            "c64_rmw_GBps": round((ab32 - orb_bytes) / (ceil["c64_rmw_ms"] * 1e-3) / 1e9, 1),
            "project_frac_of_ceiling": round(ceil["c128_gather_ms"] / proj64, 4),
            "apply_frac_of_ceiling": round(ceil["c128_rmw_ms"] / app64, 4),
            "pass_frac_of_ceiling": round((ceil["c128_gather_ms"] + ceil["c128_rmw_ms"]) / ms64, 4),
            "c64_project_frac_of_ceiling": round(ceil["c64_gather_ms"] / proj32, 4),
            "c64_apply_frac_of_ceiling": round(ceil["c64_rmw_ms"] / app32, 4)},
        "f64_native": ({"ms_per_step": round(msn, 4), "GBps": round(step_bytes64 / (msn * 1e-3) / 1e9, 2),
                        "project_ms": round(projn, 4), "apply_ms": round(appn, 4),
                        "note": "plain FP64 FMAs on this GPU's FP64 pipe (DFTU_F64_NATIVE), same states"}
                       if msn else None),
        "results": {"U_eV": [round(x * dftu.HARTREE_EV, 6) for x in r64["U"]],
                    "J_eV": [round(x * dftu.HARTREE_EV, 6) for x in r64["J"]], "EU_eV": r64["EU"] * dftu.HARTREE_EV},
        "clocks": clk, "e2e": e2e, "tuning": tuned, "gpu_launches": None, "device_status": int(status),
        "state_generation_s": round(gen_s, 1),
    }
    # our kernel launches in the timed FP64 region: project (2: tiles, tile reduce), occupations (2: Nbar,
    # matrices), acbn0 (2: per-atom U/J/V, energy sum), apply (coefficient vectors + 1 per colour; the oxide
    # spheres do not overlap, so one colour)
    line["gpu_launches"] = (2 + 2 + 2 + 2) * args.steps
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_baseline(args, s)
    if ws == 1 and not args.no_extra:
        # the other workloads of the method, each timed on the device with its own clock record
        h.close()
        del psi32, f
        torch.cuda.empty_cache()
        line["workloads"] = extra_workloads(args)
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()


def extra_workloads(args):
    """The non-collinear pass, the real-time step and the molecule batch, in that order, with the default
    sizes of their workloads; their JSON objects without the tuning tables."""
    import copy
    import torch
    out = {}
    for name, fn in (("nc", run_nc), ("rt", run_rt), ("molecules", run_molecules)):
        a = copy.copy(args)
        a.grid, a.nbands, a.nkgrid = 96, 256, 2
        t0 = time.time()
        r = fn(a)
        r.pop("tuning", None)
        r["wall_s"] = round(time.time() - t0, 1)
        out[name] = r
        torch.cuda.empty_cache()
    return out


def run_e2e(args, h, s, nb, f, dev, step_bytes, ws, exchange):
    """The pass end to end through the public API with the states AND the H psi result in pinned host
    memory.  The projection kernels read the sphere points of psi straight from host memory over the host
    link, the apply reads and writes the sphere points of the host H psi buffer the same way (only sphere
    points cross the link; no staging copy of whole grids), and the results (n, U, J, E_U) are read back
    every step.  Under torchrun the occupation sums are exchanged as in the device-resident pass."""
    import torch
    from paper_1711_08935_gb300 import synth
    host = torch.empty((s.nk, 2, nb, s.grid.npts), dtype=torch.complex128, pin_memory=True)
    gen = synth.make_states(s, nb, seed=7, device=dev, spin_bias=synth.afm_spin_bias(s))
    host.copy_(gen)
    del gen
    torch.cuda.empty_cache()
    hpsi = torch.zeros(host.shape, dtype=host.dtype, pin_memory=True)
    n_steps = max(1, min(args.steps, 5))

    def direct():
        h.project(host)
        h.occupations(f)
        exchange()
        h.acbn0_uj()
        h.apply(hpsi)
        return h.results()

    direct()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n_steps):
        r = direct()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / n_steps
    npts = int(sum(h.lib.dftu_atom_points(h.h, i) for i in range(len(s.atoms))))
    sphere = npts * 16 * nb * s.nk * 2               # sphere points of every state, complex128
    results = sum(x.size for x in r["n"]) * 16 + 3 * len(s.atoms) * 8 + 8
    del hpsi, host
    return {"value": round(ws * step_bytes / dt / 1e9, 2), "unit": UNIT,
            "h2d_bytes_per_step": int(2 * sphere), "d2h_bytes_per_step": int(sphere + results),
            "steps": n_steps, "ms_per_step": round(dt * 1e3, 2),
            "mode": "psi and H psi in pinned host memory: the projection reads the sphere points of psi, the apply "
                    "reads and writes those of H psi over the host link; n, U, J, E_U read back every step"}


def host_bytes(s, nb):
    return s.nk * 2 * nb * s.grid.npts * 16


def _oracle_coulomb(O, s, st):
    coul = []
    for sp in range(len(s.radials)):
        I = [a.species for a in s.atoms].index(sp)
        coul.append(O.coulomb_integrals(s.grid, s.atoms[I], st[I]))
    return coul


def cpu_sample(kind: str, target_s: float) -> dict:
    """Time the CPU FP64 oracle, as it stands, on a bounded sample of one workload (repeated for about
    target_s seconds; set-up and Coulomb integrals outside the timed loop):
      oxide:     1 k-point x 2 spins x 4 bands of the 96^3 oxide, a full pass;
      tiny:      the one-atom isolated 32^3 case, 21 states, a full pass;
      rt_prefix: 10 Taylor-4 real-time steps of 1 k-point x 1 band of the 128^3 real-time workload."""
    from oracle import dftu_oracle as O
    from paper_1711_08935_gb300 import synth
    if kind == "oxide":
        s0 = synth.oxide_system(n=96, nk=2)
        s = synth.System(s0.grid, s0.atoms, s0.radials, s0.kpts[:1], np.ones(1), nspin=2)
        nbs = 4
        f = np.ones((1, 2, nbs))
    elif kind == "tiny":
        s = synth.tiny_system()
        nbs = 21
        f = synth.fermi_occupations(1, 1, nbs)
    else:
        s0 = synth.rt_system()
        s = synth.System(s0.grid, s0.atoms, s0.radials, s0.kpts[:1], np.ones(1), nspin=1)
        nbs = 1
        f = np.full((1, 1, nbs), 1.0)
    st = O.setup_atoms(s)
    coul = _oracle_coulomb(O, s, st)
    # seeded random states (the oracle's cost does not depend on their values)
    rng = np.random.default_rng(11)
    shape = (s.nk, s.nspin, nbs, s.grid.npts)
    psi = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * math.sqrt(0.5 / (s.grid.npts * s.grid.dV))
    t0 = time.perf_counter()
    reps = 0
    while True:
        if kind == "rt_prefix":
            x = psi
            for _ in range(10):
                x, _ = O.taylor_step(s, st, x, f, 0.01, coulomb=coul)
        else:
            O.hubbard_pass(s, st, psi, f, coulomb=coul)
        reps += 1
        if time.perf_counter() - t0 > target_s:
            break
    dt = (time.perf_counter() - t0) / reps
    pts = sum(len(x["idx"]) for x in st)
    ns = 1 if kind == "rt_prefix" else (2 if kind == "oxide" else 1)
    if kind == "rt_prefix":
        bytes_ = 10 * 3 * pts * 16 * nbs            # per step one gather and one read-modify-write of the sphere points
    else:
        bytes_ = 3 * pts * 16 * nbs * ns
    return {"kind": kind, "s_per_rep": round(dt, 4), "reps": reps, "GBps": round(bytes_ / dt / 1e9, 4),
            "bytes_per_rep": int(bytes_)}


def _cpu_sample_subprocess(kind: str, target_s: float, threads=None) -> dict:
    """cpu_sample in a fresh interpreter, with the BLAS/OpenMP thread count pinned when given."""
    env = dict(os.environ)
    if threads is not None:
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
            env[k] = str(threads)
    code = f"import json, bench; print(json.dumps(bench.cpu_sample({kind!r}, {target_s!r})))"
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        return {"kind": kind, "error": (r.stderr or r.stdout)[-300:]}
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_baseline(args, s, target_s=8.0):
    """The CPU FP64 oracle, as it stands, on bounded samples: the headline figure is the oxide sample on
    all host cores; the same sample on one thread, the one-atom case and a 10-step real-time prefix are
    reported beside it."""
    cores = os.cpu_count()
    ox = _cpu_sample_subprocess("oxide", target_s)
    ox1 = _cpu_sample_subprocess("oxide", target_s, threads=1)
    tiny = _cpu_sample_subprocess("tiny", 2.0)
    tiny1 = _cpu_sample_subprocess("tiny", 2.0, threads=1)
    rt = _cpu_sample_subprocess("rt_prefix", 1.0)
    out = {"value": ox.get("GBps"), "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"1 k-point x 2 spins x 4 bands of the same 96^3 oxide workload, full pass, {ox.get('reps')} reps, "
                     f"{ox.get('s_per_rep')} s/pass, numpy BLAS on all {cores} host cores",
           "single_thread": ox1, "tiny_all_cores": tiny, "tiny_single_thread": tiny1, "rt_10_step_prefix_all_cores": rt}
    return out


def _coulomb_all(h, system):
    for sp in range(len(system.radials)):
        h.coulomb_integrals(sp)


def _sphere_bytes(h, natoms):
    return int(sum(h.lib.dftu_atom_points(h.h, i) for i in range(natoms)))


def run_rt(args):
    """Real-time TDDFT+U steps: 64 atoms of 3 species (radii 3.5/4.5/5.0) on a periodic 128^3 grid,
    512 complex64 bands, 4 k-points; 4th-order Taylor step with V_U rebuilt (occupations, ACBN0 U and J)
    from the incoming states every step; `rt_steps` steps captured as ONE CUDA graph."""
    import torch
    from paper_1711_08935_gb300 import dftu, synth
    dev = torch.device("cuda", 0)
    s = synth.rt_system(n=args.grid if args.grid != 96 else 128)
    nb = args.nbands if args.nbands != 256 else 512
    t0 = time.time()
    psi = synth.make_states(s, nb, seed=4, device=dev).to(torch.complex64)
    torch.cuda.empty_cache()
    gen_s = time.time() - t0
    f = torch.from_numpy(synth.step_occupations(s.nk, 1, nb, nb // 2)).to(dev)
    h = dftu.handle_for_system(s, nb)
    _coulomb_all(h, s)
    # kernel shapes tuned on these states (the tuner's applies go into a scratch buffer freed afterwards)
    from paper_1711_08935_gb300.autotune import autotune
    h.project(psi); h.occupations(f); h.acbn0_uj()
    tuned = None
    if not args.no_tune:
        scratch = torch.zeros_like(psi)
        tuned = autotune(h, psi, out=scratch)
        del scratch
        torch.cuda.empty_cache()
    n0 = (psi.abs() ** 2).sum(-1).double() * s.grid.dV
    dt = 0.01
    S = _sphere_bytes(h, len(s.atoms))
    unit = S * 8 * nb * s.nk                      # one read of every sphere point of every state (complex64)

    def graph_of(fn, warm):
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(args.warmup):
                warm()
        torch.cuda.current_stream().wait_stream(side)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fn()
        torch.cuda.synchronize()
        return g

    def time_graph(g, sampler=None):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if sampler:
            sampler.mark()
        e0.record()
        g.replay()
        e1.record()
        torch.cuda.synchronize()
        if sampler:
            sampler.mark()
        return e0.elapsed_time(e1)

    # all steps in one dftu_taylor_steps call: each step's scatter also gathers the updated states for the
    # next step, so a step reads and writes every sphere point once (plus the first step's gather)
    g = graph_of(lambda: h.taylor_steps(psi, f, dt, args.rt_steps), lambda: h.taylor_steps(psi, f, dt, 1))
    clocks = ClockSampler(0)
    clocks.start()
    ms = time_graph(g, clocks) / args.rt_steps
    clk = clocks.stop()
    n1 = (psi.abs() ** 2).sum(-1).double() * s.grid.dV
    del g
    # the same steps one projection and one apply at a time (dftu_taylor_step), for comparison
    n_single = max(10, args.rt_steps // 4)
    g1 = graph_of(lambda: [h.taylor_step(psi, None, f, dt) for _ in range(n_single)], lambda: h.taylor_step(psi, None, f, dt))
    ms1 = time_graph(g1) / n_single
    del g1

    def ceiling_ms(rmw, reps=5):
        for _ in range(2):
            h.access_ceiling(psi, rmw)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for e0, e1 in evs:
            e0.record()
            h.access_ceiling(psi, rmw)
            e1.record()
        torch.cuda.synchronize()
        return statistics.median(e0.elapsed_time(e1) for e0, e1 in evs)

    gather_ms, rmw_ms = ceiling_ms(False), ceiling_ms(True)
    step_bytes = 2 * unit + unit / args.rt_steps   # read + write of every sphere point per step, first gather
    peak, src = measured_peaks()
    return ({
        "metric": METRIC, "value": round(step_bytes / (ms * 1e-3) / 1e9, 2), "unit": UNIT, "n_gpus": 1,
        "steps": args.rt_steps, "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64 states, FP32 with FP64 cross-tile sums", "data": "synthetic",
        "config": {"workload": "real-time Taylor-4 steps: 64 atoms / 3 species (R 3.5/4.5/5.0), periodic 128^3 h=0.3, "
                               "512 c64 bands, 4 k, V_U and ACBN0 U/J rebuilt every step, all steps in one CUDA graph",
                   "sphere_points_sum": S, "steps_in_graph": args.rt_steps, "dt": dt},
        "bytes_per_step": "2 state passes (the scatter of step s gathers for step s+1) + the first gather / steps",
        "steps_per_s": round(1e3 / ms, 2), "graph_ms_total": round(ms * args.rt_steps, 2),
        "one_step_at_a_time": {"ms_per_step": round(ms1, 4), "steps": n_single,
                               "GBps": round(3 * unit / (ms1 * 1e-3) / 1e9, 2),
                               "note": "dftu_taylor_step per step: one projection and one apply (3 state passes)",
                               "speedup_of_fused": round(ms1 / ms, 3)},
        "access_ceiling": {"c64_gather_GBps": round(unit / (gather_ms * 1e-3) / 1e9, 1),
                           "c64_rmw_GBps": round(2 * unit / (rmw_ms * 1e-3) / 1e9, 1),
                           "step_floor_ms": round(rmw_ms, 4),
                           "frac_of_ceiling": round(rmw_ms / ms, 4)},
        "norm_drift_max": float((n1 - n0).abs().max()), "state_generation_s": round(gen_s, 1),
        "peak": peak, "peak_source": src, "frac_of_peak": round(step_bytes / (ms * 1e-3) / 1e9 / peak, 4), "clocks": clk,
        "U_eV_first_atoms": [round(x * dftu.HARTREE_EV, 5) for x in h.results()["U"][:6]], "tuning": tuned})


def run_molecules(args):
    """Many independent molecules: 256 isolated systems (edges 48-80 points at 0.3 bohr, 1-8 d shells,
    R 4-5, 20-200 states, Gamma, collinear spin).  One persistent launch per streaming kernel over all
    members (complex64 states) against one-by-one launches; FP64 one-by-one on a 64-molecule subset."""
    import torch
    from paper_1711_08935_gb300 import dftu, synth
    dev = torch.device("cuda", 0)
    systems = synth.molecule_systems(args.nsys)
    hs, psis, fs = [], [], []
    t0 = time.time()
    for i, s in enumerate(systems):
        nb = synth.bands_of(s)
        h = dftu.handle_for_system(s, nb)
        _coulomb_all(h, s)
        hs.append(h)
        psis.append(synth.make_states(s, nb, seed=1000 + i, device=dev).to(torch.complex64))
        fs.append(torch.from_numpy(synth.step_occupations(1, 2, nb, nb // 2)).to(dev))
    torch.cuda.empty_cache()
    gen_s = time.time() - t0
    S = [_sphere_bytes(h, len(s.atoms)) for h, s in zip(hs, systems)]
    nbs = [synth.bands_of(s) for s in systems]

    def pass_bytes(idx, bpp):
        return sum(3 * S[i] * bpp * nbs[i] * 2 for i in idx)

    def time_it(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    batch = dftu.Batch(hs)
    batch.bind(psis, fs)
    # the batch applies in place onto the bound states, so each step is a first-order real-time update
    # psi += -i dt V_U psi (dt = 0.01 a.u.), which keeps the states bounded over the repeated steps
    cdt = torch.tensor([-0.01j], dtype=torch.complex128, device=dev)
    from paper_1711_08935_gb300.autotune import autotune_batch
    batch.project(); batch.occupations(); batch.acbn0_uj()
    tuned = autotune_batch(batch, torch.complex64, cdt)
    for hh in hs:   # the one-by-one comparison runs with the same shapes
        hh.set_kernel_variant(1, tuned["project"]["variant"])
        hh.set_kernel_variant(3, tuned["apply"]["variant"])

    def batched():
        batch.project(); batch.occupations(); batch.acbn0_uj(); batch.apply(cdt)

    def one_by_one(idx, ps):
        for i in idx:
            hs[i].project(ps[i]); hs[i].occupations(fs[i]); hs[i].acbn0_uj(); hs[i].apply(ps[i], cdt)

    allidx = list(range(len(systems)))
    clocks = ClockSampler(0)
    clocks.start()
    clocks.mark()
    ms_b = time_it(batched, args.steps, args.warmup)
    # where a batched pass spends its time (CUDA events between the calls of one pass, after the timed ones)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    evs[0].record(); batch.project(); evs[1].record(); batch.occupations(); evs[2].record()
    batch.acbn0_uj(); evs[3].record(); batch.apply(cdt); evs[4].record()
    torch.cuda.synchronize()
    phases = {n: round(evs[i].elapsed_time(evs[i + 1]), 4) for i, n in enumerate(("project", "occupations", "acbn0", "apply"))}
    clocks.mark()
    clk = clocks.stop()
    ms_1 = time_it(lambda: one_by_one(allidx, psis), max(1, args.steps // 2), 1)
    batch.close()
    # FP64 one-by-one on a subset, against the same subset batched in complex64 and complex128
    sub = allidx[:min(64, len(allidx))]
    p64 = [psis[i].to(torch.complex128) for i in sub]
    ps64 = {i: p for i, p in zip(sub, p64)}
    ms_sub64 = time_it(lambda: one_by_one(sub, ps64), max(1, args.steps // 2), 1)
    bsub = dftu.Batch([hs[i] for i in sub])
    bsub.bind(p64, [fs[i] for i in sub])
    ms_sub64_b = time_it(lambda: (bsub.project(), bsub.occupations(), bsub.acbn0_uj(), bsub.apply(cdt)), args.steps, 1)
    bsub.close()
    del p64, ps64
    bsub32 = dftu.Batch([hs[i] for i in sub])
    bsub32.bind([psis[i] for i in sub], [fs[i] for i in sub])
    ms_sub32_b = time_it(lambda: (bsub32.project(), bsub32.occupations(), bsub32.acbn0_uj(), bsub32.apply(cdt)), args.steps, 1)
    bsub32.close()
    peak, src = measured_peaks()
    val = pass_bytes(allidx, 8) / (ms_b * 1e-3) / 1e9
    return ({
        "metric": METRIC, "value": round(val, 2), "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms_b, 4), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64 states, FP32 with FP64 cross-tile sums", "data": "synthetic",
        "config": {"workload": f"{len(systems)} isolated molecules (edge 48-80 pts, h=0.3, 1-8 d shells R 4-5, 20-200 states, "
                               "Gamma, collinear), one persistent launch per streaming kernel",
                   "atoms": sum(len(s.atoms) for s in systems), "sphere_points": sum(S), "states": 2 * sum(nbs)},
        "one_by_one_c64_ms": round(ms_1, 3), "batched_speedup_vs_one_by_one_c64": round(ms_1 / ms_b, 3),
        "batched_phases_ms": phases,
        "subset64": {"systems": len(sub), "one_by_one_c128_ms": round(ms_sub64, 3), "batched_c128_ms": round(ms_sub64_b, 3),
                     "batched_c64_ms": round(ms_sub32_b, 3),
                     "batched_c64_speedup_vs_one_by_one_fp64": round(ms_sub64 / ms_sub32_b, 3),
                     "GBps_batched_c64": round(pass_bytes(sub, 8) / (ms_sub32_b * 1e-3) / 1e9, 1),
                     "GBps_one_by_one_c128": round(pass_bytes(sub, 16) / (ms_sub64 * 1e-3) / 1e9, 1)},
        "peak": peak, "peak_source": src, "frac_of_peak": round(val / peak, 4), "clocks": clk,
        "state_generation_s": round(gen_s, 1), "tuning": tuned})


def run_nc(args):
    """Non-collinear pass: 10 Bi-like p shells (Z_eff 2, R 4.5) on the periodic 96^3 grid, 128 spinor
    bands, 6 k-points; complex128 (FP32-pair) and complex64 forms."""
    import torch
    from paper_1711_08935_gb300 import dftu, synth
    dev = torch.device("cuda", 0)
    s = synth.noncollinear_system()
    nb = args.nbands if args.nbands != 256 else 128
    psi = synth.make_states(s, nb, seed=3, device=dev)
    f = torch.from_numpy(np.ones((s.nk, nb)) * (np.arange(nb) < nb // 2)).to(dev)
    h = dftu.handle_for_system(s, nb)
    _coulomb_all(h, s)
    from paper_1711_08935_gb300.autotune import autotune
    psi32 = psi.to(torch.complex64)              # same states for both forms, before any apply
    h.project(psi); h.occupations(f); h.acbn0_uj()
    r64 = h.results()
    h.project(psi32); h.occupations(f); h.acbn0_uj()
    r32 = h.results()
    hpsi, hpsi32 = torch.zeros_like(psi), torch.zeros_like(psi32)   # H psi buffers: the states stay as generated
    autotune(h, psi, out=hpsi)
    autotune(h, psi32, out=hpsi32)

    def t(x, out):
        for _ in range(args.warmup):
            h.project(x); h.occupations(f); h.acbn0_uj(); h.apply(out)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            h.project(x); h.occupations(f); h.acbn0_uj(); h.apply(out)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    clocks = ClockSampler(0)
    clocks.start()
    clocks.mark()
    ms64 = t(psi, hpsi)
    clocks.mark()
    clk = clocks.stop()
    ms32 = t(psi32, hpsi32)
    S = _sphere_bytes(h, len(s.atoms))
    b64 = 3 * S * 16 * nb * s.nk * 2
    peak, src = measured_peaks()
    return ({
        "metric": METRIC, "value": round(b64 / (ms64 * 1e-3) / 1e9, 2), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms64, 4), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c128 spinors; FP32-pair arithmetic", "data": "synthetic",
        "config": {"workload": "non-collinear: 10 p shells (Z 2, R 4.5), periodic 96^3 h=0.25, 128 spinor bands, 6 k",
                   "sphere_points": S},
        "fp32_state": {"ms_per_step": round(ms32, 4), "speedup_vs_fp64": round(ms64 / ms32, 3),
                       "max_abs_dn": max(float(np.max(np.abs(a - b))) for a, b in zip(r64["n"], r32["n"])),
                       "max_dU_eV": float(np.max(np.abs(r64["U"] - r32["U"]))) * dftu.HARTREE_EV},
        "peak": peak, "peak_source": src, "frac_of_peak": round(b64 / (ms64 * 1e-3) / 1e9 / peak, 4), "clocks": clk})


def run_gauge(args):
    """The headline oxide pass with the gauge-invariant operator of Sec. V (Eq. 16): every step sets the
    vector potential (phase table kernel), projects with the phases, builds occupations and U/J, and
    applies with the conjugate phases; the Hubbard current of Eq. (17) is timed separately.  The plain
    pass (tuned shapes) runs on the same states for comparison."""
    import torch
    from paper_1711_08935_gb300 import dftu, synth
    dev = torch.device("cuda", 0)
    s = synth.oxide_system(n=args.grid, nk=args.nkgrid)
    nb = args.nbands
    psi = synth.make_states(s, nb, seed=2, device=dev, spin_bias=synth.afm_spin_bias(s))
    f = torch.from_numpy(synth.step_occupations(s.nk, 2, nb, nb // 2)).to(dev)
    h = dftu.handle_for_system(s, nb)
    _coulomb_all(h, s)
    npts = [h.lib.dftu_atom_points(h.h, i) for i in range(len(s.atoms))]
    orb_bytes = sum(n * (2 * a.l + 1) * 8 for n, a in zip(npts, s.atoms))
    pb, ab = algorithmic_bytes(npts, nb, s.nk, 2, 16, orb_bytes)
    gauge_bytes = int(sum(npts)) * 16                 # the phase table, read once per projection and apply
    A = torch.tensor([0.3, -0.2, 0.25], dtype=torch.float64, device=dev)
    psi32 = psi.to(torch.complex64)
    hpsi = torch.zeros_like(psi)                     # H psi accumulates V_U psi; the states stay as generated
    from paper_1711_08935_gb300.autotune import autotune
    h.project(psi); h.occupations(f); h.acbn0_uj()     # the tuner's apply needs a potential
    tuned = {"c128": autotune(h, psi, out=hpsi)}
    stream = torch.cuda.current_stream(dev)

    def timed(x, out, gauge, steps, warmup):
        def one(evs=None):
            if gauge:
                h.set_vector_potential(A)
            if evs: evs[0].record(stream)
            h.project(x)
            if evs: evs[1].record(stream)
            h.occupations(f); h.acbn0_uj()
            if evs: evs[2].record(stream)
            h.apply(out)
            if evs: evs[3].record(stream)
        for _ in range(warmup):
            one()
        torch.cuda.synchronize()
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(steps):
            one(ev[i])
        e1.record(stream)
        torch.cuda.synchronize()
        return (e0.elapsed_time(e1) / steps, statistics.mean(e[0].elapsed_time(e[1]) for e in ev),
                statistics.mean(e[2].elapsed_time(e[3]) for e in ev))

    ms_plain, pr_plain, ap_plain = timed(psi, hpsi, False, args.steps, args.warmup)
    clocks = ClockSampler(0)
    clocks.start()
    clocks.mark()
    ms_g, pr_g, ap_g = timed(psi, hpsi, True, args.steps, args.warmup)
    clocks.mark()
    clk = clocks.stop()
    # Hubbard current: three projections onto the displaced orbitals + the contraction, blocking
    h.set_vector_potential(A); h.project(psi); h.occupations(f); h.acbn0_uj()
    for _ in range(2):
        h.hubbard_current(psi, f)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    reps = max(2, args.steps // 2)
    for _ in range(reps):
        J = h.hubbard_current(psi, f)
    cur_ms = (time.perf_counter() - t0) * 1e3 / reps
    del hpsi
    hpsi32 = torch.zeros_like(psi32)
    ms_g32, pr_g32, ap_g32 = timed(psi32, hpsi32, True, args.steps, args.warmup)
    status = h.sync_status()
    peak, src = measured_peaks()
    step_bytes = pb + ab + 2 * gauge_bytes
    dom_is_apply = ap_g >= pr_g
    dom_b = (ab + gauge_bytes) if dom_is_apply else (pb + gauge_bytes)
    dom_ms = ap_g if dom_is_apply else pr_g
    achieved = dom_b / (dom_ms * 1e-3) / 1e9
    return ({
        "metric": METRIC, "value": round(step_bytes / (ms_g * 1e-3) / 1e9, 2), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_g, 4), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c128 states; FP32-pair arithmetic, gauge phases as FP32 pairs", "data": "synthetic",
        "config": {"workload": "gauge-invariant pass (Sec. V): oxide supercell 96^3 h=0.25, 8 TM(3d,R4.5)+8 O(2p,R3.5), "
                               "256 bands, 8 k, collinear, A=(0.3,-0.2,0.25) a.u. set every step",
                   "sphere_points": int(sum(npts)), "l2": "inputs (58 GB of states) far larger than L2; no flush needed"},
        "roofline": {"bound": "hbm", "kernel": "apply (gauge)" if dom_is_apply else "project (gauge)",
                     "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "peak_source": src, "traffic": (round(NCU_TRAFFIC_PER_STATE_GAUGE["apply" if dom_is_apply else "project"]
                                                           * nb * s.nk * 2)
                                                     if NCU_TRAFFIC_PER_STATE_GAUGE["apply" if dom_is_apply else "project"]
                                                     else None), "bytes_per_launch": dom_b},
        "kernels_ms": {"project_gauge": round(pr_g, 4), "apply_gauge": round(ap_g, 4), "project_plain": round(pr_plain, 4),
                       "apply_plain": round(ap_plain, 4)},
        "plain_pass_ms": round(ms_plain, 4), "gauge_overhead": round(ms_g / ms_plain, 3),
        "current": {"ms": round(cur_ms, 3), "J": [float(x) for x in J], "note": "one launch projecting onto the three displaced-orbital tables + contraction + host copy, blocking"},
        "fp32_state": {"ms_per_step": round(ms_g32, 4), "project_ms": round(pr_g32, 4), "apply_ms": round(ap_g32, 4)},
        "tuning": tuned, "gpu_launches": (1 + 2 + 2 + 2 + 2) * args.steps, "device_status": int(status), "clocks": clk})


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    from paper_1711_08935_gb300 import synth
    s = synth.oxide_system(n=args.grid, nk=args.nkgrid)
    from oracle import dftu_oracle as O
    st = O.setup_atoms(s)
    coul = []
    for sp in range(len(s.radials)):
        I = [a.species for a in s.atoms].index(sp)
        coul.append(O.coulomb_integrals(s.grid, s.atoms[I], st[I]))
    nbs = 2
    sub = synth.System(s.grid, s.atoms, s.radials, s.kpts[:1], np.ones(1), nspin=2)
    psi = synth.make_states(sub, nbs, seed=11, device="cpu").numpy()
    f = np.ones((1, 2, nbs))
    for _ in range(args.warmup):
        O.hubbard_pass(sub, st, psi, f, coulomb=coul)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.hubbard_pass(sub, st, psi, f, coulomb=coul)
    dt = (time.perf_counter() - t0) / args.steps
    pts = sum(len(x["idx"]) for x in st)
    value = 3 * pts * 16 * nbs * 2 / dt / 1e9
    try:
        import threadpoolctl
        cores = max(i.get("num_threads", 1) for i in threadpoolctl.threadpool_info()) or 1
    except Exception:
        cores = os.cpu_count()
    sample = f"1 k-point x 2 spins x {nbs} bands of the 96^3 oxide workload per step (full pass)"
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": ws,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 2), "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                      "config": {"workload": WORKLOAD}, "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": cores,
                                                                         "kind": "oracle", "sample": sample},
                      "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--grid", type=int, default=96)
    ap.add_argument("--nkgrid", type=int, default=2)
    ap.add_argument("--nbands", type=int, default=256)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--variants", default="", help="fixed kernel variants 'p128,p64,a128,a64' instead of tuning")
    ap.add_argument("--workload", default="oxide", choices=["oxide", "rt", "molecules", "nc", "gauge"],
                    help="oxide: the headline pass; rt / molecules / nc / gauge: the other workloads, one JSON line each")
    ap.add_argument("--rt-steps", type=int, default=200)
    ap.add_argument("--nsys", type=int, default=256)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the native-FP64 pass and the non-collinear, real-time and molecule workloads")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "rt":
        print(json.dumps(run_rt(args)))
    elif args.workload == "molecules":
        print(json.dumps(run_molecules(args)))
    elif args.workload == "nc":
        print(json.dumps(run_nc(args)))
    elif args.workload == "gauge":
        print(json.dumps(run_gauge(args)))
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
