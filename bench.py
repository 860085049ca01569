"""Benchmark: LJ lj/cut step on the 4,000,000-atom fcc liquid (100^3 cells),
Matom-steps/s on one GB300, FP64 (headline) and mixed precision, with the
pair kernel's roofline, an end-to-end host-buffer figure and the CPU oracle
as a reported baseline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

A step is one velocity-Verlet NVE step of the whole path: the fused
integrator, the pair force kernel and, every 20th step, the rebuild (wrap,
cell sort, neighbor build).  With N > 1 (torchrun, one rank per GPU) each
rank runs its own copy of the box (independent replicas, weak scaling); the
only collectives are the timing barrier and the max over ranks.

``--impl reference`` times the FP64 CPU oracle instead (rank 0 only), one
oracle step per bench step on a 32,000-atom periodic sample of the same
liquid (the oracle's cost per atom-step does not depend on the box size).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "LJ Matom-steps/s at 4M atoms, FP64 vs mixed, and % of HBM roofline on 1 GB300"
UNIT = "Matom-steps/s"
N_CELLS = 100  # 4 * 100^3 = 4,000,000 atoms
HBM_PEAK_FALLBACK = 6800.0
SM_COUNT = 152
FP64_OPS_PER_CLK_SM = 2  # FP64 pipe lane-ops per clock per SM (1.25 TFLOP/s nominal)

# DRAM bytes (read + write) per atom of one pair-kernel launch from 1-pass
# ncu captures at 4,000,000 atoms (commands and figures under profiles/),
# keyed by form, compacted mode, threads per atom and list entries per filter
# round (md_stats.phase1_entries).  They hold
# only for the kernel source they were taken on (hash of the files below);
# for any other source or configuration the traffic is reported as null.
PAIR_SOURCES = ("paper_2508_13523_gb300/csrc/md_pair.cuh",
                "paper_2508_13523_gb300/csrc/md_pair_q.cuh",
                "paper_2508_13523_gb300/csrc/md_device.cuh")
PAIR_TRAFFIC = {"349e1dd95a9eed30": {
    "fp64_half/2/1/2": (1422190336 + 92602112) / 4.0e6,
    "fp64_full/2/1/2": (1768076288 + 86858752) / 4.0e6,
    "mixed_half/0/2/2": (1083237888 + 83930112) / 4.0e6,
    "mixed_full/0/2/2": (1417269504 + 76367360) / 4.0e6}}


def pair_source_hash() -> str:
    """Hash of the pair kernels' sources with // comments and all white space
    removed: an edit of comments or layout leaves it unchanged."""
    import hashlib
    import re
    h = hashlib.sha1()
    for f in PAIR_SOURCES:
        with open(os.path.join(ROOT, f)) as fh:
            code = re.sub(r"//[^\n]*", "", fh.read())
        h.update(re.sub(r"\s+", "", code).encode())
    return h.hexdigest()[:16]


def pair_traffic(form: str, compacted: int, tpa: int, qu: int, n: int):
    per_atom = PAIR_TRAFFIC.get(pair_source_hash(), {}).get(f"{form}/{compacted}/{tpa}/{qu}")
    return None if per_atom is None else per_atom * n


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), float(d.get("sm_max_mhz", 2070.0)), "measured"
    except (OSError, KeyError, ValueError):
        return HBM_PEAK_FALLBACK, 2070.0, "fallback"


# ---- clocks during the timed region -------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"bench_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.25)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        try:
            self.fh.close()
        except Exception:
            pass

    def summary(self):
        rows = []
        try:
            with open(self.path) as fh:
                for line in fh:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
        except OSError:
            pass
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        loaded = [s for s in sm if mx and s >= 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ---- distributed plumbing ------------------------------------------------------

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, value: float) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64,
                     device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---- algorithmic work of the pair kernel ---------------------------------------

def fp64_ops_per_pair(compacted: int, coul: bool = False) -> int:
    """FP64-pipe operations per visit of a pair inside rc.

    With floating-point separations (per-atom kernel, compacted kernel with
    FP64 sums): separation 3, squared length 3, reciprocal refinement 3,
    r^-6 2, fpair 3, fpair * d 3 = 17 (the accumulations are reductions in
    L2, off the pipe).  The compacted kernel with fixed-point sums forms the
    separation, r^2 and fpair * d from exact fixed-point positions with
    integer instructions, leaving reciprocal 3, r^-6 2, fpair 3 = 8.  The
    lj/cut/coul/cut form takes 22 (reciprocal square root 5, r^-2 1, qq/r 1,
    one FMA, instead of the reciprocal's 3) on the floating-point path,
    which it always uses."""
    if coul:
        return 22
    return 8 if compacted == 2 else 17


def pair_work(kind: str, prec: str, n: int, entries: int, pairs: int, compacted: int = 0,
              coul: bool = False):
    """FP64-pipe operations and compulsory DRAM bytes of one pair launch.

    FP64 operations: fp64_ops_per_pair per visit of a pair inside rc; listed
    pairs outside rc need none (a certified FP32 test rejects them).  A full
    list visits each pair twice, a half list once.  The mixed form issues no
    FP64 operation per pair.  Bytes: per atom the position record (32), the
    two row counts (8) and the force (24 written; with reductions 24 zeroed +
    48 read-modify-write), plus 4 per list entry; gathered positions are
    assumed to hit in cache."""
    half = kind == "half"
    visits = pairs if half else 2 * pairs
    ops = 0 if prec == "mixed" else fp64_ops_per_pair(compacted, coul) * visits
    atomics = half or prec == "fp64"  # the FP64 kernels reduce into f in L2
    per_atom = 32 + 8 + (24 + 48 if atomics else 24)
    return ops, n * per_atom + 4 * entries


def step_bytes_per_atom(kind: str, entries_per_atom: float, every: int = 20) -> float:
    """Compulsory bytes per atom-step of the whole step: the pair launch, the
    integrator (x r/w 64, v r/w 48, f r 24, split w 32, build snapshot r 32)
    and the rebuild amortized over `every` steps (~600 B per atom plus the
    list write)."""
    half = kind == "half"
    pair = 32 + 8 + (72 if half else 24) + 4 * entries_per_atom
    integ = 64 + 48 + 24 + 32 + 32
    rebuild = (600 + 4 * entries_per_atom) / every
    return pair + integ + rebuild


# ---- one measured form -----------------------------------------------------------

COUL_Q = (0.5, -0.5)  # lj/cut/coul/cut form: charges of the two fcc site types


def kernel_code(st, persistent: int = 0) -> int:
    """md_set_kernel's `compacted` argument for the kernel md_get_stats reports
    (3: the fixed-point kernel with two list entries per filter round; the
    one-launch-per-step schedule, persistent 2, has one entry a round)."""
    two = st["compacted"] == 2 and st["phase1_entries"] == 2 and persistent != 2
    return 3 if two else st["compacted"]


def run_form(md, sysm, kind, prec, K, W, pair_reps, sampler_gpu=None, compacted=-1, tpa=0,
             carveout=-1, persistent=False, coul=False, drift=True):
    import torch
    lk = md.MD_LIST_HALF if kind == "half" else md.MD_LIST_FULL
    pr = md.MD_PREC_MIXED if prec == "mixed" else md.MD_PREC_FP64
    if coul:
        # the same liquid with two types by fcc basis site (0, 1 | 2, 3), equal
        # LJ parameters, charges +-0.5, rc_coul = rc = 2.5
        t2 = (np.arange(sysm.n) % 4 >= 2).astype(np.int32)
        ctx = md.LJMD(sysm.x, sysm.v, t2, sysm.box, 1.0, 1.0, 2.5, [1.0, 1.0], list_kind=lk,
                      precision=pr, threads_per_atom=max(tpa, 1))
        ctx.set_coulomb(COUL_Q, 2.5)
        if tpa == 0:
            ctx.autotune()
        ctx.compute_forces(0)
    else:
        ctx = md.from_system(sysm, list_kind=lk, precision=pr, threads_per_atom=tpa)
    if compacted > 0 and prec == "fp64":  # a fixed kernel instead of the tuner's choice
        ctx.set_kernel(1, -1, compacted, 0)
        ctx.compute_forces(0)
    if carveout >= 0 or persistent:  # carveout (%) / per-SM tile scheduling of the pair kernel
        st = ctx.stats()
        ctx.set_kernel(st["threads_per_atom"], carveout, kernel_code(st, int(persistent)),
                       int(persistent))
        ctx.compute_forces(0)
    stream = ctx.stream
    ctx.step(W)
    ctx.synchronize()
    l0 = ctx.stats()["kernel_launches"]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    clocks = None
    sampler = ClockSampler(sampler_gpu) if sampler_gpu is not None else None
    if sampler:
        sampler.__enter__()
    torch.cuda.synchronize()
    e0.record(stream)
    ctx.step(K)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    if sampler:
        sampler.__exit__(None, None, None)
        clocks = sampler.summary()
    ms = e0.elapsed_time(e1)
    st = ctx.stats()
    launches = st["kernel_launches"] - l0 - 1  # minus the stats call's own count kernel
    # the pair kernel alone, same stream, same configuration
    th = ctx.energy()
    st = ctx.stats()
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    ctx.compute_forces(0)
    p0.record(stream)
    for _ in range(pair_reps):
        ctx.compute_forces(0)
    p1.record(stream)
    p1.synchronize()
    pair_ms = p0.elapsed_time(p1) / pair_reps
    # the same launch with energy and virial (md_energy's force pass)
    ctx.compute_forces(md.MD_ENERGY | md.MD_VIRIAL)
    p0.record(stream)
    for _ in range(pair_reps):
        ctx.compute_forces(md.MD_ENERGY | md.MD_VIRIAL)
    p1.record(stream)
    p1.synchronize()
    ev_ms = p0.elapsed_time(p1) / pair_reps
    # the pair kernel alone inside steps: CUDA events on the context's stream
    # around each pair launch of 10 steps (md_time_pair_kernel: the same
    # kernels, launched without the segment graphs)
    ctx.time_pair_kernel(True)
    ctx.step(10)
    tot, cnt = ctx.pair_kernel_time()
    ctx.time_pair_kernel(False)
    pair_step_ms = tot / cnt if cnt else None
    # one neighbor rebuild (wrap, sort, build; it synchronizes once to check
    # the list capacity), host-timed, median of 3
    rb = []
    for _ in range(3):
        ctx.synchronize()
        t0 = time.perf_counter()
        ctx.build_neighbors()
        ctx.synchronize()
        rb.append((time.perf_counter() - t0) * 1e3)
    rebuild_ms = sorted(rb)[1]
    ctx.compute_forces(0)
    e_drift = None
    if drift:
        # total-energy drift: 100 further steps, E_tot every 10 steps, slope
        # of a linear fit per atom and step (the unshifted cutoff makes it
        # nonzero); the long run is the --drift-steps leg
        e = []
        for k in range(11):
            e.append(ctx.energy().etot / sysm.n)
            if k < 10:
                ctx.step(10)
        e_drift = float(np.polyfit(np.arange(0, 101, 10), np.array(e), 1)[0])
    out = dict(ctx=ctx, ms=ms, launches=launches, clocks=clocks, pair_ms=pair_ms, ev_ms=ev_ms,
               pair_step_ms=pair_step_ms,
               rebuild_ms=rebuild_ms, energy_drift=e_drift,
               entries=st["list_entries"], pairs=st["pairs_in_range"], tpa=st["threads_per_atom"],
               compacted=st["compacted"], carveout=st["carveout"], persistent=st["persistent"],
               phase1_entries=st["phase1_entries"], dangerous=st["dangerous_builds"], builds=st["builds"], thermo=th)
    return out


# ---- long energy-drift runs (the mixed-precision workload's drift) -------------

def lj_u(r: float) -> float:
    """Eq. 1 pair energy with eps = sigma = 1."""
    return 4.0 * (r ** -12 - r ** -6)


def drift_summary(steps, etot, npairs, n, rc=2.5):
    """Energy drift of one run sampled at `steps`: the least-squares slope of
    E_tot/N per step and max |E(t) - E(0)| / |E(0)| for E_tot (Eq. 1,
    truncated: it jumps by -U(rc) whenever a pair crosses rc), and the same
    for H = E_tot - n_pairs U(rc) (n_pairs: pairs with r < rc), the energy of
    the cut-and-shifted potential, which the truncated-force dynamics
    conserve exactly: its drift is the integrator's and the arithmetic's
    alone."""
    steps = np.asarray(steps, dtype=np.float64)
    e = np.asarray(etot, dtype=np.float64)
    h = e - np.asarray(npairs, dtype=np.float64) * lj_u(rc)

    def one(y):
        return {"slope_per_atom_step": float(np.polyfit(steps, y / n, 1)[0]),
                "max_rel_dev": float(np.max(np.abs(y - y[0])) / abs(y[0]))}
    return {"steps": int(steps[-1]), "samples": int(steps.size),
            "etot": one(e), "shifted": one(h)}


def run_drift(md, sysm, forms, nsteps, every=100):
    """Each form from the same initial state (the fcc liquid at T* = 1.44),
    nsteps velocity-Verlet steps, E_tot and the pairs inside rc every `every`
    steps (md_energy recomputes the forces at the current positions; the
    fixed-point force sums make that recomputation bit-identical, so sampling
    does not perturb the trajectory).  Also: the mixed forms' final E_tot
    against the FP64 form's."""
    out = {}
    for name in forms:
        prec, kind = name.split("_")[:2]
        ctx = md.from_system(sysm, list_kind=md.MD_LIST_HALF if kind == "half" else
                             md.MD_LIST_FULL, precision=md.MD_PREC_MIXED if prec == "mixed"
                             else md.MD_PREC_FP64, threads_per_atom=0)
        steps, e, npr = [], [], []
        t0 = time.perf_counter()
        for k in range(nsteps // every + 1):
            th = ctx.energy()
            steps.append(k * every)
            e.append(th.etot)
            npr.append(ctx.stats()["pairs_in_range"])
            if k < nsteps // every:
                ctx.step(every)
        ctx.synchronize()
        wall = time.perf_counter() - t0
        d = drift_summary(steps, e, npr, sysm.n)
        d["wall_s"] = wall
        d["e_final_per_atom"] = e[-1] / sysm.n
        out[name] = d
        ctx.close()
    ref = out.get("fp64_half")
    for name, d in out.items():
        if ref is not None and name != "fp64_half":
            d["shifted_slope_minus_fp64"] = (d["shifted"]["slope_per_atom_step"] -
                                             ref["shifted"]["slope_per_atom_step"])
    return out


# ---- saturation sweep over box size (the paper's throughput-vs-N curve) --------

def sweep_row(cells, n, name, r, K, hbm_peak, fp64_peak):
    """One line of the size sweep: throughput, and the pair launch against its
    roofline by the same formulas as the headline line."""
    prec, kind = name.split("_")[:2]
    ops, byts = pair_work(kind, prec, n, r["entries"], r["pairs"], int(r["compacted"]))
    step_b = step_bytes_per_atom(kind, r["entries"] / n)
    value = n * K / (r["ms"] * 1e-3) / 1e6
    row = {"cells": cells, "n_atoms": n, "form": name, "steps": K,
           "value": value, "ms_per_step": r["ms"] / K, "pair_kernel_ms": r["pair_ms"],
           "rebuild_ms": r["rebuild_ms"], "threads_per_atom": r["tpa"],
           "compacted_kernel": int(r["compacted"]), "phase1_entries": r["phase1_entries"],
           "list_entries_per_atom": r["entries"] / n, "pairs_in_rc_per_atom": r["pairs"] / n,
           "pair_kernel_hbm_frac": byts / (r["pair_ms"] * 1e-3) / 1e9 / hbm_peak,
           "step_hbm_frac": value * 1e6 * step_b / 1e9 / hbm_peak,
           "clocks": r["clocks"]}
    if prec == "fp64":
        row["pair_kernel_fp64_frac"] = ops / (r["pair_ms"] * 1e-3) / 1e9 / fp64_peak
    return row


def run_sweep(md, S, sizes, forms, hbm_peak, fp64_peak, W, sampler_gpu):
    """The fcc liquid at each size in `sizes` (fcc cells per edge), each form
    timed over K steps: 100 for the 32,000-atom melt, 1,000 otherwise."""
    rows = []
    for cells in sizes:
        sysm = S.fcc_liquid(cells)
        K = 100 if cells == 20 else 1000
        for name in forms:
            prec, kind = name.split("_")[:2]
            r = run_form(md, sysm, kind, prec, K, W, pair_reps=10, sampler_gpu=sampler_gpu,
                         drift=False)
            rows.append(sweep_row(cells, sysm.n, name, r, K, hbm_peak, fp64_peak))
            r["ctx"].close()
        del sysm
    return rows


def mixed_force_error(md, ctx, coul):
    """err_i = |F_i - F_i^FP64| / rms(F^FP64), its max and rms over all atoms,
    for the mixed context's forces at its current positions, against the
    FP64 compacted kernel on the same
    positions (the FP64 path matches the CPU oracle within 1e-12 in the
    tests).  Both lists are built at these positions, so they hold the same
    pairs."""
    ctx.build_neighbors()
    ctx.compute_forces(0)
    x, v, f = ctx.get_state()
    t = (np.arange(ctx.n) % 4 >= 2).astype(np.int32) if coul else None
    nt = 2 if coul else 1
    with md.LJMD(x, v, t, ctx.params.box[:], 1.0, 1.0, 2.5, [1.0] * nt,
                 list_kind=md.MD_LIST_HALF, threads_per_atom=1) as ref:
        if coul:
            ref.set_coulomb(COUL_Q, 2.5)
        ref.set_kernel(1, -1, 2, 0)
        ref.compute_forces(0)
        fr = ref.get_state()[2]
    rms = float(fr.pow(2).sum(1).mean().sqrt())
    err = (f - fr).norm(dim=1) / rms
    return {"max": float(err.max()), "rms": float(err.pow(2).mean().sqrt())}


def run_batched(md, K, W, R=512, persistent=-1):
    """Batched form: R independent fcc boxes with n_r ~ U{3..20} (seed 7),
    T ~ U[0.7, 1.5], FP64 half list, in one context (one launch per kernel
    per step, CUDA-graph segments).  Baselines on the same boxes: one context
    per box stepped in turn (each synchronized), and all those contexts
    stepped back to back on their own streams (concurrent), K_b steps each."""
    import torch
    from paper_2508_13523_gb300 import synth as S
    systems = S.replicas(R=R, seed=7)
    n = sum(s.n for s in systems)
    ctx = md.from_systems(systems, list_kind=md.MD_LIST_HALF, threads_per_atom=0)
    st = ctx.stats()
    if persistent >= 0 and persistent != st["persistent"]:
        ctx.set_kernel(st["threads_per_atom"], st["carveout"], kernel_code(st, persistent),
                       persistent)
        ctx.compute_forces(0)
    ctx.step(W)
    ctx.synchronize()
    l0 = ctx.stats()["kernel_launches"]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(ctx.stream)
    ctx.step(K)
    e1.record(ctx.stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    st = ctx.stats()
    out = {"n_replicas": R, "n_atoms": n, "ms": ms, "value": n * K / (ms * 1e-3) / 1e6,
           "threads_per_atom": st["threads_per_atom"], "steps": K,
           "compacted_kernel": st["compacted"], "persistent": st["persistent"],
           "phase1_entries": st["phase1_entries"],
           "launches_per_step": (st["kernel_launches"] - l0 - 1) / K,
           "replica_cells_min_max": [int(min(s.meta["n_cells"] for s in systems)),
                                     int(max(s.meta["n_cells"] for s in systems))]}
    if st["compacted"] == 2 and st["persistent"] != 2:
        # the same steps as one cooperative launch per step (persistent 2),
        # from where the timed run ended
        ctx.set_kernel(st["threads_per_atom"], st["carveout"], 2, 2)
        ctx.compute_forces(0)
        ctx.step(W)
        ctx.synchronize()
        l0 = ctx.stats()["kernel_launches"]
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(ctx.stream)
        ctx.step(K)
        f1.record(ctx.stream)
        f1.synchronize()
        fms = f0.elapsed_time(f1)
        out["one_launch_per_step"] = {
            "value": n * K / (fms * 1e-3) / 1e6, "ms": fms, "steps": K,
            "launches_per_step": (ctx.stats()["kernel_launches"] - l0 - 1) / K}
    ctx.close()
    kb = min(K, 20)
    singles = [md.from_system(s, list_kind=md.MD_LIST_HALF, threads_per_atom=0)
               for s in systems]
    for c in singles:
        c.step(3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c in singles:
        c.step(kb)
        c.synchronize()
    seq = time.perf_counter() - t0
    t0 = time.perf_counter()
    for c in singles:
        c.step(kb)
    torch.cuda.synchronize()
    conc = time.perf_counter() - t0
    for c in singles:
        c.close()
    out["sequential_value"] = n * kb / seq / 1e6
    out["concurrent_streams_value"] = n * kb / conc / 1e6
    out["speedup_vs_sequential"] = out["value"] / out["sequential_value"]
    out["speedup_vs_concurrent_streams"] = out["value"] / out["concurrent_streams_value"]
    out["baseline_steps"] = kb
    return out


def run_adjoint(md, K=100, every=10):
    """Adjoint form: binary LJ mixture, 64,000 atoms (80:20, density 1.2),
    random positions (seed 42) relaxed by 200 steepest-descent steps on the
    GPU, Maxwell-Boltzmann velocities at T* = 1.  Loss sum |F_K(theta) -
    F_ref|^2 with F_ref the forces after K steps at theta * 1.05; gradient
    with respect to (eps, sigma) and (x0, v0) by reverse mode through K steps,
    checkpoints every `every` steps; half list; FP64 and mixed precision."""
    import torch
    from paper_2508_13523_gb300 import synth as S
    s = S.binary_mixture(n=64000, seed=42)
    p = s.params
    relax = md.from_system(s, rebuild_every=10, threads_per_atom=1)
    relax.minimize(200, 0.01)
    x0, _, _ = relax.get_state()
    relax.close()
    v0 = torch.as_tensor(s.v, device=x0.device)
    out = {"n_atoms": s.n, "steps": K, "checkpoint_every": every, "sd_steps": 200}
    grads = {}
    for prec, name in ((md.MD_PREC_FP64, "fp64"), (md.MD_PREC_MIXED, "mixed")):
        ctx = md.LJMD(x0, v0, s.type, s.box, p.eps, p.sigma, p.rc, p.mass, rebuild_every=every,
                      list_kind=md.MD_LIST_HALF, precision=prec, threads_per_atom=0)
        ctx.set_lj(1.05 * p.eps, 1.05 * p.sigma)
        _, _, fref = ctx.traj_forward(x0, v0, K, every)
        ctx.set_lj(p.eps, p.sigma)
        ctx.traj_forward(x0, v0, K, every)  # warm-up (graphs, buffers)
        ctx.traj_vjp(K, every, *ctx.traj_forward(x0, v0, K, every)[:2], fref)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ckx, ckv, fK = ctx.traj_forward(x0, v0, K, every)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        cot = 2.0 * (fK - fref)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        x0b, v0b, g = ctx.traj_vjp(K, every, ckx, ckv, cot)
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        fwd, bwd = t1 - t0, t3 - t2
        grads[name] = (x0b.cpu().numpy(), g)
        out[name] = {"forward_s": fwd, "backward_s": bwd,
                     "forward_matom_steps_s": s.n * K / fwd / 1e6,
                     "backprop_matom_steps_s": s.n * K / (fwd + bwd) / 1e6,
                     "backward_over_forward": bwd / fwd,
                     "loss": float((cot * cot).sum().item() / 4.0),
                     "dL_deps": g[0].tolist(), "dL_dsigma": g[1].tolist()}
        ctx.close()
    xf, gf = grads["fp64"]
    xm, gm = grads["mixed"]
    out["mixed"]["grad_x0_err_vs_fp64"] = float(np.abs(xm - xf).max() /
                                               np.sqrt(np.mean(np.sum(xf * xf, axis=1))))
    out["mixed"]["grad_theta_err_vs_fp64"] = float(np.abs(gm - gf).max() / np.abs(gf).max())
    out["mixed_speedup_vs_fp64"] = ((out["fp64"]["forward_s"] + out["fp64"]["backward_s"]) /
                                   (out["mixed"]["forward_s"] + out["mixed"]["backward_s"]))
    return out


def e2e_run(md, ctx, n, K):
    """Per step: pinned host x, v -> device (md_set_state, keeping the list
    while no atom moved more than skin/2 since its build, else a full
    restart), one step, device x, v -> pinned host (md_get_state); all
    inside the timed region.  The loop starts from a list built just before
    it (untimed), so that how far the context was into its rebuild cycle
    does not decide how many restarts the loop pays."""
    import torch
    xh = torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
    vh = torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
    ctx.build_neighbors()
    ctx.get_state_into(xh, vh, None, md.MD_MEM_HOST)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(K):
        ctx.set_state_from(xh, vh, md.MD_MEM_HOST | md.MD_MEM_KEEP_LIST)
        ctx.step(1)
        ctx.get_state_into(xh, vh, None, md.MD_MEM_HOST)
    ctx.synchronize()
    dt = time.perf_counter() - t0
    return n * K / dt / 1e6, 48 * n, 48 * n


def cpu_baseline():
    """The oracle as it stands on this host: 256,000-atom (40^3) sample of the
    same liquid, 20 steps (one list build at the start, one at step 20)."""
    import oracle as O
    from paper_2508_13523_gb300 import synth as S
    s = S.fcc_liquid(40)
    t0 = time.perf_counter()
    O.run(s.x, s.v, s.box, O.LJ(), 1.0, nsteps=20)
    dt = time.perf_counter() - t0
    return {"value": s.n * 20 / dt / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "256,000-atom fcc LJ liquid (40^3 cells, T*=1.44), 20 velocity-Verlet "
                      "steps incl. 2 list builds, single-threaded C oracle, FP64",
            "seconds": dt}


def reference_arm(args, world, rank):
    if rank != 0:
        return 0
    import oracle as O
    from paper_2508_13523_gb300 import synth as S
    s = S.fcc_liquid(20)
    O.build()
    x, v, _, _ = O.run(s.x, s.v, s.box, O.LJ(), 1.0, nsteps=max(args.warmup, 1))
    t0 = time.perf_counter()
    O.run(x, v, s.box, O.LJ(), 1.0, nsteps=args.steps, step0=max(args.warmup, 1), init=False)
    dt = time.perf_counter() - t0
    value = s.n * args.steps / dt / 1e6
    sample = ("32,000-atom periodic sample (20^3 cells) of the same fcc LJ liquid, one oracle "
              "velocity-Verlet step per bench step, list rebuilt every 20 steps plus once at "
              "the start of the timed call; single-threaded C, FP64")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "lj_fcc_liquid_4M_atoms_fp64 (oracle on a 32,000-atom sample)",
                   "n_atoms_sampled": s.n, "rc": 2.5, "skin": 0.3, "dt": 0.005,
                   "rebuild_every": 20},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cells", type=int, default=N_CELLS, help="fcc cells per edge")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tpa", type=int, default=0, choices=[0, 1, 2, 4, 8, 16, 32],
                    help="threads per atom of the per-atom pair kernel (0: the tuner's choice)")
    ap.add_argument("--carveout", type=int, default=-1,
                    help="preferred shared-memory carveout of the pair kernel in percent "
                         "(-1: the driver's default)")
    ap.add_argument("--persistent", type=int, default=0, choices=[0, 1, 2],
                    help="1: the pair kernel as one resident grid taking tiles per SM; 2: "
                         "besides, one cooperative launch per step (FP64, compacted 2)")
    ap.add_argument("--compacted", type=int, default=-1, choices=[-1, 1, 2, 3],
                    help="FP64 forms: -1 the tuner's choice, 1 warp-compacted kernel with FP64 "
                         "force sums, 2 with fixed-point force sums, 3 the same with two list "
                         "entries per filter round")
    ap.add_argument("--forms", default="fp64_full,fp64_half,mixed_full,mixed_half,"
                                        "fp64_half_coul,mixed_half_coul,batched,adjoint")
    ap.add_argument("--drift-steps", type=int, default=10000,
                    help="steps of the energy-drift runs of fp64_half, mixed_half and "
                         "mixed_full from one initial state (0: skip)")
    ap.add_argument("--sweep", default="",
                    help="comma-separated fcc cells per edge (e.g. 20,40,100,160): time each "
                         "size over 1,000 steps (100 for the 20^3 melt) for --sweep-forms")
    ap.add_argument("--sweep-forms", default="fp64_half,fp64_full,mixed_half,mixed_full")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer e2e run")
    ap.add_argument("--batch-steps", type=int, default=1000,
                    help="timed steps of the 512-replica batched form")
    ap.add_argument("--batch-persistent", type=int, default=-1, choices=[-1, 0, 1, 2],
                    help="batched form's pair scheduling (-1: the tuner's; 2: one "
                         "cooperative launch per step)")
    args = ap.parse_args()
    world, rank, local = dist_env()
    if args.impl == "reference":
        return reference_arm(args, world, rank)
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")

    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    import paper_2508_13523_gb300 as md
    from paper_2508_13523_gb300 import synth as S
    md.load(build_if_missing=False)
    hbm_peak, sm_max, peak_src = peaks()
    fp64_peak = FP64_OPS_PER_CLK_SM * SM_COUNT * sm_max * 1e6 / 1e9  # Gop/s

    sysm = S.fcc_liquid(args.cells)
    n = sysm.n
    gpu_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local]) \
        if os.environ.get("CUDA_VISIBLE_DEVICES") else local
    forms = [f for f in args.forms.split(",") if f]
    if world > 1:  # replicas: each rank times the headline forms only
        forms = [f for f in forms if f not in ("batched", "adjoint")]
    results = {}
    headline = None
    adjoint = None
    if "adjoint" in forms:
        forms.remove("adjoint")
        barrier(world)
        adjoint = run_adjoint(md)
    batched = None
    if "batched" in forms:
        forms.remove("batched")
        barrier(world)
        batched = run_batched(md, args.batch_steps, args.warmup, persistent=args.batch_persistent)
    for name in forms:
        prec, kind, *style = name.split("_")
        coul = style == ["coul"]
        barrier(world)
        r = run_form(md, sysm, kind, prec, args.steps, args.warmup, pair_reps=10,
                     sampler_gpu=gpu_index, compacted=args.compacted, tpa=args.tpa,
                     carveout=args.carveout, persistent=args.persistent, coul=coul)
        ms = max_over_ranks(world, r["ms"])
        r["value"] = world * n * args.steps / (ms * 1e-3) / 1e6
        r["ms_max"] = ms
        results[name] = r
        if prec == "fp64" and not coul and (headline is None or
                                            r["value"] > results[headline]["value"]):
            headline = name

    drift = None
    if args.drift_steps > 0 and world == 1:
        drift = run_drift(md, sysm, ["fp64_half", "mixed_half", "mixed_full"], args.drift_steps)
    sweep = None
    if args.sweep and world == 1:
        sweep = run_sweep(md, S, [int(c) for c in args.sweep.split(",") if c],
                          [f for f in args.sweep_forms.split(",") if f], hbm_peak, fp64_peak,
                          args.warmup, gpu_index)

    if not results:  # only the batched / adjoint forms were asked for: their figures alone
        extra = {}
        if batched is not None:
            extra["batched_fp64_half"] = batched
        if adjoint is not None:
            extra["adjoint_mixture_64k"] = adjoint
        if rank == 0:
            print(json.dumps({"metric": METRIC, "unit": UNIT, "n_gpus": world,
                              "forms": extra}), flush=True)
        return 0
    if headline is None:  # no FP64 form requested: the fastest form heads the line
        headline = max(results, key=lambda k: results[k]["value"])
    h = results[headline]
    prec, kind = headline.split("_")[:2]
    ops, byts = pair_work(kind, prec, n, h["entries"], h["pairs"], int(h["compacted"]))
    # the kernel's own launch time inside steps when it was recorded (the
    # one-launch-per-step schedule brackets the combined launches instead)
    in_step = bool(h.get("pair_step_ms")) and h["persistent"] != 2
    kern_ms = h["pair_step_ms"] if in_step else h["pair_ms"]
    achieved_ops = ops / (kern_ms * 1e-3) / 1e9
    achieved_gbs = byts / (kern_ms * 1e-3) / 1e9
    epa = h["entries"] / n
    step_b = step_bytes_per_atom(kind, epa)
    step_gbs = h["value"] / world * 1e6 * step_b / 1e9
    label = {0: f"k_pair<{prec},{kind},TPA={h['tpa']}>",
             1: f"k_pair_q<{kind}> (warp-compacted, FP64 force sums)",
             2: f"k_pair_q<{kind}> (warp-compacted, fixed-point force sums)"}[h["compacted"]]
    if prec == "fp64":
        roofline = {"bound": "alu", "achieved": achieved_ops, "peak": fp64_peak,
                    "unit": "Gop/s (FP64 pipe)", "frac": achieved_ops / fp64_peak,
                    "peak_source": "2 FP64 lane-ops/clk/SM x 152 SMs x max SM clock (1.25 "
                                   "TFLOP/s nominal); DFMA measured at 628 Gop/s",
                    "ops_per_pair_visit": fp64_ops_per_pair(int(h["compacted"]))}
    else:  # the mixed form issues no FP64 operation per pair: HBM is its roof
        roofline = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                    "frac": achieved_gbs / hbm_peak, "peak_source": peak_src}
    roofline.update({"traffic": pair_traffic(headline, h["compacted"], h["tpa"], h["phase1_entries"], n),
                     "traffic_unit": "bytes per launch of the pair kernel",
                     "algorithmic_bytes": byts, "kernel": label,
                     "timed_as": ("the pair kernel's launches inside md_step, CUDA events "
                                  "around each (md_time_pair_kernel), mean of 10"
                                  if in_step else
                                  "md_compute_forces (zeroing, pair kernel, fixed-point fold)"),
                     "launch_ms": kern_ms,
                     "compute_forces_ms": h["pair_ms"],
                     "hbm_achieved_gbs": achieved_gbs, "hbm_peak_gbs": hbm_peak,
                     "hbm_frac": achieved_gbs / hbm_peak, "hbm_peak_source": peak_src})

    # end to end through the public API with host buffers
    e2e_val, bi, bo = (None, 0, 0) if args.no_e2e else e2e_run(md, h["ctx"], n,
                                                               min(args.steps, 10))
    if e2e_val is not None:
        e2e_val = world * e2e_val  # replicas: each rank moves its own box

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline()

    forms_out = {}
    for name, r in results.items():
        p, k, *style = name.split("_")
        o, b = pair_work(k, p, n, r["entries"], r["pairs"], int(r["compacted"]),
                         style == ["coul"])
        f = {"value": r["value"], "ms_per_step": r["ms_max"] / args.steps,
             "pair_kernel_ms": r["pair_ms"], "pair_kernel_in_step_ms": r["pair_step_ms"],
             "rebuild_ms": r["rebuild_ms"],
             "energy_virial_pair_ms": r["ev_ms"],
             "energy_virial_over_force_only": r["ev_ms"] / r["pair_ms"],
             "threads_per_atom": r["tpa"],
             "compacted_kernel": int(r["compacted"]), "carveout": r["carveout"],
             "persistent": r["persistent"], "phase1_entries": r["phase1_entries"],
             "force_sums": "fixed-point" if r["compacted"] == 2 else "fp64",
             "clocks": r["clocks"],
             "pair_kernel_gbs": b / (r["pair_ms"] * 1e-3) / 1e9,
             "pair_kernel_hbm_frac": b / (r["pair_ms"] * 1e-3) / 1e9 / hbm_peak,
             "pair_kernel_traffic": pair_traffic(name, r["compacted"], r["tpa"], r["phase1_entries"], n),
             "step_hbm_frac": r["value"] / world * 1e6 * step_bytes_per_atom(k, r["entries"] / n)
             / 1e9 / hbm_peak,
             "speedup_vs_fp64_headline": r["value"] / h["value"],
             "list_entries_per_atom": r["entries"] / n, "pairs_in_rc_per_atom": r["pairs"] / n,
             "dangerous_builds": r["dangerous"], "builds": r["builds"],
             "pe_per_atom": r["thermo"].pe / n, "temperature": r["thermo"].temperature,
             "energy_drift_per_atom_step": r["energy_drift"]}
        if p == "mixed":
            f["force_err_vs_fp64"] = mixed_force_error(md, r["ctx"], style == ["coul"])
        if p == "fp64":
            f["pair_kernel_fp64_gops"] = o / (r["pair_ms"] * 1e-3) / 1e9
        if style == ["coul"]:
            f["pair_style"] = "lj/cut/coul/cut, charges +-0.5 by fcc site, rc_coul 2.5"
            f["ops_per_pair_visit"] = 22
        forms_out[name] = f

    if drift is not None:
        for name, d in drift.items():
            forms_out.setdefault(name, {})["drift_long"] = d
    if batched is not None:
        batched["speedup_vs_fp64_headline"] = batched["value"] / (h["value"] / world)
        forms_out["batched_fp64_half"] = batched
    if adjoint is not None:
        forms_out["adjoint_mixture_64k"] = adjoint

    line = {
        "metric": METRIC, "value": h["value"], "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": h["ms_max"] / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == "fp64" else "f32 pair arithmetic, f64 positions and sums",
        "data": "synthetic",
        "config": {"workload": f"lj_fcc_liquid_{n}_atoms_{prec}_{kind}_list",
                   "n_atoms": n, "fcc_cells": args.cells, "density": 0.8442, "T": 1.44,
                   "rc": 2.5, "skin": 0.3, "dt": 0.005, "rebuild_every": 20,
                   "list": kind, "precision": prec, "threads_per_atom": h["tpa"],
                   "pair_kernel": label,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": f"inputs larger than L2 (positions {32 * n / 1e6:.0f} MB, neighbor "
                         f"list {4 * h['entries'] / 1e9:.2f} GB)"},
        "roofline": roofline,
        "step_hbm": {"bytes_per_atom_step": step_b, "achieved_gbs": step_gbs,
                     "frac": step_gbs / hbm_peak},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": bi,
                "d2h_bytes_per_step": bo, "steps": min(args.steps, 10),
                "path": "md_set_state(host, keep list while valid) + md_step(1) + "
                        "md_get_state(host) per step"},
        "gpu_launches": h["launches"],
        "clocks": h["clocks"],
        "forms": forms_out,
    }
    if sweep is not None:
        line["sweep"] = sweep
    if rank == 0:
        print(json.dumps(line), flush=True)
    for r in results.values():
        r["ctx"].close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
