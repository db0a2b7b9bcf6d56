#!/usr/bin/env python
"""Throughput of the dense-suspension time step on GB300 (particle-steps/s).

One step = the whole per-timestep path on one synthetic suspension: predictor
and Lees-Edwards wrap, counting sort, half-stencil neighbour enumeration,
contact-history carry, pair forces (lubrication + frictional contact),
deterministic symmetric accumulation, Stokes drag, corrector and bulk stress.

Workload (default): 100,000 bidisperse spheres (radii 1.0 / 1.4, equal
numbers), volume fraction 0.55, friction mu = 1.0, k_n = 1e4, shear rate 1,
dt = 1e-4, seeded random packing.  Its working set (~70 MB) fits in the 129 MB
L2, so the L2 is flushed (a 256 MB write) before every timed step and every
step is timed on its own with CUDA events recorded inside the step's CUDA
graph (per-kernel events; the step time runs from the first kernel's start to
the last kernel's end).

More modes are measured in the same run and reported under "modes":
"fp64", the same workload with the FP64 pair arithmetic; "batched", a
flow-curve sweep of 256 independent bidisperse suspensions (N uniform in
[500, 20000], volume fraction uniform in [0.40, 0.58], shear rate log-uniform
in [1e-2, 1e2], mixed precision) advanced together in one handle after the
cell edge is autotuned (working set ~1.5 GB, beyond the L2); "poly1m",
1,000,000 spheres with radii log-uniform in [1, 10] in mixed precision and
FP64; "adjoint", the gradient of the 200-step time-averaged viscosity of
20,000 spheres (checkpoint every 20 steps) against the forward alone;
"echem", the headline packing with the electro-chemical forces of Eq. 6-7;
"analysis", the analysis pass; "wavy", the Table 5 suspension (2^16 spheres,
radius ratio 3) in the uniform and the wavy shear flow of Eq. 17, with and
without rolling resistance.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                       [--modes fp64,echem,analysis,wavy,batched,poly1m,adjoint|none]
Under torchrun each rank runs an independent replica (replicas only: the
single-instance path has no data-parallel exchange); value = total particle
steps of all ranks / max over ranks of the timed GPU time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_FALLBACK = {"hbm_gbs": 6800.0}
METRIC = "particle-timesteps/s"
L2_FLUSH_BYTES = 256 << 20

# Method bytes per particle-step of the paper's path (the algorithmic
# minimum: every input read once, every output written once), per particle
# (n), cell (c), listed pair (p) and contact (k), FP64 / mixed:
#   neighbour + force step: sorted state read (x, u, w, a, id: 84 n), permuted
#   state written (84 n), F and T written (48 n / 24 n), the pair list
#   written and read (8 p), the contact history read and written (key and
#   stretch: 64 k), the cell table (8 c);
#   integration (Eq. 15): 168 n read, 120 n written.
# Each item is charged to the kernel that performs it.  The state read is
# split between the enumeration (positions and radii, 32 n) and the pair
# kernel (velocities, angular velocities and ids, 52 n).
METHOD_BYTES = {
    #                  fp64 (n, c, p, k)      mixed (n, c, p, k)
    "k_key_hist":    ((120, 0, 0, 0),       (120, 0, 0, 0)),     # predictor of x, u: 72 read, 48 written
    "k_scan_cells":  ((0, 8, 0, 0),         (0, 8, 0, 0)),       # cell table
    "k_scatter":     ((0, 0, 0, 0),         (0, 0, 0, 0)),
    "k_rank_gather": ((156, 0, 0, 0),       (156, 0, 0, 0)),     # permuted state 84, w predictor 72
    "k_enumerate":   ((32, 0, 4, 0),        (32, 0, 4, 0)),      # positions and radii, list written
    "k_pairs":       ((100, 0, 4, 64),      (76, 0, 4, 64)),     # u, w, id; F, T; list read; history
    "k_gather":      ((96, 0, 0, 0),        (96, 0, 0, 0)),      # corrector: u, w read and written
}
# Bytes of this design's own data structures per kernel (partner records,
# 32-byte stretch records, FP32 copies of the sorted state, ...): what the
# kernels actually move when every access hits DRAM once.  Reported beside the
# method bytes as implementation overhead.
IMPL_BYTES = {
    "k_key_hist":    ((133, 0, 0, 0),       (133, 0, 0, 0)),
    "k_scan_cells":  ((0, 12, 0, 0),        (0, 12, 0, 0)),
    "k_scatter":     ((16, 0, 0, 0),        (16, 0, 0, 0)),
    "k_rank_gather": ((269, 0, 0, 0),       (301, 0, 0, 0)),
    "k_enumerate":   ((52, 8, 16, 0),       (52, 8, 16, 0)),     # + rows read back, compacted (12 p)
    "k_pairs":       ((144, 0, 112, 56),    (108, 0, 80, 56)),   # pair-balanced (one instance)
    "k_gather":      ((220, 0, 64, 0),      (220, 0, 32, 0)),
}
# The neighbour + force step alone (without the integration's 288 n).
NF_BYTES = ((216, 8, 8, 64), (192, 8, 8, 64))
ALG_BYTES = METHOD_BYTES
KERNELS_PER_STEP = len(ALG_BYTES)

# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) from
# an ncu capture of the kernel, keyed by kernel, precision and particle count,
# with the sources it was built from and their hash; reported only while
# those files are unchanged (pair kernel: profiles/ncu_full_c2_mixed_100k.md,
# profiles/ncu_full_c3_mixed_1m.md; enumeration:
# profiles/ncu_enumerate_screened_c3_mixed_1m.md; the 1M captures ran with the
# row capacity cut to 64, which changes the rows' stride, not the pairs or the
# work).
_PAIR_SRC = ("dss_force.cu", "dss_internal.cuh", "dss_pair_model.cuh")
_ENUM_SRC = ("dss_neighbour.cu", "dss_internal.cuh")
NCU_TRAFFIC = {
    ("k_pairs", "mixed", 100_000): (30_699_520, _PAIR_SRC, "9557dfb1c9e0b948"),
    ("k_enumerate", "mixed", 100_000): (7_125_760, _ENUM_SRC, "614103effa34d4d4"),
    ("k_pairs", "mixed", 1_000_000): (300_538_112, _PAIR_SRC, "9557dfb1c9e0b948"),
    ("k_enumerate", "mixed", 1_000_000): (110_382_848, _ENUM_SRC, "614103effa34d4d4"),
}


def src_hash(files) -> str:
    d = os.path.join(ROOT, "paper_2108_01013_gb300", "csrc")
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="c2")
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--modes", default="fp64,echem,analysis,wavy,batched,poly1m,adjoint,cpu",
                    help="extra modes measured in the same run: fp64 (the headline workload in "
                         "FP64), echem (the headline packing with the electro-chemical forces, "
                         "mixed), analysis (clusters, dispersion, rheology calls on it), batched (256-instance flow-curve sweep, mixed), poly1m (1M "
                         "polydisperse, mixed and FP64), adjoint (gradient of the 200-step "
                         "viscosity of 20k spheres), cpu (the oracle on the host cores: 1000 "
                         "brute-force steps of the 1k configuration, whole steps of the 1M "
                         "and Table 5 packings); 'none' for none")
    ap.add_argument("--capacity-m", type=int, default=0,
                    help="row capacity M of the headline workload's half lists (0: the shell "
                         "estimate of Sec. II A); a smaller M keeps an ncu capture of the 1M "
                         "workload (--workload c3) within a few GB")
    ap.add_argument("--mode-steps", type=int, default=400)
    ap.add_argument("--batch-instances", type=int, default=256,
                    help="instances of the batched mode (the first K of the 256-instance sweep)")
    return ap.parse_args()


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", "dss_clocks_%d_%d.csv" % (os.getpid(), index))

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), util=float(parts[4]),
                                 hw=parts[6], hwt=parts[7], swt=parts[8], pcap=parts[9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        load = [r for r in rows if r["util"] > 0] or rows
        reasons = set()
        for r in load:
            for k, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                            ("swt", "sw_thermal_slowdown"), ("pcap", "sw_power_cap")):
                if r[k].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median([r["sm"] for r in load])),
                "sm_max_mhz": max(r["smax"] for r in rows), "samples": len(load),
                "reasons": sorted(reasons)}


def host_cores() -> int:
    """Threads the oracle's OpenMP loops use on this host."""
    env = os.environ.get("OMP_NUM_THREADS")
    if env and env.isdigit() and int(env) > 0:
        return int(env)
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def oracle_steps(g, params_kw, steps: int, cells: bool = True, warmup: int = 1):
    """Times whole oracle time steps (Eq. 15 with every force of the model)
    on the host: the cell-list search with the half stencil of Sec. II A
    (cells=True, the pair set checked equal to the brute force) or the O(N^2)
    brute force, pairs evaluated on all host cores.  Returns (seconds per
    step, pairs of the last step)."""
    import oracle
    oracle.build()
    po = oracle.make_params(g["box"], **params_kw)
    o = oracle.System(po, g["x"], g["a"], ids=g["ids"], cells=cells)
    o.init_accel()
    if warmup:
        o.step(warmup)
    t0 = time.perf_counter()
    o.step(steps)
    dt = (time.perf_counter() - t0) / max(steps, 1)
    return dt, o.npairs


def cpu_baseline(g, params_kw, seconds: float, steps: int = 0):
    """The oracle timed on whole time steps of the workload: cell-list search
    with the half stencil, pairs on all host cores; the number of steps is
    chosen so that the run takes about ``seconds``."""
    n = g["a"].shape[0]
    per, _ = oracle_steps(g, params_kw, 1, warmup=0)
    k = steps or max(2, min(50, int(seconds / max(per, 1e-6))))
    per, npairs = oracle_steps(g, params_kw, k, warmup=0)
    return {"value": n / per, "unit": METRIC, "cores": host_cores(), "kind": "oracle",
            "sample": "%d whole time steps of the %d-particle workload (%d pairs per step; cell list "
                      "with the half stencil, pair evaluations in parallel, FP64) at %.3f s per "
                      "step" % (k, n, npairs, per)}


def cpu_oracle_modes(inputs: dict, seconds: float):
    """The oracle on the other workloads, for context: the 1000-particle FP64
    configuration over its full 1000 steps by brute force, and about
    ``seconds`` of whole steps with the cell list on the 1M polydisperse and
    the Table 5 packings (without the electro-chemical forces, as the paper's
    timing table is quoted with them; the force settings differ)."""
    out = {"cores": host_cores()}
    if "c1" in inputs:
        spec, g = inputs["c1"]
        kw = dict(mu=spec.mu, kn=spec.kn, shear_rate=spec.shear_rate, dt=spec.dt)
        per, P = oracle_steps(g, kw, spec.steps, cells=False, warmup=0)
        out["c1_bruteforce_1000_steps"] = {"seconds": per * spec.steps, "value": g["a"].shape[0] / per,
                                           "unit": "particle-steps/s", "steps": spec.steps, "pairs": P}
    for key, name in (("c3", "c3_cell_list"), ("c6", "c6_cell_list")):
        if key not in inputs:
            continue
        spec, g = inputs[key]
        kw = dict(mu=spec.mu, kn=spec.kn, shear_rate=spec.shear_rate, dt=spec.dt)
        if key == "c6":
            kw.update({k: v for k, v in spec.extra.items()
                       if k not in ("f_er", "hamaker", "wave_amp", "wave_n")})
        per1, _ = oracle_steps(g, kw, 1, warmup=0)
        k = max(1, min(10, int(seconds / max(per1, 1e-6))))
        per, P = oracle_steps(g, kw, k, warmup=0)
        out[name] = {"value": g["a"].shape[0] / per, "unit": "particle-steps/s", "s_per_step": per,
                     "steps": k, "pairs": P}
    return out


def max_over_ranks(x: float, world: int, device=None) -> float:
    """Largest value of x over the ranks (x itself on one rank); device is
    where the reduction's tensor lives (a GPU under NCCL, the CPU under gloo)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int, device=None) -> float:
    """Sum of x over the ranks (x itself on one rank)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_rate(units: float, seconds: float, world: int, device=None) -> float:
    """Whole-job rate of N independent replicas (weak scaling): the units all
    ranks processed (summed, since the seeded workloads of the ranks may
    differ in size) over the slowest rank's time."""
    return sum_over_ranks(units, world, device) / max_over_ranks(seconds, world, device)


def reduce_modes(extra: dict, world: int, device=None) -> None:
    """Every measured mode (an entry, or an entry of a mode's sub-table,
    carrying ms_per_step and value) becomes a whole-job figure: the slowest
    rank's ms per step and the units per step of all ranks over it.  Every
    rank walks the same modes in the same order, so the reductions pair up."""
    if world <= 1:
        return
    for m in extra.values():
        if not isinstance(m, dict):
            continue
        subs = [m] if "ms_per_step" in m else [v for v in m.values() if isinstance(v, dict) and "ms_per_step" in v]
        for e in subs:
            units = sum_over_ranks(e["value"] * e["ms_per_step"], world, device)
            slowest = max_over_ranks(e["ms_per_step"], world, device)
            e["value"] = units / slowest
            e["ms_per_step"] = slowest


def roofline(prof, nprof, c, n, precision, peaks, src, step_ms):
    """Roofline records from the method bytes: the dominant kernel's (its
    method bytes per launch over its mean event time), the whole step's
    (method bytes of the step, and of the neighbour + force part alone, over
    the step time), and a per-kernel table with this design's own bytes
    beside the method bytes."""
    mode = 0 if precision == "fp64" else 1
    P, K = c["npairs"], c["ncontacts"]
    ncell = int(np.prod(c["ncell"]))

    def nbytes(t):
        bn, bc, bp, bk = t
        return bn * n + bc * ncell + bp * P + bk * K

    per_kernel = {}
    for k, ms in prof.items():
        avg = ms / max(nprof, 1)
        mb, ib = nbytes(METHOD_BYTES[k][mode]), nbytes(IMPL_BYTES[k][mode])
        per_kernel[k] = {"ms": avg, "method_bytes": mb, "impl_bytes": ib,
                         "gbs": mb / (avg * 1e-3) / 1e9 if avg > 0 else 0.0,
                         "impl_over_method": ib / mb if mb else None}
    dom = max(per_kernel, key=lambda k: per_kernel[k]["ms"])
    d = per_kernel[dom]
    peak = float(peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"]))
    traffic = None
    rec = NCU_TRAFFIC.get((dom, precision, n))
    if rec is not None and src_hash(rec[1]) == rec[2]:
        traffic = rec[0]
    roof = {"bound": "hbm", "kernel": dom, "achieved": d["gbs"], "peak": peak, "unit": "GB/s",
            "frac": d["gbs"] / peak, "traffic": traffic, "peak_source": src,
            "bytes_per_launch": d["method_bytes"],
            "share": d["ms"] / max(sum(v["ms"] for v in per_kernel.values()), 1e-12)}
    step_bytes = sum(v["method_bytes"] for v in per_kernel.values())
    nf_bytes = nbytes(NF_BYTES[mode])
    step_s = step_ms * 1e-3
    roof_step = {"bound": "hbm", "unit": "GB/s", "peak": peak, "peak_source": src,
                 "bytes_per_particle_step": step_bytes / n,
                 "achieved": step_bytes / step_s / 1e9, "frac": step_bytes / step_s / 1e9 / peak,
                 "neighbour_force_bytes_per_particle_step": nf_bytes / n,
                 "neighbour_force_achieved": nf_bytes / step_s / 1e9,
                 "neighbour_force_frac": nf_bytes / step_s / 1e9 / peak,
                 "pairs_per_particle": P / n, "contacts_per_particle": K / n,
                 "impl_bytes_per_particle_step": sum(v["impl_bytes"] for v in per_kernel.values()) / n}
    return roof, roof_step, per_kernel


def workload(name: str, rank: int):
    from paper_2108_01013_gb300 import synth
    spec = synth.SPECS[name]
    if rank:
        from dataclasses import replace
        spec = replace(spec, seed=spec.seed + 1000 * rank)
    return spec, synth.generate(spec)


def time_steps(s, steps, flush=None):
    """GPU time (ms) of ``steps`` single-step graph replays, each after an
    optional L2 flush; returns the total."""
    t = 0.0
    for _ in range(steps):
        if flush is not None:
            flush.fill_(1.0)
        s.step(1)
        t += s.last_step_ms()
    return t


def profile_pass(s, steps, flush=None):
    s.set_profiling(True)
    for _ in range(steps):
        if flush is not None:
            flush.fill_(1.0)
        s.step(1)
    prof, nprof = s.profile()
    s.set_profiling(False)
    return {k: round(v / max(nprof, 1), 5) for k, v in prof.items()}


def mode_fp64(dss, g, spec, kw, args, flush, stream):
    """The headline workload with the FP64 pair arithmetic."""
    n = g["a"].shape[0]
    p = dss.default_params(g["box"], precision="fp64", **kw)
    s = dss.Suspension(g["x"], g["a"], g["box"], p, ids=g["ids"], stream=stream)
    time_steps(s, 5, flush)
    steps = min(args.mode_steps * 2, args.steps)
    t = time_steps(s, steps, flush)
    out = {"value": n * steps / (t * 1e-3), "unit": "particle-steps/s", "ms_per_step": t / steps,
           "steps": steps, "dtype": "f64", "config": {"workload": spec.name, "n": n, "precision": "fp64",
                                                      "l2": "flushed before every timed step"},
           "kernels_ms": profile_pass(s, 20, flush)}
    s.close()
    return out


# The electro-chemical settings of the paper's shear-rate studies (Table 3:
# lambda_D = 0.05 a0, repulsion only, delta_lub = 0.10 a0; Table 4 (SI):
# lambda_D = 0.0225 a0, F^R/F^A = 19 at contact, delta_lub = 0.25 a0, mu = 0.5),
# at gdot/gdot_0 = 0.1 (F_ER = 10 eta0 a0^2 gdot with gdot = 1).  The van der
# Waals constant follows from the contact ratio: F^A(0) = A / (12 eps^2) for
# abar = a0 and eps = 0.01 abar.
ECHEM_SETTINGS = {
    "repulsion": dict(f_er=10.0, lambda_d=0.05, hamaker=0.0, vdw_eps=0.01, delta_lub=0.10),
    "repulsion_attraction": dict(f_er=10.0, lambda_d=0.0225, hamaker=10.0 / 19.0 * 12.0 * 1e-4,
                                 vdw_eps=0.01, delta_lub=0.25, mu=0.5),
}


def mode_echem(dss, g, spec, kw, args, flush, stream):
    """The headline packing with the electro-chemical forces of Eq. 6-7 (mixed
    precision): pairs are listed out to their range."""
    n = g["a"].shape[0]
    out = {"config": {"workload": spec.name + "_echem", "n": n, "precision": "mixed",
                      "l2": "flushed before every timed step"}}
    for name, e in ECHEM_SETTINGS.items():
        kk = dict(kw)
        kk.update(e)
        p = dss.default_params(g["box"], precision="mixed", **kk)
        s = dss.Suspension(g["x"], g["a"], g["box"], p, ids=g["ids"], stream=stream)
        time_steps(s, 5, flush)
        steps = max(args.mode_steps // 2, 1)
        t = time_steps(s, steps, flush)
        c = s.counters()
        out[name] = {"value": n * steps / (t * 1e-3), "unit": "particle-steps/s", "ms_per_step": t / steps,
                     "steps": steps, "params": e, "pairs": c["npairs"], "contacts": c["ncontacts"], "M": c["M"],
                     "cells": list(c["ncell"]), "kernels_ms": profile_pass(s, 10, flush)}
        s.close()
    return out


def mode_wavy(dss, g, spec, args, flush, stream):
    """Table 5: 2^16 spheres of radius ratio 3 (V2/V1 = 0.25, phi = 0.5) with
    the electro-chemical forces, in the uniform shear (NW) and in the wavy
    shear flow of Eq. 17 (YW, U = 20 gdot a0, n = 1, Faxen drag), and YW with
    the rolling resistance of App. B (k_r = 0.05 k_n); YW also on the
    size-class grid (cell_mode 1: the small spheres search cells sized for
    their own range, Sec. II A)."""
    n = g["a"].shape[0]
    base = dict(mu=spec.mu, kn=spec.kn, shear_rate=spec.shear_rate, dt=spec.dt, **spec.extra)
    cases = {
        "NW_mixed": (dict(base, wave_amp=0.0, wave_n=0), "mixed"),
        "YW_mixed": (base, "mixed"),
        "YW_fp64": (base, "fp64"),
        "YW_rolling_mixed": (dict(base, k_r=0.05 * spec.kn), "mixed"),
        "YW_rolling_fp64": (dict(base, k_r=0.05 * spec.kn), "fp64"),
        "YW_mixed_size_classes": (dict(base, cell_mode=1), "mixed"),
        # the same packing with lubrication and contact only (the paper's
        # timing workload shape without the electro-chemical forces)
        "context_no_echem_fp64": (dict(base, wave_amp=0.0, wave_n=0, f_er=0.0, hamaker=0.0), "fp64"),
        "context_no_echem_mixed": (dict(base, wave_amp=0.0, wave_n=0, f_er=0.0, hamaker=0.0), "mixed"),
    }
    out = {"config": {"workload": spec.name, "n": n, "a2_a1": spec.a_large / spec.a_small,
                      "l2": "flushed before every timed step"}}
    for name, (k, prec) in cases.items():
        p = dss.default_params(g["box"], precision=prec, **k)
        s = dss.Suspension(g["x"], g["a"], g["box"], p, ids=g["ids"], stream=stream)
        time_steps(s, 5, flush)
        steps = max(args.mode_steps // 2, 1)
        t = time_steps(s, steps, flush)
        c = s.counters()
        out[name] = {"value": n * steps / (t * 1e-3), "unit": "particle-steps/s", "ms_per_step": t / steps,
                     "steps": steps, "precision": prec, "pairs": c["npairs"], "contacts": c["ncontacts"],
                     "M": c["M"], "cells": list(c["ncell"]), "kernels_ms": profile_pass(s, 10, flush)}
        s.close()
    return out


def mode_analysis(dss, g, spec, kw, args, stream):
    """The analysis pass on the headline workload (mixed): after 50 steps the
    dispersion is marked, after 50 more every analysis call is timed (host
    clock around calls that synchronise, mean of 10)."""
    import time as _t
    import numpy as _np
    n = g["a"].shape[0]
    p = dss.default_params(g["box"], precision="mixed", **kw)
    s = dss.Suspension(g["x"], g["a"], g["box"], p, ids=g["ids"], stream=stream)
    s.step(50)
    s.dispersion_mark()
    s.step(50)

    def timed(f):
        f()
        t0 = _t.perf_counter()
        for _ in range(10):
            r = f()
        return (_t.perf_counter() - t0) / 10 * 1e3, r

    t_cl, (label, ncl) = timed(s.contact_clusters)
    t_di, disp = timed(s.dispersion)
    t_rh, rh = timed(lambda: s.rheology(mean=True))
    sizes = _np.unique(label, return_counts=True)[1]
    out = {"config": {"workload": spec.name, "n": n, "precision": "mixed", "steps_before": 100},
           "contact_clusters": {"ms": t_cl, "clusters": ncl, "largest": int(sizes.max()),
                                "contacts": s.counters()["ncontacts"]},
           "dispersion": {"ms": t_di, "D_y": float(disp[0, 0]), "C_v": float(disp[0, 1]),
                          "t_minus_t0": float(disp[0, 2])},
           "rheology": {"ms": t_rh, "sigma_N1_N2_Pi_eta_r_eta_n": [float(v) for v in rh[0]]}}
    s.close()
    return out


def mode_batched(dss, b, bspec, args, stream):
    """The flow-curve sweep: every instance of the batch advanced together,
    cell edge autotuned first."""
    p = dss.default_params(precision="mixed", mu=bspec.mu, kn=bspec.kn, dt=bspec.dt)
    s = dss.Batch(b["x"], b["a"], b["n"], b["boxes"], b["shear_rates"], p, ids=b["ids"], stream=stream)
    N = int(b["n"].sum())
    cs, trials = s.autotune(trial_steps=10)
    time_steps(s, 5)
    s.batch_stress(reset=True)
    steps = args.mode_steps
    t = time_steps(s, steps)
    _, mean, nmean = s.batch_stress()
    eta = mean[:, 0, 1] / b["shear_rates"]          # eta0 = 1: relative viscosity per instance
    c = s.counters()
    out = {"value": N * steps / (t * 1e-3), "unit": "particle-steps/s", "ms_per_step": t / steps,
           "steps": steps, "dtype": "f32+f64",
           "config": {"workload": bspec.name, "instances": int(bspec.K), "n_total": N,
                      "n_range": [int(b["n"].min()), int(b["n"].max())],
                      "phi_range": [round(float(b["phi"].min()), 4), round(float(b["phi"].max()), 4)],
                      "shear_rate_range": [float(b["shear_rates"].min()), float(b["shear_rates"].max())],
                      "precision": "mixed", "mu": bspec.mu,
                      "l2": "working set > L2 (no flush)",
                      "packing": "random insertion + %d relaxation sweeps" % bspec.max_iter},
           "autotune": {"cell_edge": cs, "ms_per_step_by_factor": trials},
           "mean_stress_steps": nmean,
           "eta_r_quartiles": [float(q) for q in np.percentile(eta, [0, 25, 50, 75, 100])],
           "pairs": c["npairs"], "kernels_ms": profile_pass(s, 10)}
    s.close()
    return out


def mode_poly1m(dss, g, spec, args):
    """1,000,000 spheres, radii log-uniform in [1, 10] (M = 728), in mixed
    precision and in FP64; its working set exceeds L2."""
    n = g["a"].shape[0]
    out = {"config": {"workload": spec.name, "n": n, "phi": spec.phi, "radii": "log-uniform [1, 10]",
                      "mu": spec.mu, "l2": "working set > L2 (no flush)",
                      "packing": "random insertion + %d relaxation sweeps" % spec.max_iter}}
    cmin = (2.0 + 0.05) * float(g["a"].max()) * (1 + 1e-9)
    for prec, steps in (("mixed", args.mode_steps // 2), ("fp64", args.mode_steps // 8),
                        ("mixed_size_classes", args.mode_steps // 4)):
        # one cell list (cells >= 2 a_max + delta); for comparison the size
        # classes of Sec. II A (cells of half that edge, larger stencils for the
        # larger particles)
        classes = prec.endswith("size_classes")
        p = dss.default_params(g["box"], precision=prec.split("_")[0], mu=spec.mu, kn=spec.kn,
                               shear_rate=spec.shear_rate, dt=spec.dt, cell_mode=1 if classes else 0,
                               cell_size=0.5 * cmin if classes else 0.0)
        s = dss.Suspension(g["x"], g["a"], g["box"], p, ids=g["ids"])
        time_steps(s, 3)
        t = time_steps(s, steps)
        c = s.counters()
        kms = profile_pass(s, 5)
        peaks, src = load_peaks()
        roof, roof_step, _ = roofline(kms, 1, c, n, prec.split("_")[0], peaks, src, t / steps)
        out[prec] = {"value": n * steps / (t * 1e-3), "unit": "particle-steps/s", "ms_per_step": t / steps,
                     "steps": steps, "device_gb": round(s.device_bytes() / 1e9, 1), "pairs": c["npairs"],
                     "contacts": c["ncontacts"], "M": c["M"], "cells": list(c["ncell"]), "kernels_ms": kms,
                     "roofline": roof, "roofline_step": roof_step}
        s.close()
    return out


def mode_adjoint(dss, g, spec, args):
    """Gradient of the time-averaged relative viscosity of a 200-step rollout
    of 20,000 spheres with respect to the model constants and the initial
    positions (checkpoint every 20 steps, mixed-precision forward)."""
    n = g["a"].shape[0]
    T = spec.steps
    p = dss.default_params(g["box"], precision="mixed", mu=spec.mu, kn=spec.kn,
                           shear_rate=spec.shear_rate, dt=spec.dt, lub_taper=0.2)
    W = dss.viscosity_weights(T, shear_rate=spec.shear_rate)
    s = dss.Suspension(g["x"], g["a"], g["box"], p, ids=g["ids"])
    ck = s.save()
    s.adjoint(T, W, ckpt_every=20)                    # warm-up (allocations, graphs)
    s.load(ck)
    time_steps(s, T)                                   # forward alone, same steps
    s.load(ck)
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = s.adjoint(T, W, ckpt_every=20)
    t_adj = time.perf_counter() - t0
    s.load(ck)
    t_fwd = time_steps(s, T) * 1e-3
    # the same forward through the API, wall clock (like the adjoint's own
    # time: host calls and synchronisation included)
    s.load(ck)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.step(T)
    torch.cuda.synchronize()
    t_fwd_wall = time.perf_counter() - t0
    s.close()
    return {"value": n * T / t_adj, "unit": "particle-steps/s (forward + reverse)",
            "seconds": t_adj, "forward_seconds": t_fwd, "reverse_over_forward": t_adj / t_fwd,
            "forward_wall_seconds": t_fwd_wall, "reverse_over_forward_wall": t_adj / t_fwd_wall,
            "note": "seconds: wall clock of dss_adjoint (its checkpointed forward, the taped replays "
                    "and the reverse sweep); forward_seconds: GPU time of the 200 step graphs alone",
            "config": {"workload": spec.name, "n": n, "steps": T, "checkpoint_every": 20,
                       "precision": "mixed forward, FP64 reverse", "lub_taper": 0.2,
                       "objective": "time-averaged relative viscosity"},
            "J": r["J"], "dJ": dict(zip(("kn", "kt", "gamma_n", "mu", "delta_lub"), r["params"].tolist())),
            "dJ_dx0_norm": float(np.linalg.norm(r["x0"]))}


def run_reference(args, rank, world):
    """The reference arm: the oracle itself (the paper publishes no code), on
    rank 0 alone, stepping the headline workload whole time step by whole
    time step on the host cores (cell list with the half stencil, pair
    evaluations in parallel): W untimed steps, then K timed ones."""
    spec, g = workload(args.workload, 0)
    if rank != 0:
        return
    kw = dict(mu=spec.mu, kn=spec.kn, shear_rate=spec.shear_rate, dt=spec.dt)
    import oracle
    oracle.build()
    po = oracle.make_params(g["box"], **kw)
    o = oracle.System(po, g["x"], g["a"], ids=g["ids"], cells=True)
    n = g["a"].shape[0]
    o.init_accel()
    if args.warmup:
        o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    t = time.perf_counter() - t0
    value = n * args.steps / t
    cores = host_cores()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "particle-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": spec.name, "n": n, "phi": spec.phi, "mu": spec.mu,
                       "radii": "1.0/1.4 equal numbers", "precision": "fp64", "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": "particle-steps/s", "cores": cores, "kind": "oracle",
                             "sample": "%d whole time steps after %d untimed ones (cell list with the "
                                       "half stencil, pair evaluations on %d host threads, FP64)"
                                       % (args.steps, args.warmup, cores)},
            "e2e": {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    modes = [] if args.modes in ("", "none") else args.modes.split(",")
    batch = None
    extra_inputs = {}
    # the oracle's timings on the other workloads (rank 0, before any CUDA call)
    cpu_inputs = {}
    if rank == 0 and world == 1 and not args.no_cpu_baseline and "cpu" in modes:
        cpu_inputs["c1"] = workload("c1", 0)
    if "poly1m" in modes:
        from paper_2108_01013_gb300 import synth
        extra_inputs["poly1m"] = workload("c3", rank)
        if cpu_inputs:
            cpu_inputs["c3"] = extra_inputs["poly1m"]
    if "adjoint" in modes:
        extra_inputs["adjoint"] = workload("c5", rank)
    if "wavy" in modes:
        extra_inputs["wavy"] = workload("c6", rank)
    if cpu_inputs:
        cpu_inputs["c6"] = extra_inputs["wavy"] if "wavy" in extra_inputs else workload("c6", 0)
    if "batched" in modes:
        # packed by spawned worker processes before the first CUDA call
        from paper_2108_01013_gb300 import synth
        bspec = synth.BATCH_SPECS["c4"]
        if args.batch_instances != bspec.K:
            from dataclasses import replace
            bspec = replace(bspec, K=args.batch_instances)
        if rank:
            from dataclasses import replace
            bspec = replace(bspec, seed=bspec.seed + 1000 * rank)
        batch = synth.generate_batch(bspec)

    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2108_01013_gb300 as dss
    dss.build()

    spec, g = workload(args.workload, rank)
    n = g["a"].shape[0]
    kw = dict(mu=spec.mu, kn=spec.kn, shear_rate=spec.shear_rate, dt=spec.dt)
    params = dss.default_params(g["box"], precision=args.precision, capacity_M=args.capacity_m, **kw)
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        s = dss.Suspension(g["x"], g["a"], g["box"], params, ids=g["ids"], stream=stream)
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        for _ in range(args.warmup):
            flush.fill_(1.0)
            s.step(1)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        clocks = Clocks(local)
        clocks.start()
        t_wall = time.perf_counter()
        t_gpu_ms = 0.0
        with torch.cuda.nvtx.range("headline"):
            for _ in range(args.steps):
                flush.fill_(1.0)                   # L2 flush between timed steps
                s.step(1)
                t_gpu_ms += s.last_step_ms()       # events around the step graph
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t_wall = time.perf_counter() - t_wall
        clk = clocks.stop()
        c = s.counters()
        step_ms = t_gpu_ms / args.steps
        value = job_rate(n * args.steps, t_gpu_ms * 1e-3, world, dev)
        # per-kernel shares: a separate pass with events between the kernels
        s.set_profiling(True)
        for _ in range(min(args.steps, 50)):
            flush.fill_(1.0)
            s.step(1)
        prof, nprof = s.profile()
        s.set_profiling(False)

        # end to end through the public API: per step upload the full state
        # from pinned host memory, advance, read state and stress back, in one
        # call (dss_step_io: upload, step graph, download and stress read
        # issued back to back, one synchronisation)
        host = [torch.empty((3, n), dtype=torch.float64, pin_memory=True) for _ in range(5)]
        sig = torch.empty(9, dtype=torch.float64, pin_memory=True)
        s.get_state_into(*host)
        for _ in range(3):                         # untimed: first calls
            s.step_io(host, 1, host, sig)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            s.step_io(host, 1, host, sig)
        torch.cuda.synchronize()
        t_e2e = time.perf_counter() - t0
        e2e_value = job_rate(n * args.e2e_steps, t_e2e, world, dev)
        bytes_state = 5 * 3 * n * 8
        s.close()
        extra = {}
        if "fp64" in modes:
            with torch.cuda.nvtx.range("fp64"):
                extra["fp64"] = mode_fp64(dss, g, spec, kw, args, flush, stream)
        if "echem" in modes:
            with torch.cuda.nvtx.range("echem"):
                extra["echem"] = mode_echem(dss, g, spec, kw, args, flush, stream)
        if "analysis" in modes:
            with torch.cuda.nvtx.range("analysis"):
                extra["analysis"] = mode_analysis(dss, g, spec, kw, args, stream)
        if "wavy" in extra_inputs:
            sp, gp = extra_inputs.pop("wavy")
            with torch.cuda.nvtx.range("wavy"):
                extra["wavy"] = mode_wavy(dss, gp, sp, args, flush, stream)
        del flush
        if batch is not None:
            with torch.cuda.nvtx.range("batched"):
                extra["batched"] = mode_batched(dss, batch, bspec, args, stream)
        if "poly1m" in extra_inputs:
            sp, gp = extra_inputs.pop("poly1m")
            with torch.cuda.nvtx.range("poly1m"):
                extra["poly1m"] = mode_poly1m(dss, gp, sp, args)
        if "adjoint" in extra_inputs:
            sp, gp = extra_inputs.pop("adjoint")
            with torch.cuda.nvtx.range("adjoint"):
                extra["adjoint"] = mode_adjoint(dss, gp, sp, args)
        reduce_modes(extra, world, dev)
        if "fp64" in extra:
            extra["mixed_vs_fp64"] = value / extra["fp64"]["value"]
            if "batched" in extra:
                extra["batched_vs_fp64_single"] = extra["batched"]["value"] / extra["fp64"]["value"]

    # roofline of the dominant kernel and of the whole step
    peaks, src = load_peaks()
    roof, roof_step, per_kernel = roofline(prof, nprof, c, n, args.precision, peaks, src, step_ms)
    P = c["npairs"]

    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline:
        cpu = cpu_baseline(g, kw, args.cpu_seconds)
        if cpu_inputs:
            extra["cpu_oracle"] = cpu_oracle_modes(cpu_inputs, args.cpu_seconds)
    line = {
        "metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32+f64",
        "data": "synthetic",
        "config": {"workload": spec.name, "n": n, "phi": spec.phi, "mu": spec.mu,
                   "radii": ("log-uniform in [%g, %g]" % (spec.a_min, spec.a_max) if spec.radii == "loguniform"
                             else "%g/%g, %g%% large" % (spec.a_small, spec.a_large, 100 * spec.frac_large)),
                   "capacity_M": c["M"], "precision": args.precision,
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "flushed before every timed step (256 MB write)",
                   "pairs": P, "contacts": c["ncontacts"], "cells": list(c["ncell"])},
        "roofline": roof,
        "roofline_step": roof_step,
        "kernels_ms": {k: round(v["ms"], 5) for k, v in per_kernel.items()},
        "kernels_bytes": {k: {"method": v["method_bytes"], "impl": v["impl_bytes"],
                              "method_gbs": round(v["gbs"], 1)} for k, v in per_kernel.items()},
        "kernels_note": "per-kernel times from a separate pass with CUDA events between kernels",
        "wall_s_timed_region": t_wall,
        "clocks": clk,
        "gpu_launches": KERNELS_PER_STEP * args.steps,
        "gpu_launches_note": "headline timed region: %d kernels per step graph" % KERNELS_PER_STEP,
        "e2e": {"value": e2e_value, "unit": "particle-steps/s", "h2d_bytes_per_step": bytes_state,
                "d2h_bytes_per_step": bytes_state + 72},
        "cpu_baseline": cpu,
        "modes": extra,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
