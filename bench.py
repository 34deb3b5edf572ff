#!/usr/bin/env python3
"""Zone-cycles/s of the Z4c RHS + RK4 hot path on GB300 (paper Sec. 5 metric).

Workload (default): single puncture, 128^3 cells as 2x2x2 MeshBlocks of 64^3
with 4 ghosts, [-16,16]^3, Sommerfeld outer boundary, 6th-order FD, KO 0.5,
1+log lapse, Gamma-driver (eta = 2), kappa1 = 0.02, Schwarzschild M = 1
(pre-collapsed lapse), RK4 at CFL 0.25.  A step is one full RK4 step (4
stages: ghost fill, fused RHS + stage update + enforcement, Sommerfeld
cells), replayed from a CUDA graph.  One zone-cycle = one interior cell
advanced by one RK4 step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--variant fp64|fp32]
  python bench.py --impl reference ...   (the FP64 CPU oracle as the reference arm)

Multi-GPU: one process per GPU, each evolving its own independent instance
(weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2409_10383_gb300 import inputs  # noqa: E402

METRIC = "Z4c zone-cycles/s per RK4 step on 1 GB300, FP64 vs FP32-RHS; % of roofline"
UNIT = "zone-cycles/s"
NOMINAL_FP64 = 1.25e12     # GB300 FP64, nominal (profiling recipe)
L2_BYTES = 129 * 2 ** 20

# Executed FP64 operations per interior cell per stage of the dominant kernel
# (interior_pre_kernel<6,false,1,false,72>: fused RHS + RK stage +
# enforcement, mixed derivatives from the pre-pass, strides of the 72^3
# storage of a 64^3 block with 4 ghosts), from the ncu instruction counters
# (dadd, dfma, dmul; exact integers per cell) of a one-block 64^3 order-6
# capture, stage-1 launch:
# flops = dadd + dmul + 2 dfma.
FP64_OPS_PER_CELL_STAGE = {6: dict(dadd=537, dfma=1389, dmul=469),
                           # 2nd order, 2 ghosts: interior_pre_kernel<2,false,1,false,68>
                           2: dict(dadd=353, dfma=928, dmul=456)}
# The same method as the oracle writes it out (oracle/flopcount.py: the
# oracle's RK4 step on a counting scalar type, per interior cell and stage):
# 49-point mixed stencils, separate KO and advection, full index loops.
# Reported beside the executed count as the cross-check; dividing it by the
# kernel time would read several times the FP64 peak.
ORACLE_FLOPS_PER_CELL_STAGE = {6: 21266.0, 4: 14184.6, 2: 9146.7}
# DRAM bytes (read + write) per interior cell of that launch
FP64_DRAM_BYTES_PER_CELL = {6: (121358336 + 91584512) / 262144, 2: (114248960 + 64636672) / 262144}
# FP32-RHS split schedule (interior_pre_kernel<6,true,4,split,72> storing k
# + split_epilogue_kernel): executed FP32 operations and the FP64 residue per
# interior cell per stage, from the same kind of capture
FP32_OPS_PER_CELL_STAGE = {6: dict(fadd=1085, ffma=1274, fmul=507)}
FP32_F64_RESIDUE_PER_CELL_STAGE = {6: dict(dadd=47, dfma=22, dmul=25)}
# keyed by (order, schedule, tile): the RHS kernel as it stands (with its L2
# prefetch of the rows 4 planes ahead, chi / gt diagonal / alpha stored
# minus one) + split_epilogue_kernel on the same tiles, one 64^3 block, RK
# stage 2 (which reads both u0 and the accumulator).  Schedules 4 and 6
# changed after their last capture, so they report no traffic.
FP32_DRAM_BYTES_PER_CELL = {(6, 5, "64x2"): (65961472 + 2135552 + 126968064 + 25498880) / 262144}
# algorithmic HBM bytes per zone-cycle (fused 3-register RK4, 22 FP64 fields;
# the same for the FP32-RHS path, whose state stays FP64)
ALG_BYTES_PER_ZONE_CYCLE = 352 * 8


def _rounded(x, sig=5):
    """Floats to `sig` significant digits (a shorter JSON line)."""
    if isinstance(x, float):
        return float(f"{x:.{sig}g}") if np.isfinite(x) else x
    if isinstance(x, dict):
        return {k: _rounded(v, sig) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [_rounded(v, sig) for v in x]
    return x


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(torch, x, ws, device="cuda"):
    """The largest x over the ranks: the job waits for its slowest rank."""
    if ws <= 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, ws, ms):
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (every rank runs its own instance: weak scaling)."""
    return units_per_rank * ws / (ms * 1e-3)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_sample(workload, steps, warmup, n0=None, threads=None):
    """The FP64 CPU oracle on a bounded sample of the workload: one block
    (the workload's block size unless n0 is given) of the same physics
    (order 6, KO 0.5, Sommerfeld boundary, puncture data), RK4 steps at CFL
    0.25, on all host cores unless threads is given."""
    from oracle import oracle
    oracle.build()
    cores = threads or host_cores()
    oracle.set_threads(cores)
    w = workload
    n0 = int(n0 or w["n"][0][0])
    lo = -float(w["h"][0]) * n0 / 2
    m = oracle.Mesh(n=[[n0] * 3], lo=[[lo] * 3], h=[float(w["h"][0])], ghosts=w["ghosts"],
                    order=w["order"], dom_lo=(lo,) * 3, dom_hi=(-lo,) * 3, periodic=w["periodic"],
                    lapse=w["lapse"], shift=w["shift"], ko_sigma=w["ko_sigma"], kappa1=w["kappa1"],
                    kappa2=w["kappa2"], eta=w["eta"], chi_floor=w["chi_floor"])
    u = m.initial_data(w["id_kind"], w["id_par"])
    dt = w["cfl"] * float(w["h"][0])
    for _ in range(warmup):
        m.rk4(u, dt, 1)
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        m.rk4(u, dt, 1)
        times.append(time.perf_counter() - t0)
    cells = n0 ** 3
    return dict(value=cells * steps / sum(times), unit=UNIT, cores=cores, kind="oracle",
                sample=f"{steps} RK4 step(s) of one {n0}^3 block on [{lo:g},{-lo:g}]^3 at h = {float(w['h'][0]):g} "
                       f"(order {w['order']}, KO {w['ko_sigma']}, Sommerfeld on all faces, puncture data at its "
                       f"centre; the per-cell work of the workload's blocks) after {warmup} warm-up",
                ms_per_step=1e3 * sum(times) / steps)


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None:
            return None
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.file.name)
        if not rows:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")
        sm = np.array([num(r[1]) for r in rows])
        mx = np.nanmax([num(r[2]) for r in rows])
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[q] for r in rows for q in range(4) if r[5 + q].lower().startswith("active")})
        return {"sm_mhz": float(np.nanmedian(sm)), "sm_max_mhz": float(mx), "reasons": reasons,
                "samples": len(rows), "power_w_max": float(np.nanmax([num(r[3]) for r in rows]))}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def run_reference(args, workload):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    res = oracle_sample(workload, max(1, args.steps), max(0, args.warmup))
    line = {"impl": "reference", "metric": METRIC, "value": res["value"], "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": res["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload["name"], "sample": res["sample"]},
            "cpu_baseline": {"value": res["value"], "unit": UNIT, "cores": res["cores"],
                             "kind": "oracle", "sample": res["sample"]},
            "e2e": {"value": res["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def measure(z4c, torch, workload, prec, args, ws, local):
    """Device-timed RK4 steps (CUDA graph replays) of one context, plus the
    live per-kernel timing, the roofline of the dominant kernel and the
    end-to-end host-buffer throughput."""
    g = z4c.Z4c.from_workload(workload, precision=prec)
    cells = int(np.prod(workload["n"], axis=1).sum())
    dt = workload["cfl"] * float(workload["h"][0])
    g.z4c_set_initial_data(workload["id_kind"], workload["id_par"])
    st = g.stream
    # pick the kernel variant (schedule, occupancy) on this GPU; U0 unchanged.
    # --no-autotune keeps the built-in default (FP64 schedule 2; FP32 split
    # schedule 4), e.g. for a profiler run whose serialised timings would
    # mislead the tuner
    variant = ((2, 1) if prec == 64 else (args.fp32_schedule, 4)) if args.no_autotune else g.z4c_autotune(8)
    if args.no_autotune:
        g.z4c_set_variant(*variant)
        if prec == 32:
            g.z4c_set_epilogue(args.fp32_epilogue)

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()

    # warm-up (also captures the CUDA graph of one RK4 step)
    g.z4c_rk4_step(dt, max(3, args.warmup))
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        e0.record(st)
        g.z4c_rk4_step(dt, args.steps)
        e1.record(st)
        barrier()
    ms = max_over_ranks(torch, e0.elapsed_time(e1), ws)
    value = job_value(cells * args.steps, ws, ms)

    # live per-kernel timing: CUDA events around each launch on the context's
    # stream (plain launches of the same kernels on the same state)
    kms = g.z4c_profile_steps(dt, 2)
    interior_ms = kms[1] / 4.0  # per launch (4 stages per step)
    peak64 = z4c.z4c_peak_fma(True, st)
    peak32 = z4c.z4c_peak_fma(False, st)
    conv = None
    if prec == 32:  # the FP32-RHS path converts every field twice per stage
        conv = {k: z4c.z4c_peak_convert(m, st) for k, m in
                (("f2d_hw", 0), ("f2d_int", 1), ("d2f_hw", 2), ("d2f_int", 3))}
    order = workload["order"]
    if prec == 64 and order in FP64_OPS_PER_CELL_STAGE:
        ops = FP64_OPS_PER_CELL_STAGE[order]
        flops = (ops["dadd"] + ops["dmul"] + 2 * ops["dfma"]) * cells
        insts = (ops["dadd"] + ops["dmul"] + ops["dfma"]) * cells
        achieved = flops / (interior_ms * 1e-3)
        ext = int(workload["n"][0][0]) + 2 * int(workload["ghosts"])  # storage extent the kernel is built for
        roof = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak64 / 1e12, "unit": "TFLOP/s",
                "frac": achieved / peak64,
                "traffic": FP64_DRAM_BYTES_PER_CELL[order] * cells,
                "traffic_note": "ncu dram bytes of a one-block 64^3 capture (stage 1) scaled by cells",
                "kernel": f"interior_pre_kernel<{order},false,1,false,{ext}> (fused RHS + RK stage + enforcement)",
                "peak_source": "measured DFMA throughput (z4c_peak_fma), FMA = 2 flops",
                "peak_nominal": NOMINAL_FP64 / 1e12,
                "fp64_issue_frac": insts / (interior_ms * 1e-3) / (peak64 / 2),
                "flops_per_cell_stage": flops / cells,
                "oracle_flops_per_cell_stage": ORACLE_FLOPS_PER_CELL_STAGE.get(order),
                "flops_note": "achieved counts the FP64 flops the kernel executes (ncu); the oracle's "
                              "plain formulation of the same step counts oracle_flops_per_cell_stage"}
    elif prec == 32 and order in FP32_OPS_PER_CELL_STAGE:
        # the slower of: FP32 flops at the FP32 peak, FP64-residue flops at
        # the FP64 peak, algorithmic bytes at the HBM bandwidth
        # (the FP64 residue is costed in pipe instructions: a DADD or DMUL
        # occupies the FP64 pipe as long as a DFMA, whose rate is peak64 / 2)
        o32, o64 = FP32_OPS_PER_CELL_STAGE[order], FP32_F64_RESIDUE_PER_CELL_STAGE[order]
        f32 = (o32["fadd"] + o32["fmul"] + 2 * o32["ffma"]) * cells
        f64 = (o64["dadd"] + o64["dmul"] + 2 * o64["dfma"]) * cells
        i64 = (o64["dadd"] + o64["dmul"] + o64["dfma"]) * cells
        byt = ALG_BYTES_PER_ZONE_CYCLE / 4 * cells
        hbm = measured_peaks().get("hbm_gbs", 6800.0) * 1e9
        t = {"fp32_alu": f32 / peak32, "fp64_residue": i64 / (peak64 / 2), "hbm": byt / hbm}
        kind = max(t, key=t.get)
        sec = interior_ms * 1e-3
        if kind == "hbm":
            roof = {"bound": "hbm", "achieved": byt / sec / 1e9, "peak": hbm / 1e9, "unit": "GB/s",
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)"}
        elif kind == "fp32_alu":
            roof = {"bound": "alu", "achieved": f32 / sec / 1e12, "peak": peak32 / 1e12, "unit": "TFLOP/s",
                    "peak_source": "measured FP32 FMA throughput (z4c_peak_fma), FMA = 2 flops"}
        else:
            roof = {"bound": "alu", "achieved": i64 / sec / 1e12, "peak": peak64 / 2 / 1e12,
                    "unit": "T FP64-pipe instructions/s",
                    "peak_source": "measured DFMA instruction rate (z4c_peak_fma FP64 / 2)",
                    "fp64_residue_flops_per_cell_stage": f64 / cells}
        ext = int(workload["n"][0][0]) + 2 * int(workload["ghosts"])
        n0 = int(workload["n"][0][0])
        shape = "64x2" if n0 % 64 == 0 else "32x4" if n0 % 32 == 0 else "16x8"
        per_cell = FP32_DRAM_BYTES_PER_CELL.get((order, variant[0], shape if variant[0] >= 5 else "16x8"))
        traffic = per_cell * cells if per_cell is not None else None
        kname = {4: f"interior_pre_kernel<{order},true,4,split,{ext}> (16x8 tiles)",
                 5: f"interior_pre_kernel<{order},true,4,split,{ext},wide> ({shape} tiles)",
                 6: f"interior_pair_kernel<{order},{ext},wide> (two cells per thread, f32x2, {shape} tiles)"}
        roof.update({"frac": t[kind] / sec, "limiter": kind,
                     "traffic": traffic,
                     "traffic_note": "ncu dram bytes of the RHS and stage-update kernels, one 64^3 block, "
                                     "scaled by cells (RK stage 2: u0 and accumulator read)",
                     "kernel": (kname[variant[0]] + " + split_epilogue_kernel (FP32 RHS, FP64 state/RK/enforcement)")
                     if variant[0] in kname else
                     f"interior_pre_kernel<{order},true,{variant[1]}> (FP32 RHS, FP64 state/RK/enforcement)",
                     "bound_ms_per_launch": {k: v * 1e3 for k, v in t.items()},
                     "fracs": {k: v / sec for k, v in t.items()}})
    else:
        bytes_launch = ALG_BYTES_PER_ZONE_CYCLE / 4 * cells
        hbm = measured_peaks().get("hbm_gbs", 6800.0)
        achieved = bytes_launch / (interior_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": None, "kernel": f"interior_pre_kernel<{order},{'true' if prec == 32 else 'false'}>",
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)",
                "note": "algorithmic bytes view (no instruction counts taken for this order)"}
    roof["kernel_ms_per_launch"] = interior_ms
    roof["step_share"] = {"ghost": kms[0] / kms.sum(), "prepass": kms[3] / kms.sum(),
                          "interior": kms[1] / kms.sum(), "sommerfeld": kms[2] / kms.sum()}
    roof["fp64_fma_peak_tflops"] = peak64 / 1e12
    roof["fp32_fma_peak_tflops"] = peak32 / 1e12
    if conv:
        roof["conversions_per_s"] = conv

    # end to end through the C ABI with pinned host buffers: every step copies
    # the state host -> device, runs one RK4 step and copies it back
    nbytes = g.state_bytes
    hin = torch.empty(nbytes // 8, dtype=torch.float64, pin_memory=True)
    hout = torch.empty(nbytes // 8, dtype=torch.float64, pin_memory=True)
    hin.numpy()[:] = g.z4c_get_state()
    g.z4c_evolve_host(hin, hout, dt, 1)
    e2e_steps = max(2, min(args.steps, 10))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        g.z4c_evolve_host(hin, hout, dt, 1)
    t1 = time.perf_counter()
    barrier()
    e2e = {"value": cells * e2e_steps * ws / (t1 - t0), "unit": UNIT, "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": nbytes}
    tx, ty, cpt = g.z4c_tile_shape(0)
    roof["variant"] = {"schedule": variant[0], "occupancy": variant[1],
                       "tile": f"{tx}x{ty}", "cells_per_thread": cpt}
    if prec == 32:  # which y/z pre-pass the kept variant runs
        roof["variant"]["prepass"] = "tma" if g.z4c_prepass_tma_blocks() > 0 else "plane"
    # the Weyl scalar Psi4 on the grid (Sec. 3.3 diagnostic, FP64): one
    # synchronous call = ghost fill + Psi4 at every interior cell
    psi4 = None
    if prec == 64:
        buf = g.z4c_psi4()
        reps = 3
        t0 = time.perf_counter()
        for _ in range(reps):
            g.z4c_psi4(out=buf)
        t1 = time.perf_counter()
        psi4 = {"ms_per_call": (t1 - t0) / reps * 1e3, "value": cells * reps / (t1 - t0), "unit": "cells/s",
                "note": "z4c_psi4 on the benchmark state: ghost fill + Psi4 (coordinate tetrad) at every interior cell"}
        del buf
    out = dict(value=value, ms_per_step=ms / args.steps, roofline=roof, e2e=e2e,
               gpu_launches=g.z4c_launches_per_step() * args.steps, clocks=clk.summary(),
               cells=cells, dt=dt, state_bytes=nbytes, psi4=psi4)
    g.close()
    del g
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------------------
# FP32-RHS acceptance against the FP64 truncation error (Sec. 4.1: accuracy
# is judged by convergence under resolution).  The FP32-induced difference
# of each field, |u32 - u64| at spacing h, is compared with a Richardson
# estimate of the FP64 truncation error at h, |u64(2h) - u64(h)| / (2^p - 1),
# both away from the puncture (r > r_min).  The spacings are cell-centred,
# so the fine solution is carried to the coarse cell centres by the
# 6-point midpoint Lagrange interpolation per axis (exact to degree 5).
# ---------------------------------------------------------------------------
MIDPOINT_W = np.array([3.0, -25.0, 150.0, 150.0, -25.0, 3.0]) / 256.0


def puncture_workload(N, nb, half):
    """The single-puncture physics of the benchmark (order 6, 4 ghosts, KO
    0.5, 1+log, Gamma-driver, Sommerfeld, Schwarzschild M = 1) on N^3 cells
    of [-half, half]^3 as nb^3 blocks."""
    w = inputs.workload("single_puncture_128")
    n, lo, h = inputs.uniform_blocks((nb,) * 3, N // nb, (-half,) * 3, (half,) * 3)
    w.update(name=f"single_puncture_{N}_{nb}_L{half:g}", n=n, lo=lo, h=h, dom_lo=(-half,) * 3,
             dom_hi=(half,) * 3)
    return w


def global_interior(w, state):
    """(22, N, N, N) interior values [f][k][j][i] of a uniform block layout."""
    n = np.asarray(w["n"][0], int)
    gw = int(w["ghosts"])
    h = float(w["h"][0])
    e = n + 2 * gw
    nblk = len(w["n"])
    u = state.reshape(nblk, 22, e[2], e[1], e[0])
    N = np.rint((np.asarray(w["dom_hi"]) - np.asarray(w["dom_lo"])) / h).astype(int)
    G = np.empty((22, N[2], N[1], N[0]))
    for b in range(nblk):
        o = np.rint((np.asarray(w["lo"][b]) - np.asarray(w["dom_lo"])) / h).astype(int)
        G[:, o[2]:o[2] + n[2], o[1]:o[1] + n[1], o[0]:o[0] + n[0]] = \
            u[b][:, gw:gw + n[2], gw:gw + n[1], gw:gw + n[0]]
    return G


def to_coarse(G):
    """Fine cell-centred values (.., N, N, N) at the centres of the 2h cells
    (.., N/2, N/2, N/2): per axis, coarse cell c from fine cells 2c-2..2c+3;
    coarse cells whose stencil leaves the array are NaN."""
    out = G
    for ax in (-1, -2, -3):
        N = out.shape[ax]
        Nc = N // 2
        x = np.moveaxis(out, ax, -1)
        r = np.full(x.shape[:-1] + (Nc,), np.nan)
        for c in range(1, Nc - 1):
            r[..., c] = x[..., 2 * c - 2:2 * c + 4] @ MIDPOINT_W
        out = np.moveaxis(r, -1, ax)
    return out


def radius(N, half):
    h = 2.0 * half / N
    x = -half + h * (np.arange(N) + 0.5)
    return np.sqrt(x[None, None, :] ** 2 + x[None, :, None] ** 2 + x[:, None, None] ** 2)


def rms(x, mask):
    v = x[..., mask]
    return np.sqrt(np.nanmean(v * v, axis=-1))


def fp32_acceptance(fine64, fine32, coarse64, half, p=None, finer64=None, r_min=1.0):
    """Per field: the FP32-induced RMS difference at spacing h over the
    Richardson estimate of the FP64 truncation error at h, over r > r_min.
    fineXX / coarse64 / finer64: (22, N, N, N) interior arrays at h, 2h,
    h/2.  p: the convergence order; measured from the three FP64 runs when
    finer64 is given (per field, then the median over fields), else as
    given.  Also the same for the puncture lapse (min alpha) and the raw
    differences, so that any other order can be applied."""
    N = fine64.shape[-1]
    # the coarse cells next to the outer face have no full stencil: leave
    # out those and the fine cells they cover
    inner = np.zeros(N, bool)
    inner[2:N - 2] = True
    rf = (radius(N, half) > r_min) & inner[None, None, :] & inner[None, :, None] & inner[:, None, None]
    rc = radius(N // 2, half) > r_min
    d32 = rms(fine32 - fine64, rf)
    dc = rms(to_coarse(fine64) - coarse64, rc)
    orders = None
    if finer64 is not None:
        dff = rms(to_coarse(finer64) - fine64, rf)
        moved = (dc > 0) & (dff > 0)
        orders = np.where(moved, np.log2(np.where(moved, dc, 1) / np.where(moved, dff, 1)), np.nan)
        if p is None:
            p = float(np.nanmedian(orders))
    est = dc / (2.0 ** p - 1.0)
    ratio = np.where(est > 0, d32 / np.where(est > 0, est, 1), 0.0)
    a64, a32, a2h = fine64[18].min(), fine32[18].min(), coarse64[18].min()
    lap_est = abs(a2h - a64) / (2.0 ** p - 1.0)
    out = {"order_p": p, "r_min": r_min, "fp32_rms_diff": d32.tolist(), "fp64_trunc_est_rms": est.tolist(),
           "ratio": ratio.tolist(), "max_ratio": float(ratio.max()), "worst_field": int(ratio.argmax()),
           "puncture_lapse": {"fp64": float(a64), "fp32": float(a32), "fp64_2h": float(a2h),
                              "ratio": float(abs(a32 - a64) / lap_est) if lap_est > 0 else 0.0}}
    if orders is not None:
        out["orders_per_field"] = orders.tolist()
    return out


def run_puncture(z4c, w, prec, t_end):
    """Evolve w to t_end at CFL 0.25; its interior, ||H||_2 over r > 1 and
    min alpha."""
    g = z4c.Z4c.from_workload(w, precision=prec)
    g.z4c_set_initial_data(w["id_kind"], w["id_par"])
    dt = w["cfl"] * float(w["h"][0])
    steps = int(round(t_end / dt))
    g.z4c_rk4_step(dt, steps)
    G = global_interior(w, g.z4c_get_state())
    H = float(g.z4c_constraints(r_mask=1.0)[0][0])
    g.close()
    return G, H, steps


def fp32_truncation_check(z4c, N=128, nb=2, half=16.0, steps=50, finer=False):
    """The FP32-RHS path at N^3 against the FP64 truncation error there
    (FP64 at N^3 and (N/2)^3, and at (2N)^3 if finer): `steps` RK4 steps
    at N^3 (t = steps * 0.25 h), the coarse run to the same time."""
    wf, wc = puncture_workload(N, nb, half), puncture_workload(N // 2, nb, half)
    t_end = steps * 0.25 * float(wf["h"][0])
    f64, H64, _ = run_puncture(z4c, wf, 64, t_end)
    f32, H32, _ = run_puncture(z4c, wf, 32, t_end)
    c64, H2h, _ = run_puncture(z4c, wc, 64, t_end)
    ff64 = None
    Hh2 = None
    if finer:
        ff64, Hh2, _ = run_puncture(z4c, puncture_workload(2 * N, nb, half), 64, t_end)
    res = fp32_acceptance(f64, f32, c64, half, p=None if finer else 4.0, finer64=ff64)
    res.update({"N": N, "half": half, "steps": steps, "t": t_end,
                "hamiltonian_l2": {"fp64": H64, "fp32": H32, "fp64_2h": H2h, "fp64_h2": Hh2,
                                   "ratio_to_own": abs(H32 - H64) / H64}})
    if not finer:
        res["order_note"] = "p = 4 (RK4 at fixed CFL) assumed: no third resolution in this run"
    return res


def measure_batch(z4c, torch, steps, warmup, autotune=True):
    """The uneven batch (80 independent single-block problems: punctures and
    gauge waves of 24^3..96^3, orders 4/6, FP64 and FP32-RHS) evolved
    together, one CUDA-graph launch per RK4 step, each instance with its
    own dt; kernel variants autotuned (else the built-in defaults)."""
    ws = inputs.uneven_batch()
    g = z4c.Z4c.batch(ws)
    for i, w in enumerate(ws):
        g.z4c_set_initial_data_instance(i, w["id_kind"], w["id_par"])
    variant = g.z4c_autotune(2) if autotune else (4, 4)
    if not autotune:
        g.z4c_set_variant(*variant)
    dts = [w["cfl"] * float(w["h"][0]) for w in ws]
    cells = sum(int(np.prod(w["n"], axis=1).sum()) for w in ws)
    g.z4c_rk4_step_batch(dts, max(1, warmup))
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(g.stream)
    g.z4c_rk4_step_batch(dts, steps)
    e1.record(g.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    mix = {}
    for w in ws:
        key = f"order{w['order']}_fp{w['precision']}"
        mix[key] = mix.get(key, 0) + int(np.prod(w["n"], axis=1).sum())
    out = {"value": cells * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps, "steps": steps,
           "instances": len(ws), "cells": cells, "cells_by_kind": mix,
           "gpu_launches": g.z4c_launches_per_step() * steps, "graph_launches_per_step": 1,
           "variant_fp32": {"schedule": variant[0], "occupancy": variant[1]},
           "workload": "uneven batch: 64 punctures (M in [0.5,2]) + 16 gauge waves (A in [0.001,0.1]), "
                       "sizes {24,48,64,96}^3, orders 4/6, FP64/FP32-RHS, seed 20240916"}
    g.close()
    del g
    torch.cuda.empty_cache()
    return out


def measure_smr(z4c, torch, steps, warmup):
    """The refined two-puncture mesh (680 blocks of 16^3 on levels 0..6,
    h = 2 .. 1/32, Brill-Lindquist m = 1/2 at x = +-3): whole RK4 steps with
    restriction / prolongation ghost transfer, one CUDA-graph launch per
    step, dt = 1/128 for every block; plus the per-kind time split of one
    step (ghost fill including the refinement transfer, pre-pass, fused
    RHS + update, Sommerfeld)."""
    w = inputs.workload("bl_binary_smr")
    g = z4c.Z4c.from_workload(w)
    g.z4c_set_initial_data(w["id_kind"], w["id_par"])
    dt = w["dt"]
    cells = int(np.prod(w["n"], axis=1).sum())
    g.z4c_rk4_step(dt, max(1, warmup))
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(g.stream)
    g.z4c_rk4_step(dt, steps)
    e1.record(g.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    split = g.z4c_profile_steps(dt, 1)
    h_norm = float(g.z4c_constraints()[0][0])
    # diagnostics beside the step: per-block refinement indicators and one
    # tracker step of both punctures (synchronous calls, each including a
    # ghost fill of U0 and the small device-to-host copy)
    reps = 10
    t0 = time.perf_counter()
    for _ in range(reps):
        g.z4c_block_indicators()
    t1 = time.perf_counter()
    pts = np.array([[3.0, 0.0, 0.0], [-3.0, 0.0, 0.0]])
    for _ in range(reps):
        pts, _ = g.z4c_track_punctures(pts, dt)
    t2 = time.perf_counter()
    out = {"value": cells * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps, "steps": steps,
           "blocks": int(len(w["h"])), "levels": np.bincount(w["level"]).tolist(), "cells": cells,
           "storage_per_register_bytes": int(g.nelem * 8),
           "split_ms_per_step": {"ghost_fill_incl_refinement": split[0], "prepass": split[3],
                                 "fused_rhs_update": split[1], "sommerfeld": split[2]},
           "ghost_share": float(split[0] / split.sum()),
           "hamiltonian_l2_after": h_norm,
           "diagnostics_ms_per_call": {"block_indicators": 1e3 * (t1 - t0) / reps,
                                       "track_punctures": 1e3 * (t2 - t1) / reps},
           "gpu_launches": g.z4c_launches_per_step() * steps, "graph_launches_per_step": 1,
           "workload": "Brill-Lindquist binary m=0.5 at x=+-3, 680 blocks of 16^3, levels 0..6 "
                       "(h=2..1/32), [-32,32]^3, order 6, 4 ghosts, dt=1/128"}
    g.close()
    del g
    torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--variant", default="both", choices=["fp64", "fp32", "both"])
    ap.add_argument("--workload", default="single_puncture_128")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-steps", type=int, default=2)
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--batch-steps", type=int, default=5)
    ap.add_argument("--no-smr", action="store_true")
    ap.add_argument("--smr-steps", type=int, default=50)
    ap.add_argument("--no-order2", action="store_true",
                    help="skip the 2nd-order (2 ghosts) variant of the workload")
    ap.add_argument("--no-table1", action="store_true",
                    help="skip the paper's Table-1 workload (linear wave on 64^3 blocks)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default kernel variant instead of timing the candidates")
    ap.add_argument("--fp32-schedule", type=int, default=4, choices=[4, 5, 6],
                    help="with --no-autotune: the FP32-RHS split schedule (4: 16x8 tiles; 5: wide tiles; "
                         "6: wide tiles, two cells per thread)")
    ap.add_argument("--fp32-epilogue", type=int, default=0, choices=[0, 1],
                    help="with --no-autotune: the FP32-RHS stage-update kernel (0 plain, 1 fed by bulk copies)")
    ap.add_argument("--smr-only", action="store_true",
                    help="time only the refined two-puncture workload (prints its object)")
    args = ap.parse_args()
    workload = inputs.workload(args.workload)

    if args.impl == "reference":
        run_reference(args, workload)
        return

    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_2409_10383_gb300 import z4c

    if args.smr_only:
        print(json.dumps({"smr": measure_smr(z4c, torch, args.smr_steps, args.warmup)}), flush=True)
        return
    res = {}
    if args.variant in ("fp64", "both"):
        res[64] = measure(z4c, torch, workload, 64, args, ws, local)
    if args.variant in ("fp32", "both"):
        res[32] = measure(z4c, torch, workload, 32, args, ws, local)
    prim = 64 if 64 in res else 32
    r = res[prim]
    batched = None
    if not args.no_batch and args.variant == "both":
        batched = measure_batch(z4c, torch, args.batch_steps, 2, autotune=not args.no_autotune)
        if ws > 1:
            batched["value"] = job_value(batched["cells"], ws, max_over_ranks(torch, batched["ms_per_step"], ws))

    smr = None
    if not args.no_smr and args.variant == "both":
        smr = measure_smr(z4c, torch, args.smr_steps, 2)
        if ws > 1:
            smr["value"] = job_value(smr["cells"], ws, max_over_ranks(torch, smr["ms_per_step"], ws))

    order2 = None
    if not args.no_order2 and args.variant == "both" and workload["order"] != 2:
        w2 = inputs.workload(args.workload + "_o2")
        q = measure(z4c, torch, w2, 64, args, ws, local)
        order2 = {"value": q["value"], "unit": UNIT, "ms_per_step": q["ms_per_step"], "dtype": "f64",
                  "config": {"workload": w2["name"], "fd_order": 2, "ghosts": 2, "cells": q["cells"],
                             "dt": q["dt"]},
                  "roofline": q["roofline"], "e2e": q["e2e"], "gpu_launches": q["gpu_launches"],
                  "clocks": q["clocks"]}

    acc32 = None
    if rank == 0 and 64 in res and 32 in res and args.workload == "single_puncture_128":
        # the FP32-RHS configuration: 50 steps of the benchmark workload
        t = fp32_truncation_check(z4c, N=128, nb=2, half=16.0, steps=50)
        acc32 = {"steps": t["steps"], "t": t["t"], "order_p": t["order_p"], "r_min": t["r_min"],
                 "max_ratio_fp32_diff_to_fp64_trunc": t["max_ratio"], "worst_field": t["worst_field"],
                 "ratio_per_field": [round(x, 5) for x in t["ratio"]],
                 "puncture_lapse": t["puncture_lapse"], "hamiltonian_l2": t["hamiltonian_l2"],
                 "note": "per field: RMS |u32 - u64| at h over the Richardson FP64 truncation estimate "
                         "|u64(2h) - u64(h)| / (2^p - 1), r > r_min; " + t.get("order_note", "")}

    # the paper's Table-1 throughput workload (context: the paper's numbers
    # are on other hardware)
    table1 = None
    if not args.no_table1 and args.variant == "both" and args.workload == "single_puncture_128":
        w1 = inputs.workload("linear_wave_256")
        q = measure(z4c, torch, w1, 64, args, ws, local)
        table1 = {"value": q["value"], "unit": UNIT, "ms_per_step": q["ms_per_step"], "dtype": "f64",
                  "config": {"workload": w1["name"], "blocks": int(len(w1["n"])), "block": [64, 64, 64],
                             "cells": q["cells"], "fd_order": 6, "ghosts": 4},
                  "paper_zcps_context": {"GH200": 2.46e7, "A100": 1.36e7, "MI250X_die": 5.08e6},
                  "roofline": {k: q["roofline"][k] for k in ("frac", "fp64_issue_frac", "kernel_ms_per_launch")},
                  "e2e": q["e2e"], "gpu_launches": q["gpu_launches"], "clocks": q["clocks"]}

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        c = oracle_sample(workload, args.cpu_steps, 1)
        cpu = {k: c[k] for k in ("value", "unit", "cores", "kind", "sample")}
        # the same oracle on one core (a smaller block keeps it to about a second)
        c1 = oracle_sample(workload, 1, 0, n0=32, threads=1)
        cpu["single_thread"] = {k: c1[k] for k in ("value", "unit", "cores", "sample")}
    order = workload["order"]
    line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prim == 64 else "f32+f64",
            "data": "synthetic",
            "config": {"workload": workload["name"], "variant": "fp64" if prim == 64 else "fp32_rhs",
                       "cells": r["cells"], "blocks": int(len(workload["n"])),
                       "block": list(map(int, workload["n"][0])), "ghosts": workload["ghosts"],
                       "fd_order": order, "dt": r["dt"],
                       "l2": f"inputs larger than L2 ({4 * r['state_bytes'] / 2**30:.2f} GiB of "
                             f"registers vs {L2_BYTES / 2**20:.0f} MiB L2)",
                       "parallelism": f"{ws} independent instance(s)"},
            "roofline": r["roofline"], "cpu_baseline": cpu, "e2e": r["e2e"],
            "gpu_launches": r["gpu_launches"], "clocks": r["clocks"]}
    # detail objects first, then the batched and FP32-RHS results, then a
    # compact headline: a reader of the end of the line sees all three paths
    if r.get("psi4"):
        line["psi4"] = r["psi4"]
    if smr is not None:
        line["smr"] = smr
    if order2 is not None:
        line["order2"] = order2
    if table1 is not None:
        line["paper_table1"] = table1
    if batched is not None:
        line["batched"] = batched
    head = {("fp64" if prim == 64 else "fp32_rhs"): {
        "value": r["value"], "ms_per_step": r["ms_per_step"], "roofline_frac": r["roofline"]["frac"],
        "bound": "FP64 pipe" if prim == 64 else r["roofline"].get("limiter")}}
    if prim == 64 and 32 in res:
        q = res[32]
        qr = q["roofline"]
        line["fp32_rhs"] = {"value": q["value"], "unit": UNIT, "ms_per_step": q["ms_per_step"],
                            "dtype": "f32 stencils/algebra + f64 state, RK, 1/chi, enforcement",
                            "speedup_vs_fp64": q["value"] / r["value"], "roofline": qr,
                            "e2e": q["e2e"], "gpu_launches": q["gpu_launches"], "clocks": q["clocks"],
                            "accuracy_vs_fp64": acc32}
        head["fp32_rhs"] = {"value": q["value"], "ms_per_step": q["ms_per_step"],
                            "speedup_vs_fp64": q["value"] / r["value"], "roofline_frac": qr["frac"],
                            "limiter": qr.get("limiter"), "kernel_ms_per_launch": qr["kernel_ms_per_launch"],
                            "e2e": q["e2e"]["value"], "clocks_sm_mhz": (q["clocks"] or {}).get("sm_mhz")}
        if acc32:
            head["fp32_rhs"]["max_ratio_fp32_diff_to_fp64_trunc"] = acc32["max_ratio_fp32_diff_to_fp64_trunc"]
            head["fp32_rhs"]["hamiltonian_l2_rel_diff"] = acc32["hamiltonian_l2"]["ratio_to_own"]
    if batched is not None:
        head["batched"] = {"value": batched["value"], "ms_per_step": batched["ms_per_step"],
                           "speedup_vs_fp64": batched["value"] / r["value"], "instances": batched["instances"]}
    line["headline"] = head
    line = _rounded(line)
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
