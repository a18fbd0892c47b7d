#!/usr/bin/env python
"""Benchmark of the multipole Poisson solve on one GB300 (or N replicas).

Workload: presupernova-like core, 512 x 128 x 256 cells (geometric shells over
[1e5, 1e10] cm), l_max = 16, density rho_c/(1+(r/r_c)^2)^1.5 times seeded
l <= 4 harmonic perturbations (seed 2).  One step = one full solve (moments,
radial recurrences, potential) of that density, resident in HBM, through the
C ABI (mp_solve) on the split-precision BF16x3 tensor-core path.

Also reported on the same line: the float64 GPU path on the same workload,
the accuracy of both against the FP64 CPU oracle, an end-to-end number with
pinned host buffers (mp_solve_host_async: every step copies rho host->device,
solves and copies Phi device->host; one step's download overlaps the next step's
upload), per-kernel timing with the dominant kernel's HBM roofline fraction,
SM clocks sampled during the timed region, and the oracle timed on the host
cores as a CPU baseline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 the script runs under torch.distributed.run, one rank per GPU, each
rank solving its own replica of the workload (no data exchange); the job value
is the total solves/s over ranks timed by the slowest rank.  --impl reference
times the FP64 CPU oracle on the host cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Poisson solves/s & Gcell*mode/s, BF16x3 vs FP64 GPU at <=1e-6 rel err in Phi"
WORKLOADS = {
    # the benchmarked configuration (default)
    "presn": "presupernova core 512x128x256 cells, geometric r in [1e5,1e10] cm, l_max=16, seed 2",
    # a larger one for measurement and profiling of the large-table kernels
    "lognormal": "log-normal angular field 1024x256x512 cells, geometric r in [1e5,1e12] cm, l_max=32, seed 3",
}
SPLIT_PRECISION = "bf16x3"

# DRAM bytes (read + write) per launch from one ncu capture of the same
# workload, valid while the kernel source hashes match.
# kernel name: (DRAM bytes read + written per launch from one ncu capture (profiles/),
#               source file of the kernel, sha1 of that file and the shared headers at
#               capture time); an entry whose sources changed since is ignored
NCU_TRAFFIC = {
    "split_phi_project_tc": (134318592 + 3101952, "mp_split.cu", "055b2c945b2aba8b5d946b7478e317e01773fdc1"),
}
KERNEL_HEADERS = ("ptx.cuh", "mp_internal.h", "mp_errors.h")


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10000)
    p.add_argument("--warmup", type=int, default=50)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--cpu-seconds", type=float, default=10.0, help="oracle CPU-baseline budget")
    p.add_argument("--workload", choices=sorted(WORKLOADS), default="presn",
                   help="mesh and density (presn is the benchmarked configuration)")
    return p.parse_args()


def dist_info():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def source_hash(source: str):
    """sha1 over one CUDA source file of the package and the headers it shares."""
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_2602_02507_gb300", "csrc")
    for name in (source,) + KERNEL_HEADERS:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.proc = None
        self.path = None
        self.dev = device_index

    def start(self):
        try:
            import torch
            bus = None
            props = torch.cuda.get_device_properties(self.dev)
            if hasattr(props, "pci_bus_id"):
                bus = "%08x:%02x:%02x.0" % (getattr(props, "pci_domain_id", 0), props.pci_bus_id,
                                            getattr(props, "pci_device_id", 0))
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
            if bus:
                cmd += ["--id=" + bus]
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception as e:  # no nvidia-smi: clocks stay unknown
            log("clock sampler unavailable:", e)
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 7:
                    continue
                try:
                    sm.append(float(parts[0]))
                    smax.append(float(parts[1]))
                    power.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[3:7]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


# ---------------------------------------------------------------- oracle timing
def cpu_baseline_leg(w, budget_s: float, max_reps: int = 200):
    """The oracle on the host cores: solves of the workload for about budget_s seconds.
    Returns (solves/s, solves, seconds, threads, Phi of the first solve); that Phi is the
    reference the GPU paths' accuracy is stated against."""
    from oracle import oracle as O
    m = w.mesh
    tab = O.build_tables(m.r, m.theta, m.phi, m.L)
    phi_ref = O.solve(tab, w.rho, m.G)["phi"]  # also warms caches and threads
    reps, t0 = 0, time.perf_counter()
    while True:
        O.solve(tab, w.rho, m.G)
        reps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or reps >= max_reps:
            break
    return reps / el, reps, el, O.get_threads(), phi_ref


# ---------------------------------------------------------------- reference arm
def run_reference(args):
    world, rank, _ = dist_info()
    if rank != 0:
        return 0
    from oracle import build as oracle_build
    from oracle import oracle as O
    from paper_2602_02507_gb300 import workloads as W
    oracle_build.build()
    w = getattr(W, args.workload)()
    m = w.mesh
    tab = O.build_tables(m.r, m.theta, m.phi, m.L)
    for _ in range(args.warmup):
        O.solve(tab, w.rho, m.G)
    steps = max(1, min(args.steps, 30))
    t0 = time.perf_counter()
    for _ in range(steps):
        O.solve(tab, w.rho, m.G)
    el = time.perf_counter() - t0
    value = steps / el
    sample = f"the whole workload per step: factored FP64 oracle solve, tables prebuilt, {steps} steps"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "precision": "fp64 (CPU oracle)", "cells": m.cells,
                   "l_max": m.L},
        "gcell_mode_per_s": value * m.cells * m.KL / 1e9,
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": O.get_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- multi-rank helpers
def max_over_ranks_on(x: float, world: int, device) -> float:
    """Largest x over the ranks of the default process group (x itself at world 1)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, steps: int, total_ms: float) -> float:
    """Solves per second of the whole job: every rank solves `steps` replicas of the
    workload; the slowest rank's time (total_ms) bounds the job."""
    return world * steps / (total_ms * 1e-3)


# ---------------------------------------------------------------- our arm
def alg_bytes(kernel: str, cells: int, rows: int, n_r: int, L: int, KL: int):
    """Algorithmic DRAM bytes per launch (each input read once, each output written once)."""
    P = 2 * L + 1
    table = {
        "split_phi_project_tc": 8 * cells + 4 * rows * P,        # rho in, F out (float32, 2L+1 columns)
        "split_synth_tc": 8 * cells,                             # Phi out (coefficients are L2-resident)
        "split_theta_contract": 4 * rows * P + 8 * n_r * KL,     # F in, moments out
        "radial_scan": 8 * n_r * KL * 2 + 16 * (n_r + 1) * KL + 4 * n_r * KL,  # A in; C, MR, MI, C32 out
        "split_theta_synth": rows * (4 * ((2 * L + 15) // 16 * 16) + 4),       # bf16 x2 G terms + m = 0 column out
        "fp64_phi_project": 8 * cells + 8 * rows * P,
        "fp64_theta_contract": 8 * rows * P + 8 * n_r * KL,
        "fp64_theta_synth": 8 * rows * P,
        "fp64_phi_synth": 8 * cells + 8 * rows * P,
    }
    return table.get(kernel)


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    world, rank, local = dist_info()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__ as g
    g.build()
    from paper_2602_02507_gb300 import multipole as mpl
    from paper_2602_02507_gb300 import workloads as W

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(x: float) -> float:
        return max_over_ranks_on(x, world, "cuda")

    w = getattr(W, args.workload)()
    m = w.mesh
    cells, KL = m.cells, m.KL
    rows = m.shape[0] * m.shape[1]
    stream = torch.cuda.current_stream()
    rho = torch.from_numpy(w.rho).cuda()
    phi = torch.empty_like(rho)
    phi64 = torch.empty_like(rho)
    mesh = mpl.Mesh(m.r, m.theta, m.phi, m.L, m.G, precision=SPLIT_PRECISION, stream=stream)
    mesh64 = mpl.Mesh(m.r, m.theta, m.phi, m.L, m.G, precision="fp64", stream=stream)
    for ms_, out in ((mesh, phi), (mesh64, phi64)):
        ms_.set_density(rho)
        ms_.set_phi_output(out)
        ms_.solve()
        ms_.synchronize()

    # accuracy against the FP64 CPU oracle (rank 0) and between the GPU paths
    acc = {"tolerance": 1e-6}
    p_split = phi.cpu().numpy()
    p64 = phi64.cpu().numpy()
    acc["phi_max_rel_err_split_vs_fp64_gpu"] = float(np.max(np.abs(p_split - p64) / np.abs(p64)))
    cpu = None
    if rank == 0 and world == 1:
        v, reps, el, cores, ref = cpu_baseline_leg(w, args.cpu_seconds)
        cpu = {"value": v, "unit": "solves/s", "cores": cores, "kind": "oracle",
               "sample": f"{reps} whole-workload solves (factored FP64 oracle, tables prebuilt) in {el:.1f} s"}
        acc["phi_max_rel_err_split_vs_oracle"] = float(np.max(np.abs(p_split - ref) / np.abs(ref)))
        acc["phi_max_rel_err_fp64_gpu_vs_oracle"] = float(np.max(np.abs(p64 - ref) / np.abs(ref)))

    # ---- timed region: split path, K solves (each one CUDA graph launch of the kernel chain)
    for _ in range(args.warmup):
        mesh.solve()
    mesh.synchronize()
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        mesh.solve()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    mesh.synchronize()
    local_ms = ev0.elapsed_time(ev1)
    total_ms = max_over_ranks(local_ms)
    ms_per_step = total_ms / args.steps
    value = whole_job_rate(world, args.steps, total_ms)

    # ---- per-kernel durations: the same solves launched kernel by kernel with CUDA events
    # between them on the mesh stream (events cost a little time of their own)
    kp = max(3, min(args.steps, 1000))
    mesh.profile(True)
    for _ in range(kp):
        mesh.solve()
    prof = mesh.profile_read()
    mesh.profile(False)
    prof_ms_per_step = sum(v["total_ms"] for v in prof.values()) / kp

    # ---- float64 GPU path on the same workload
    k64 = max(3, min(args.steps // 50, 200))
    for _ in range(2):
        mesh64.solve()
    mesh64.synchronize()
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(k64):
        mesh64.solve()
    e1.record(stream)
    torch.cuda.synchronize()
    ms64 = max_over_ranks(e0.elapsed_time(e1)) / k64
    mesh64.synchronize()

    # ---- end to end through the C ABI with pinned host buffers
    rho_h = torch.from_numpy(w.rho).pin_memory()
    phi_h = torch.empty_like(rho_h).pin_memory()
    ke = max(3, min(args.steps // 100, 100))
    mesh.solve_host_ptr(rho_h.data_ptr(), phi_h.data_ptr())
    barrier()
    t0 = time.perf_counter()
    # each step uploads its density and downloads its potential; consecutive steps
    # overlap one download with the next upload, and the clock stops at the last copy
    for _ in range(ke):
        mesh.solve_host_ptr_async(rho_h.data_ptr(), phi_h.data_ptr())
    mesh.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e_err = float(np.max(np.abs(phi_h.numpy() - p_split)))

    rates = mpl.probe_rates()

    # ---- gravitational source terms (Sec. 3) of this solve's potential: momentum S and
    # energy E from a synthetic velocity; float64, bound by the float64 pipe
    gen = torch.Generator(device="cuda")
    gen.manual_seed(7)
    gvel = torch.randn(3 * cells, dtype=torch.float64, device="cuda", generator=gen)
    gS = torch.empty(3 * cells, dtype=torch.float64, device="cuda")
    gE = torch.empty(cells, dtype=torch.float64, device="cuda")
    kg = max(3, min(args.steps // 200, 50))
    for _ in range(2):
        mesh.gravity_sources(v=gvel, S=gS, E=gE)
    mesh.synchronize()
    e0.record(stream)
    for _ in range(kg):
        mesh.gravity_sources(v=gvel, S=gS, E=gE)
    e1.record(stream)
    torch.cuda.synchronize()
    g_us = max_over_ranks(e0.elapsed_time(e1)) / kg * 1e3
    fp64_instr_peak = rates["fp64_tflops"] * 1e12 / 2.0  # one FMA instruction = 2 flops
    gravity = {"kernel": "gravity_sources", "launches": kg, "avg_launch_us": g_us,
               "algorithmic_bytes_per_cell": 72, "hbm_gbs": 72 * cells / g_us / 1e3,
               "hbm_frac": 72 * cells / g_us / 1e3 / measured_peaks()[0],
               "fp64_instr_per_cell": 12, "fp64_instr_per_s": 12 * cells / (g_us * 1e-6),
               "fp64_frac": 12 * cells / (g_us * 1e-6) / fp64_instr_peak, "bound": "fp64",
               "note": "S [3] and E from Phi, rho, v [3]: 9 float64 reads + 4 writes per cell"}
    del gvel, gS, gE

    # ---- coarsening-block averaging (Sec. 2.1 / 2.3) on the paper's standard dimensionless
    # mesh (N_theta = 256, r_core = 0.25, R_radial = 3.68, N_phi = 2 N_theta), one field in place
    pm = W.paper_mesh(256, 0.25, 3.68, 0, 3)
    cmesh = mpl.Mesh(pm.r, pm.theta, pm.phi, 2, 1.0, precision="fp64", stream=stream)
    c_t, c_p = cmesh.coarsening_factors()
    n_pm = (pm.r.size - 1) * (pm.theta.size - 1) * (pm.phi.size - 1)
    coarse_cells = int(((c_t[:, None] > 1) | (c_p > 1)).sum()) * (pm.phi.size - 1)
    cfield = torch.randn(n_pm, dtype=torch.float64, device="cuda", generator=gen)
    kc = max(3, min(args.steps // 200, 50))
    for _ in range(2):
        cmesh.coarsen(cfield)
    cmesh.synchronize()
    e0.record(stream)
    for _ in range(kc):
        cmesh.coarsen(cfield)
    e1.record(stream)
    torch.cuda.synchronize()
    c_us = max_over_ranks(e0.elapsed_time(e1)) / kc * 1e3
    coarsen = {"kernel": "coarsen_blocks", "mesh": "paper rule N_theta = 256: 942 x 256 x 512",
               "cells": n_pm, "coarsened_cells": coarse_cells, "launches": kc, "avg_launch_us": c_us,
               "algorithmic_bytes": 16 * coarse_cells, "hbm_gbs": 16 * coarse_cells / c_us / 1e3,
               "hbm_frac": 16 * coarse_cells / c_us / 1e3 / measured_peaks()[0], "bound": "fp64",
               "note": "every coarsened cell read once and written once (in place); the float64 pipe "
                       "(about 1.6 float64 instructions a coarsened cell) bounds it before HBM"}
    cmesh.close()
    del cfield

    # ---- roofline of the dominant kernel
    log("kernels:", json.dumps(prof))
    dom = max(prof, key=lambda k: prof[k]["total_ms"])
    avg_ms = prof[dom]["total_ms"] / prof[dom]["launches"]
    nbytes = alg_bytes(dom, cells, rows, m.shape[0], m.L, KL)
    peak, peak_kind = measured_peaks()
    achieved = nbytes / (avg_ms * 1e-3) / 1e9
    traffic = None
    rec = NCU_TRAFFIC.get(dom) if args.workload == "presn" else None  # the record is for that workload
    if rec and rec[2] == source_hash(rec[1]):
        traffic = rec[0]
    kernels = {k: {"launches": v["launches"], "avg_us": 1e3 * v["total_ms"] / v["launches"],
                   "share": v["total_ms"] / sum(x["total_ms"] for x in prof.values())} for k, v in prof.items()}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": SPLIT_PRECISION, "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "cells": cells, "l_max": m.L, "moments": KL,
                       "precision": SPLIT_PRECISION, "parallelism": f"replicas x{world}",
                       "l2": f"inputs larger than L2 (rho {8 * cells / 1e6:.0f} MB + Phi {8 * cells / 1e6:.0f} MB per step)"},
            "gcell_mode_per_s": value * cells * KL / 1e9,
            "fp64_gpu": {"solves_per_s": world / (ms64 * 1e-3), "ms_per_solve": ms64, "steps": k64,
                         "gcell_mode_per_s": world / (ms64 * 1e-3) * cells * KL / 1e9},
            "speedup_split_vs_fp64_gpu": ms64 / ms_per_step,
            "accuracy": acc,
            "roofline": {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                         "algorithmic_bytes": nbytes, "avg_launch_us": avg_ms * 1e3},
            "kernels": kernels,
            "kernels_note": f"per-kernel CUDA-event durations from {kp} separately profiled solves "
                            f"(sum {prof_ms_per_step * 1e3:.1f} us/solve)",
            "e2e": {"value": world * ke / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": 8 * cells,
                    "d2h_bytes_per_step": 8 * cells, "steps": ke, "max_abs_diff_vs_device_solve": e2e_err},
            # kernels of the split chain per solve (one graph launch each) x timed solves
            "gpu_launches": len(prof) * args.steps,
            "gravity_sources": gravity,
            "coarsen_blocks": coarsen,
            "device_rates": {"fp64_tflops_measured": rates["fp64_tflops"],
                             "cvt_f64_to_f32_per_s_measured": rates["cvt_f64_f32_per_s"]},
            "clocks": clk,
        }
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    mesh.close()
    mesh64.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
