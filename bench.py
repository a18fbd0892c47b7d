#!/usr/bin/env python
"""Benchmark of the multipole Poisson solve on one GB300 (or N replicas).

Headline workload (default): the large single solve, 2048 x 512 x 1024 cells (1.07e9),
geometric shells over [1e5, 1e10] cm, l_max = 64, density rho_c/(1+(r/r_c)^2)^1.5 times
seeded harmonic perturbations (l <= 4 at 1e-2, l <= 64 at 1e-3; seed 4).  One step = one
full solve (moments, radial recurrences, potential) of that density, resident in HBM,
through the C ABI (mp_solve) on the split-precision BF16x3 tensor-core path.

The timed region repeats blocks of K solves (each block bracketed by a barrier and a
device synchronize) until about a second of device time has passed, so that the clock
sampler sees the load; ms_per_step is the median block time / K.  Also on the line: the
float64 GPU path on the same density, the accuracy of both against the FP64 CPU oracle
(Phi pointwise over every cell, the angular and edge moments per degree), per-kernel
times with the dominant kernel's HBM roofline and the tensor-pipe fraction of the two
tcgen05 contractions, an end-to-end number (mp_solve_host_async with pinned host
buffers: every step copies rho host->device and Phi device->host), SM clocks sampled
during the timed region, the oracle on the host cores (all threads: one whole solve;
one thread: a slab of shells) as the CPU baseline, and the other workloads (presupernova
512x128x256 L=16, log-normal 1024x256x512 L=32, homogeneous spheroid 64x32x64 L=8, and
the batch of 64 uneven meshes) with their own accuracy and HBM fractions.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload large|presn|lognormal|spheroid] [--lean]

With N > 1 the script runs under torch.distributed.run, one rank per GPU, each rank
solving its own replica of the workload (no data exchange); the job value is the total
solves/s over ranks timed by the slowest rank.  --impl reference times the FP64 CPU
oracle on the host cores instead (rank 0 only).  --lean times the split path alone
(no oracle, float64 path, end-to-end leg or side workloads), for profiler runs.
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
    # the headline configuration (default): the largest single-GPU configuration
    "large": "large single solve 2048x512x1024 cells (1.07e9), geometric r in [1e5,1e10] cm, l_max=64, "
             "presn profile x (1 + l<=4 harmonics at 1e-2 + l<=64 harmonics at 1e-3), seed 4",
    "presn": "presupernova core 512x128x256 cells, geometric r in [1e5,1e10] cm, l_max=16, seed 2",
    "lognormal": "log-normal angular field 1024x256x512 cells, geometric r in [1e5,1e12] cm, l_max=32, seed 3",
    "spheroid": "homogeneous oblate spheroid a1=1, a3=0.6, 64x32x64 uniform cells over r in [0,1.5], l_max=8, G=1",
}
BATCH_DESC = ("64 uneven meshes (n_r,n_theta,n_phi) from {(256,64,128),(512,128,256),(768,192,384),"
              "(1024,256,512)}, l_max from {8,16,32}, presn densities with per-mesh rho_c, r_c, seed 5")
SPLIT_PRECISION = "bf16x3"

# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the dominant
# kernel, keyed (workload, kernel): (bytes, source file, sha1 of that file and the shared
# headers at capture time).  A record stands only while the source it was taken on is
# unchanged.  The large workload's figure is a capture of the whole 2048-shell mesh with
# those two counters alone (one pass, as on a 128-shell cut first): 8.60 GB of density read
# and 0.49 GB of F written back (F, 545 MB, outgrows L2 at this size; on the cut it stays).
NCU_TRAFFIC = {
    ("large", "split_phi_project_tc"): (8.60e9 + 489.97e6, "mp_split.cu", "db667758754e9e99133af3c6f11f0db47869fecb"),
}
KERNEL_HEADERS = ("ptx.cuh", "mp_internal.h", "mp_errors.h")


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=sorted(WORKLOADS), default="large",
                   help="mesh and density of the headline (large is the benchmarked configuration)")
    p.add_argument("--min-seconds", type=float, default=1.0, help="device time the timed blocks fill")
    p.add_argument("--lean", action="store_true", help="split path timing only (profiler runs)")
    p.add_argument("--shells", type=int, default=0,
                   help="profiling captures: the workload with this many shells (same angular grid, "
                        "l_max and density recipe); 0 keeps its own")
    p.add_argument("--theta-engine", choices=["auto", "tensor", "cuda"], default="auto",
                   help="theta stages of the split path (auto: the mesh's default)")
    return p.parse_args()


def dist_info():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def measured_peaks():
    """(HBM GB/s, bf16 TFLOP/s sustained, kind): the peaks measured on these GB300s
    (MEASURED_PEAKS.json: a copy stream and a bf16 GEMM), else fallback figures."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d.get("bf16_tflops_sustained", d["bf16_tflops"])), "measured"
    except Exception:
        return 6800.0, 1700.0, "fallback"


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

    def stop(self, skip_s: float = 0.0):
        """Clock summary of the samples taken after the first skip_s seconds (the idle lead-in
        before the timed region)."""
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
        skip = min(len(sm) - 1, int(skip_s / 0.1)) if sm else 0
        load = sm[skip:]
        return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "samples_under_load": len(load),
                "power_w_max": max(power) if power else None}


# ---------------------------------------------------------------- workloads
def make_workload(name, shells=0):
    """Mesh and host density of a headline workload (seeded, synthetic); shells > 0 replaces
    its number of shells."""
    from paper_2602_02507_gb300 import workloads as W
    kw = {"n_r": shells} if shells > 0 else {}
    if name == "large":
        return W.large(materialize=True, **kw)
    return getattr(W, name)(**kw)


# ---------------------------------------------------------------- oracle leg (host cores)
def oracle_reference(w, want_phi=True):
    """One FP64 oracle solve of the whole workload on every host thread: (result with the
    oracle's tables, seconds, threads).  Its Phi and moments are the reference the GPU
    paths' accuracy is stated against."""
    from oracle import oracle as O
    m = w.mesh
    tab = O.build_tables(m.r, m.theta, m.phi, m.L)
    t0 = time.perf_counter()
    ref = O.solve(tab, w.rho, m.G, want_phi=want_phi)
    el = time.perf_counter() - t0
    ref["tables"] = tab
    return ref, el, O.get_threads()


def oracle_one_thread(w, tab, seconds_all, threads, target_s=3.0):
    """The oracle on one host thread, timed on a slab of the workload's first shells (about
    target_s seconds of work) and scaled to the whole mesh by its share of the shells:
    (solves/s, shells, seconds)."""
    from oracle import oracle as O
    m = w.mesh
    n_r = m.shape[0]
    per_shell = seconds_all * threads / n_r
    ns = int(max(1, min(n_r, round(target_s / max(per_shell, 1e-9)))))
    WR, WI, V = O.radial_integrals(m.L, m.r[:ns + 1], tab.r_ref)
    slab = O.Tables(r=m.r[:ns + 1], theta=tab.theta, phi=tab.phi, L=m.L, r_ref=tab.r_ref, Ith=tab.Ith,
                    Iph=tab.Iph, WR=WR, WI=WI, V=V)
    prev = O.get_threads()
    O.set_threads(1)
    try:
        t0 = time.perf_counter()
        O.solve(slab, w.rho[:ns], m.G)
        el = time.perf_counter() - t0
    finally:
        O.set_threads(prev)
    return (ns / n_r) / el, ns, el


def r3(xs):
    return [float(f"{x:.3g}") for x in xs]


def phi_error_vs_oracle(phi_dev, ref_phi, chunk=64):
    """max over every cell of |Phi_gpu - Phi_oracle| / |Phi_oracle| (shells in chunks)."""
    import numpy as np
    n_r = ref_phi.shape[0]
    g3 = phi_dev.view(n_r, -1)
    err = 0.0
    for i0 in range(0, n_r, chunk):
        g = g3[i0:i0 + chunk].cpu().numpy().reshape(ref_phi[i0:i0 + chunk].shape)
        r = ref_phi[i0:i0 + chunk]
        err = max(err, float(np.max(np.abs(g - r) / np.abs(r))))
    return err


def phi_diff_on_device(a, b, chunk_cells=1 << 26):
    """max |a - b| / |b| over two device potentials (chunked)."""
    out = 0.0
    fa, fb = a.view(-1), b.view(-1)
    for c0 in range(0, fa.numel(), chunk_cells):
        x, y = fa[c0:c0 + chunk_cells], fb[c0:c0 + chunk_cells]
        out = max(out, float(((x - y).abs() / y.abs()).max().item()))
    return out


def moment_report(mesh, w, ref, S, prec):
    """Per-degree errors of the exported moments against the oracle: angular moments and
    edge moments relative to the sum of the magnitudes of each moment's terms (with the
    split path's error-model bar), and angular moments relative to their degree's largest."""
    import torch
    from oracle.error_metrics import edge_term_errors, moment_term_errors, per_l_errors, split_moment_bar
    m = w.mesh
    n_r, K = m.shape[0], m.KL
    A = torch.empty(n_r * K, dtype=torch.float64, device="cuda")
    MR = torch.empty((n_r + 1) * K, dtype=torch.float64, device="cuda")
    MI = torch.empty((n_r + 1) * K, dtype=torch.float64, device="cuda")
    mesh.get_moments(A, MR, MI)
    mesh.synchronize()
    got = {"A": A.cpu().numpy().reshape(n_r, K), "MR": MR.cpu().numpy().reshape(n_r + 1, K),
           "MI": MI.cpu().numpy().reshape(n_r + 1, K)}
    eA = moment_term_errors(got["A"], ref["A"], S, m.L)
    eM = edge_term_errors(got, ref, S)
    eD = per_l_errors(got["A"], ref["A"], m.L)
    bar = split_moment_bar(m, prec) if prec != "fp64" else 1e-12
    return {"moments_bar_rel_terms": bar,
            "max_over_l": {"A_rel_terms": max(eA), "MR_rel_terms": max(eM["MR"]), "MI_rel_terms": max(eM["MI"]),
                           "A_rel_degree_max": max(eD)},
            "within_bar": bool(max(eA + eM["MR"] + eM["MI"]) <= bar),
            "per_l": {"A_rel_terms": r3(eA), "MR_rel_terms": r3(eM["MR"]), "MI_rel_terms": r3(eM["MI"]),
                      "A_rel_degree_max": r3(eD)}}


# ---------------------------------------------------------------- device timing
def timed_blocks(solve, steps, min_seconds, stream, barrier, max_over_ranks):
    """Device times (ms) of blocks of `steps` calls of solve(), each block bracketed by a
    barrier and a device synchronize and timed with CUDA events on the launching stream;
    blocks repeat until about min_seconds of device time (at least 3 blocks)."""
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def block():
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            solve()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        return e0.elapsed_time(e1)

    times = [block()]
    more = int(max_over_ranks(float(min(2000, max(2, math.ceil(min_seconds * 1e3 / max(times[0], 1e-3)) - 1)))))
    times += [block() for _ in range(more)]
    return times


# ---------------------------------------------------------------- roofline bookkeeping
def alg_bytes(kernel: str, cells: int, rows: int, n_r: int, L: int, KL: int):
    """Algorithmic DRAM bytes per launch: the step's inputs read once and outputs written
    once.  The two streaming steps count the density read (8 B/cell) and the potential
    write (8 B/cell); the intermediates of the other kernels are listed for reference."""
    P = 2 * L + 1
    table = {
        "split_phi_project_tc": 8 * cells,                       # rho in (step (a) reads S once)
        "split_synth_tc": 8 * cells,                             # Phi out (step (d) writes Phi once)
        "split_theta_contract": 4 * rows * P + 8 * n_r * KL,     # F in, moments out
        "split_theta_contract_tc": 4 * rows * (P - 1) + 8 * n_r * (KL - L - 1),  # F rows p >= 1 in
        "split_theta_contract_m0": 4 * rows + 8 * n_r * (L + 1),  # F row p = 0 in, m = 0 moments out
        # A in, edge moments out, coefficients out (float32, or two bf16 terms)
        "radial_scan": 8 * n_r * KL + 16 * (n_r + 1) * KL + 4 * n_r * KL,
        "split_theta_synth": rows * (4 * ((2 * L + 15) // 16 * 16) + 8),
        "split_theta_synth_tc": rows * 4 * ((2 * L + 15) // 16 * 16),  # A operand of the synthesis out
        "split_theta_synth_m0": rows * 8,                           # m = 0 column out (float pairs)
        "fp64_phi_project": 8 * cells + 8 * rows * P,
        "fp64_theta_contract": 8 * rows * P + 8 * n_r * KL,
        "fp64_theta_synth": 8 * rows * P,
        "fp64_phi_synth": 8 * cells + 8 * rows * P,
    }
    return table.get(kernel)


def mma_flops(kernel: str, shape, L: int, nprod: int):
    """(useful, executed) tensor-core flops per launch of the two tcgen05 contractions:
    useful = bf16 products x 2 x cells x columns; executed uses the padded GEMM dimensions
    (projection N = 2L+1 rounded up to 16, K = n_phi rounded up to 32; synthesis K = 2L
    rounded up to 16, N = n_phi rounded up to 16)."""
    n_r, n_t, n_p = shape
    rows = n_r * n_t
    rows_pad = -(-rows // 128) * 128
    if kernel == "split_phi_project_tc":
        useful = nprod * 2 * rows * n_p * (2 * L + 1)
        executed = nprod * 2 * rows_pad * (-(-n_p // 32) * 32) * (-(-(2 * L + 1) // 16) * 16)
    elif kernel == "split_synth_tc":
        useful = nprod * 2 * rows * n_p * (2 * L)
        executed = nprod * 2 * rows_pad * (-(-n_p // 16) * 16) * max(16, -(-(2 * L) // 16) * 16)
    else:
        return None
    return useful, executed


# ---------------------------------------------------------------- reference arm
def run_reference(args):
    """The FP64 CPU oracle on the host cores, on the headline workload: each step solves a
    bounded sample of it (the whole mesh when one solve takes under half a second, else a
    slab of its first shells sized to about half a second), scaled to whole solves by the
    sample's share of the shells."""
    world, rank, _ = dist_info()
    if rank != 0:
        return 0
    import numpy as np
    from oracle import build as oracle_build
    from oracle import oracle as O
    oracle_build.build()
    w = make_workload(args.workload)
    m = w.mesh
    n_r = m.shape[0]
    tab = O.build_tables(m.r, m.theta, m.phi, m.L)
    # size the sample: time one shell-slab solve, grow it to about half a second
    ns = max(1, n_r // 256)
    while True:
        WR, WI, V = O.radial_integrals(m.L, m.r[:ns + 1], tab.r_ref)
        slab = O.Tables(r=m.r[:ns + 1], theta=tab.theta, phi=tab.phi, L=m.L, r_ref=tab.r_ref, Ith=tab.Ith,
                        Iph=tab.Iph, WR=WR, WI=WI, V=V)
        rho = np.ascontiguousarray(w.rho[:ns])
        t0 = time.perf_counter()
        O.solve(slab, rho, m.G)
        el = time.perf_counter() - t0
        if el >= 0.25 or ns == n_r:
            break
        ns = min(n_r, max(ns + 1, int(ns * 0.5 / max(el, 1e-3))))
    warm = min(args.warmup, 2)
    for _ in range(warm):
        O.solve(slab, rho, m.G)
    steps = max(1, args.steps)
    t0 = time.perf_counter()
    for _ in range(steps):
        O.solve(slab, rho, m.G)
    el = time.perf_counter() - t0
    value = steps * (ns / n_r) / el
    sample = (f"FP64 oracle (tables prebuilt), each step the first {ns} of {n_r} shells "
              f"({ns / n_r:.4g} of the workload), {steps} steps in {el:.2f} s, scaled by shells")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": steps, "warmup": warm, "ms_per_step": 1e3 * el / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "precision": "fp64 (CPU oracle)", "cells": m.cells,
                   "l_max": m.L},
        "gcell_mode_per_s": value * m.cells * m.KL / 1e9,
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": O.get_threads(), "kind": "oracle",
                         "sample": sample, "nproc": os.cpu_count()},
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


# ---------------------------------------------------------------- side workloads
def side_workload(name, args, stream, with_oracle, hbm_peak):
    """One of the other configurations: split and float64 GPU solves timed (blocks filling
    about 0.3 s), their accuracy against the oracle, the whole-step HBM fraction."""
    import numpy as np
    import torch
    from paper_2602_02507_gb300 import multipole as mpl
    w = make_workload(name)
    m = w.mesh
    rho = torch.from_numpy(np.ascontiguousarray(w.rho)).cuda()
    out = {"workload": WORKLOADS[name], "cells": m.cells, "l_max": m.L}
    nothing = lambda: None  # noqa: E731
    ident = lambda x: x  # noqa: E731
    for prec in (SPLIT_PRECISION, "fp64"):
        phi = torch.empty_like(rho)
        with mpl.Mesh(m.r, m.theta, m.phi, m.L, m.G, precision=prec, stream=stream) as mesh:
            mesh.set_density(rho)
            mesh.set_phi_output(phi)
            for _ in range(3):
                mesh.solve()
            mesh.synchronize()
            steps = max(args.steps, 20) if prec != "fp64" else 5
            times = timed_blocks(mesh.solve, steps, 0.3 if prec != "fp64" else 0.2, stream, nothing, ident)
            mesh.synchronize()
            ms = statistics.median(times) / steps
            key = "split" if prec != "fp64" else "fp64_gpu"
            out[key] = {"solves_per_s": 1e3 / ms, "ms_per_solve": ms,
                        "hbm_frac_16B_per_cell": 16 * m.cells / (ms * 1e-3) / 1e9 / hbm_peak,
                        "effective_precision": mesh.info()["effective_precision"]}
            if with_oracle:
                if "ref" not in out:
                    ref, el, thr = oracle_reference(w)
                    from oracle.error_metrics import term_scales
                    out["_ref"], out["_S"] = ref, term_scales(w.rho, ref["tables"], m.G)
                    out["oracle_solves_per_s"] = {"value": 1.0 / el, "threads": thr}
                    out["ref"] = True
                out[key]["phi_max_rel_err_vs_oracle"] = phi_error_vs_oracle(phi, out["_ref"]["phi"])
                rep = moment_report(mesh, w, out["_ref"], out["_S"], prec)
                rep.pop("per_l")
                out[key].update(rep)
        del phi
    out.pop("ref", None)
    out.pop("_ref", None)
    out.pop("_S", None)
    out["speedup_split_vs_fp64_gpu"] = out["fp64_gpu"]["ms_per_solve"] / out["split"]["ms_per_solve"]
    del rho, w
    torch.cuda.empty_cache()
    return out


def batch_workload(args, stream, with_oracle, hbm_peak):
    """The 64 uneven meshes: one graph-launched batch (split path) against a loop of
    per-mesh float64 solves; densities built on the device from their separable factors;
    the smallest mesh of each l_max and the three smallest overall against the oracle."""
    import numpy as np
    import torch
    from paper_2602_02507_gb300 import multipole as mpl
    from paper_2602_02507_gb300 import workloads as W
    draws = W.batch_draws()
    meshes, meshes64, rhos, phis, phis64, cells = [], [], [], [], [], 0
    for n in range(len(draws)):
        w = W.batch_instance(n, draws, materialize=False)
        m = w.mesh
        prof = torch.from_numpy(w.extra["profile"]).cuda()
        ang = torch.from_numpy(w.extra["angular"]).cuda()
        rho = (prof[:, None, None] * ang[None, :, :]).contiguous()
        phi, phi64 = torch.empty_like(rho), torch.empty_like(rho)
        ms = mpl.Mesh(m.r, m.theta, m.phi, m.L, m.G, precision=SPLIT_PRECISION, stream=stream)
        ms.set_density(rho)
        ms.set_phi_output(phi)
        m64 = mpl.Mesh(m.r, m.theta, m.phi, m.L, m.G, precision="fp64", stream=stream)
        m64.set_density(rho)
        m64.set_phi_output(phi64)
        meshes.append(ms)
        meshes64.append(m64)
        rhos.append(rho)
        phis.append(phi)
        phis64.append(phi64)
        cells += m.cells
    batch = mpl.Batch(meshes)
    for _ in range(3):
        batch.solve()
    torch.cuda.synchronize()
    nothing = lambda: None  # noqa: E731
    ident = lambda x: x  # noqa: E731
    times = timed_blocks(batch.solve, max(5, args.steps // 4), 0.5, stream, nothing, ident)
    ms = statistics.median(times) / max(5, args.steps // 4)

    def loop64():
        for mm in meshes64:
            mm.solve()

    loop64()
    torch.cuda.synchronize()
    t64 = statistics.median(timed_blocks(loop64, 1, 0.2, stream, nothing, ident))
    out = {"workload": BATCH_DESC, "instances": len(draws), "cells": cells,
           "split": {"batches_per_s": 1e3 / ms, "ms_per_batch": ms,
                     "hbm_frac_16B_per_cell": 16 * cells / (ms * 1e-3) / 1e9 / hbm_peak,
                     "launch": "one CUDA graph launch per batch"},
           "fp64_gpu": {"ms_per_batch": t64, "launch": "per-mesh float64 solves in a loop"},
           "speedup_split_vs_fp64_gpu": t64 / ms}
    if with_oracle:
        order = sorted(range(len(draws)), key=lambda n: np.prod(draws[n][0]) * draws[n][1])
        picks = list(order[:3])
        for L in sorted({d[1] for d in draws}):
            n = min((k for k in range(len(draws)) if draws[k][1] == L), key=lambda k: np.prod(draws[k][0]))
            if n not in picks:
                picks.append(n)
        worst = 0.0
        for n in picks:
            w = W.batch_instance(n, draws)
            ref, _, _ = oracle_reference(w)
            worst = max(worst, phi_error_vs_oracle(phis[n], ref["phi"]))
        out["split"]["phi_max_rel_err_vs_oracle"] = worst
        out["split"]["oracle_checked_instances"] = [f"{draws[n][0]} L={draws[n][1]}" for n in picks]
    out["split"]["phi_max_rel_err_vs_fp64_gpu"] = max(phi_diff_on_device(a, b) for a, b in zip(phis, phis64))
    batch.close()
    for mm in meshes + meshes64:
        mm.close()
    del rhos, phis, phis64
    torch.cuda.empty_cache()
    return out


def beside_solve(stream, hbm_peak, rates, steps):
    """Gravitational source terms (Sec. 3) of a presupernova solve's potential and the
    coarsening-block averaging on the paper's N_theta = 256 mesh: float64 kernels bound by
    the float64 pipe, timed beside (not inside) the solve."""
    import torch
    from paper_2602_02507_gb300 import multipole as mpl
    from paper_2602_02507_gb300 import workloads as W
    w = W.presn()
    m = w.mesh
    cells = m.cells
    rho = torch.from_numpy(w.rho).cuda()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    mesh = mpl.Mesh(m.r, m.theta, m.phi, m.L, m.G, precision=SPLIT_PRECISION, stream=stream)
    mesh.set_density(rho)
    mesh.solve()
    gen = torch.Generator(device="cuda")
    gen.manual_seed(7)
    gvel = torch.randn(3 * cells, dtype=torch.float64, device="cuda", generator=gen)
    gS = torch.empty(3 * cells, dtype=torch.float64, device="cuda")
    gE = torch.empty(cells, dtype=torch.float64, device="cuda")
    kg = max(10, steps)
    for _ in range(2):
        mesh.gravity_sources(v=gvel, S=gS, E=gE)
    mesh.synchronize()
    e0.record(stream)
    for _ in range(kg):
        mesh.gravity_sources(v=gvel, S=gS, E=gE)
    e1.record(stream)
    torch.cuda.synchronize()
    g_us = e0.elapsed_time(e1) / kg * 1e3
    fp64_instr_peak = rates["fp64_tflops"] * 1e12 / 2.0  # one FMA instruction = 2 flops
    gravity = {"kernel": "gravity_sources", "workload": WORKLOADS["presn"], "launches": kg, "avg_launch_us": g_us,
               "algorithmic_bytes_per_cell": 72, "hbm_gbs": 72 * cells / g_us / 1e3,
               "hbm_frac": 72 * cells / g_us / 1e3 / hbm_peak,
               "fp64_instr_per_cell": 12, "fp64_instr_per_s": 12 * cells / (g_us * 1e-6),
               "fp64_frac": 12 * cells / (g_us * 1e-6) / fp64_instr_peak, "bound": "fp64",
               "note": "S [3] and E from Phi, rho, v [3]: 9 float64 reads + 4 writes per cell"}
    mesh.close()
    del gvel, gS, gE, rho
    pm = W.paper_mesh(256, 0.25, 3.68, 0, 3)
    cmesh = mpl.Mesh(pm.r, pm.theta, pm.phi, 2, 1.0, precision="fp64", stream=stream)
    c_t, c_p = cmesh.coarsening_factors()
    n_pm = (pm.r.size - 1) * (pm.theta.size - 1) * (pm.phi.size - 1)
    coarse_cells = int(((c_t[:, None] > 1) | (c_p > 1)).sum()) * (pm.phi.size - 1)
    cfield = torch.randn(n_pm, dtype=torch.float64, device="cuda", generator=gen)
    kc = max(10, steps)
    for _ in range(2):
        cmesh.coarsen(cfield)
    cmesh.synchronize()
    e0.record(stream)
    for _ in range(kc):
        cmesh.coarsen(cfield)
    e1.record(stream)
    torch.cuda.synchronize()
    c_us = e0.elapsed_time(e1) / kc * 1e3
    coarsen = {"kernel": "coarsen_blocks", "mesh": "paper rule N_theta = 256: 942 x 256 x 512",
               "cells": n_pm, "coarsened_cells": coarse_cells, "launches": kc, "avg_launch_us": c_us,
               "algorithmic_bytes": 16 * coarse_cells, "hbm_gbs": 16 * coarse_cells / c_us / 1e3,
               "hbm_frac": 16 * coarse_cells / c_us / 1e3 / hbm_peak, "bound": "fp64",
               "note": "every coarsened cell read once and written once (in place); the float64 pipe "
                       "(about 1.6 float64 instructions a coarsened cell) bounds it before HBM"}
    cmesh.close()
    del cfield
    torch.cuda.empty_cache()
    return gravity, coarsen


# ---------------------------------------------------------------- our arm
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

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(x: float) -> float:
        return max_over_ranks_on(x, world, "cuda")

    hbm_peak, tc_peak, peak_kind = measured_peaks()
    full = not args.lean
    with_oracle = full and rank == 0 and world == 1
    w = make_workload(args.workload, args.shells)
    m = w.mesh
    cells, KL = m.cells, m.KL
    rows = m.shape[0] * m.shape[1]
    stream = torch.cuda.current_stream()
    rho = torch.from_numpy(w.rho).cuda()
    phi = torch.empty_like(rho)
    # the end-to-end leg's pinned host buffers, allocated up front as an application would,
    # before the oracle leg's large host arrays come and go
    rho_h = phi_h = None
    if full:
        rho_h = torch.empty(rho.shape, dtype=torch.float64, pin_memory=True)
        rho_h.copy_(torch.from_numpy(w.rho))
        phi_h = torch.empty(rho.shape, dtype=torch.float64, pin_memory=True)
    mesh = mpl.Mesh(m.r, m.theta, m.phi, m.L, m.G, precision=SPLIT_PRECISION, stream=stream)
    mesh.set_theta_engine(args.theta_engine)
    mesh.set_density(rho)
    mesh.set_phi_output(phi)
    mesh.solve()
    mesh.synchronize()

    # ---- accuracy of both GPU paths against the FP64 CPU oracle (rank 0), which also gives
    # the CPU baseline (one whole solve on every host thread; one thread on a slab of shells)
    acc = {"tolerance_phi": 1e-6, "phi_metric": "max over every cell of |dPhi| / |Phi_oracle|"}
    cpu = None
    ref = S = None
    if with_oracle:
        from oracle.error_metrics import term_scales
        log("oracle solve of the whole workload ...")
        ref, t_all, threads = oracle_reference(w)
        v1, ns, el1 = oracle_one_thread(w, ref["tables"], t_all, threads)
        cpu = {"value": 1.0 / t_all, "unit": "solves/s", "cores": threads, "nproc": os.cpu_count(), "kind": "oracle",
               "sample": f"one whole-workload solve (FP64 oracle, tables prebuilt) on {threads} threads in {t_all:.1f} s",
               "one_thread": {"value": v1, "unit": "solves/s",
                              "sample": f"the first {ns} shells on 1 thread in {el1:.2f} s, scaled by shells"}}
        S = term_scales(w.rho, ref["tables"], m.G)
        acc["split"] = {"phi_max_rel_err_vs_oracle": phi_error_vs_oracle(phi, ref["phi"]),
                        **moment_report(mesh, w, ref, S, SPLIT_PRECISION)}
    mesh64 = phi64 = None
    if full:
        phi64 = torch.empty_like(rho)
        mesh64 = mpl.Mesh(m.r, m.theta, m.phi, m.L, m.G, precision="fp64", stream=stream)
        mesh64.set_density(rho)
        mesh64.set_phi_output(phi64)
        mesh64.solve()
        mesh64.synchronize()
        if with_oracle:
            acc["fp64_gpu"] = {"phi_max_rel_err_vs_oracle": phi_error_vs_oracle(phi64, ref["phi"]),
                               **moment_report(mesh64, w, ref, S, "fp64")}
        acc["phi_max_rel_err_split_vs_fp64_gpu"] = phi_diff_on_device(phi, phi64)
    ref = S = None

    # ---- timed region: split path, blocks of K solves (each solve one CUDA graph launch)
    for _ in range(args.warmup):
        mesh.solve()
    mesh.synchronize()
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    t_region = time.perf_counter()
    times = timed_blocks(mesh.solve, args.steps, args.min_seconds, stream, barrier, max_over_ranks)
    t_region = time.perf_counter() - t_region
    clk = clocks.stop(skip_s=0.3)
    mesh.synchronize()
    local_ms = statistics.median(times)
    total_ms = max_over_ranks(local_ms)
    ms_per_step = total_ms / args.steps
    value = whole_job_rate(world, args.steps, total_ms)

    # ---- per-kernel durations: the same solves launched kernel by kernel with CUDA events
    # between them on the mesh stream (events cost a little time of their own)
    kp = max(3, min(args.steps * 5, 200))
    mesh.profile(True)
    for _ in range(kp):
        mesh.solve()
    prof = mesh.profile_read()
    mesh.profile(False)
    prof_ms_per_step = sum(v["total_ms"] for v in prof.values()) / kp

    line_extra = {}
    if full:
        # ---- float64 GPU path on the same density, at least 20 solves
        k64 = 20
        for _ in range(2):
            mesh64.solve()
        mesh64.synchronize()
        t64 = timed_blocks(mesh64.solve, k64, 0.0, stream, barrier, max_over_ranks)
        ms64 = max_over_ranks(statistics.median(t64)) / k64
        mesh64.synchronize()
        mesh64.close()
        del phi64
        torch.cuda.empty_cache()
        line_extra["fp64_gpu"] = {"solves_per_s": world / (ms64 * 1e-3), "ms_per_solve": ms64, "steps": k64,
                                  "blocks": len(t64), "gcell_mode_per_s": world / (ms64 * 1e-3) * cells * KL / 1e9}
        line_extra["speedup_split_vs_fp64_gpu"] = ms64 / ms_per_step

        # ---- end to end through the C ABI with pinned host buffers: every step uploads its
        # density and downloads its potential; consecutive steps overlap one download with the
        # next upload, and the clock stops at the last copy
        w.rho = None
        mesh.solve_host_ptr(rho_h.data_ptr(), phi_h.data_ptr())
        # the floor of a step: one upload and one download of the same sizes, concurrent
        up_s, down_s = torch.cuda.Stream(), torch.cuda.Stream()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(up_s):
            rho.copy_(rho_h.view_as(rho), non_blocking=True)
        with torch.cuda.stream(down_s):
            phi_h.view_as(phi).copy_(phi, non_blocking=True)
        torch.cuda.synchronize()
        copy_pair_ms = 1e3 * (time.perf_counter() - t0)
        t0 = time.perf_counter()
        mesh.solve_host_ptr(rho_h.data_ptr(), phi_h.data_ptr())
        one = time.perf_counter() - t0
        ke = max(20, min(5000, int(math.ceil(1.0 / max(one, 1e-6)))))
        barrier()
        t0 = time.perf_counter()
        for _ in range(ke):
            mesh.solve_host_ptr_async(rho_h.data_ptr(), phi_h.data_ptr())
        mesh.synchronize()
        e2e_s = max_over_ranks(time.perf_counter() - t0)
        e2e_err = float((phi_h.view(-1)[:1 << 24].cuda() - phi.view(-1)[:1 << 24]).abs().max().item())
        line_extra["e2e"] = {"value": world * ke / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": 8 * cells,
                             "d2h_bytes_per_step": 8 * cells, "steps": ke,
                             "max_abs_diff_vs_device_solve_first_16M_cells": e2e_err,
                             "copy_pair_ms": copy_pair_ms,
                             "api": "mp_solve_host_async, pinned host buffers, host clock"}
        del rho_h, phi_h
    theta_tc = bool(mesh.info()["theta_tensor_cores"])
    mesh.close()
    del rho, phi
    w = None
    torch.cuda.empty_cache()

    rates = mpl.probe_rates()
    if full:
        line_extra["other_workloads"] = {}
        for name in [n for n in ("presn", "lognormal", "spheroid") if n != args.workload]:
            log(f"side workload {name} ...")
            line_extra["other_workloads"][name] = side_workload(name, args, stream, with_oracle, hbm_peak)
        log("batch workload ...")
        line_extra["other_workloads"]["batch"] = batch_workload(args, stream, with_oracle, hbm_peak)
        gravity, coarsen = beside_solve(stream, hbm_peak, rates, args.steps)
        line_extra["gravity_sources"] = gravity
        line_extra["coarsen_blocks"] = coarsen

    # ---- roofline of the dominant kernel, whole-step roofline, tensor-pipe fractions
    log("kernels:", json.dumps(prof))
    # (the largest share among the kernels with stated algorithmic bytes: under a profiler
    # the captured launches are serialised and can take the lead)
    dom = max((k for k in prof if alg_bytes(k, cells, rows, m.shape[0], m.L, KL) is not None),
              key=lambda k: prof[k]["total_ms"])
    avg_ms = prof[dom]["total_ms"] / prof[dom]["launches"]
    nbytes = alg_bytes(dom, cells, rows, m.shape[0], m.L, KL)
    achieved = nbytes / (avg_ms * 1e-3) / 1e9
    traffic = None
    rec = NCU_TRAFFIC.get((args.workload, dom)) if not args.shells else None
    if rec and rec[2] == source_hash(rec[1]):
        traffic = rec[0]
    kernels = {k: {"launches": v["launches"], "avg_us": 1e3 * v["total_ms"] / v["launches"],
                   "share": v["total_ms"] / sum(x["total_ms"] for x in prof.values())} for k, v in prof.items()}
    tensor = {}
    for k in ("split_phi_project_tc", "split_synth_tc"):
        if k in prof:
            useful, executed = mma_flops(k, m.shape, m.L, 3)
            t = prof[k]["total_ms"] / prof[k]["launches"] * 1e-3
            tensor[k] = {"executed_tflops": executed / t / 1e12, "useful_tflops": useful / t / 1e12,
                         "peak_tflops": tc_peak, "frac": executed / t / 1e12 / tc_peak,
                         "hbm_gbs": 8 * cells / t / 1e9, "hbm_frac": 8 * cells / t / 1e9 / hbm_peak}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": SPLIT_PRECISION, "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload] + (f" (profiling cut: {args.shells} shells)"
                                                               if args.shells else ""),
                       "cells": cells, "l_max": m.L, "moments": KL,
                       "precision": SPLIT_PRECISION, "parallelism": f"replicas x{world}",
                       "theta_stages": "tensor cores (tcgen05), m >= 1" if theta_tc else "CUDA cores",
                       "l2": f"inputs larger than L2 (rho {8 * cells / 1e6:.0f} MB + Phi {8 * cells / 1e6:.0f} MB per step)",
                       "timing": f"{len(times)} blocks of {args.steps} solves ({t_region:.2f} s), median block / steps"},
            "gcell_mode_per_s": value * cells * KL / 1e9,
            "accuracy": acc,
            "roofline": {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "traffic": traffic, "peak_kind": peak_kind,
                         "algorithmic_bytes": nbytes, "avg_launch_us": avg_ms * 1e3},
            "roofline_step": {"algorithmic_bytes": 16 * cells, "achieved_gbs": 16 * cells / (ms_per_step * 1e-3) / 1e9,
                              "frac": 16 * cells / (ms_per_step * 1e-3) / 1e9 / hbm_peak,
                              "note": "rho read once + Phi written once per solve (16 B/cell), whole solve"},
            "tensor_pipe": tensor,
            "kernels": kernels,
            "kernels_note": f"per-kernel CUDA-event durations from {kp} separately profiled solves "
                            f"(sum {prof_ms_per_step * 1e3:.1f} us/solve)",
            "gpu_launches": len(prof) * args.steps * len(times),
            "device_rates": {"fp64_tflops_measured": rates["fp64_tflops"],
                             "cvt_f64_to_f32_per_s_measured": rates["cvt_f64_f32_per_s"]},
            "clocks": clk,
        }
        line.update(line_extra)
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
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
