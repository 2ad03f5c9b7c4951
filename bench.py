#!/usr/bin/env python3
"""Throughput of one ADER-HWENO time step on a B300: triangle-updates per second.

Workload (default): 2D Euler isentropic vortex (strength 5, background
(1, 1, 1, 1), gamma 1.4) on the periodic square [0, 10]^2, meshed by a
periodic Delaunay triangulation of a seeded Poisson-disk point set (about
1.0M points, 2.0M triangles).  Synthetic inputs, built on the host.

A step is one full pass of the scheme over every triangle and edge:
reconstruction + Lax-Wendroff (k_recon), then flux, cell-average and
Green-Gauss update and the next CFL step (k_edge).  The headline line is the
FP32 form; the FP64 form is measured on the same mesh and reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank runs an independent replica on its own GPU
(the method does not shard across GPUs here); value = all ranks' triangle
updates / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2607_10809_b300 import inputs as I  # noqa: E402

METRIC = "triangle-updates/s (Euler, 2M tris)"
UNIT = "tri-updates/s"

# Algorithmic bytes per cell and step of each kernel, per precision word s
# (4 or 8 bytes), for the Euler system (m = 4):
#   k_recon reads the cell state 3m words, the reconstruction geometry 76 words
#   and 3 neighbour indices; writes the edge-point buffer 6 * 3 * m words.
#   k_edge reads the edge-point buffer 6 * 3 * m words, the cell averages m
#   words, 10 geometry words and 4 index words; writes the state 3m words; in
#   FP32 it also reads and writes the m compensation words of the averages.
# Neighbour data are counted once (perfect reuse through the caches).
#   k_fused (one kernel for the whole step) reads the cell state 3m words, the
#   reconstruction and flux geometry 76 + 10 words, 4 index words and one slot
#   word; writes the state 3m words; in FP32 it also reads and writes the m
#   compensation words.  The edge-point records stay in shared memory.
def alg_bytes(kernel: str, s: int, m: int = 4) -> int:
    comp = 2 * m * 4 if s == 4 else 0
    if kernel == "recon":
        return (3 * m + 76 + 18 * m) * s + 3 * 4
    if kernel == "fused":
        return (3 * m + 76 + 10 + 3 * m) * s + 4 * 4 + 4 + comp
    return (18 * m + m + 10 + 3 * m) * s + 4 * 4 + comp


# DRAM traffic per cell (bytes) measured with ncu (dram__bytes_read.sum +
# dram__bytes_write.sum per launch / cells) and the hash of the kernel sources
# it was measured on; it is reported only while the sources are unchanged.
TRAFFIC = {
    "sources_sha": "2378e78abc0a979f",
    # full-size (1,999,928-cell) single-pass ncu capture, per cell; FP64 with
    # the edge-once flux phase (its two kernels)
    "per_cell": {"recon_fp32": 632.9, "edge_fp32": 467.1,
                 "recon_fp64": 1275.7, "edge_flux_fp64": 954.1, "edge_update_fp64": 471.9},
}

# Floating-point operations per cell and launch (FMA counted as 2), from the
# executed-instruction counters of one ncu capture of the 499,942-cell vortex in
# FP64 (smsp__sass_thread_inst_executed_op_d{fma,add,mul}_pred_on.sum / cells),
# valid for the sources hash of TRAFFIC.
FLOPS = {"recon_fp64": 4376, "edge_fp64": 1227 + 256}   # edge: k_edge_flux + k_edge_update

# FP64 peak of the B300 per SM clock: the nominal 1.25 TFLOP/s at the 2032 MHz
# maximum clock is 2 FP64 FMA per SM per clock on 148 SMs (a one-off FMA probe
# measured 1.132 TFLOP/s at 1935 MHz, the same rate per clock).
FP64_FLOP_PER_CLOCK = 148 * 2 * 2


def kernel_sources_sha() -> str:
    """Hash of the step kernels' code (comments and blank space ignored)."""
    import re
    h = hashlib.sha256()
    for f in ("kernels.cu", "kernels.h", "device.cuh", "tma.cuh", "internal.h"):
        with open(os.path.join(ROOT, "paper_2607_10809_b300", "csrc", f)) as fh:
            src = fh.read()
        src = re.sub(r"//[^\n]*", "", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.dev), "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        time.sleep(0.25)
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if "Active" in r[5 + k] and "Not" not in r[5 + k]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- workload
def workload(name: str):
    if name == "vortex2m":
        mesh = I.config3_mesh(1_000_000, seed=3)
    elif name == "vortex500k":
        mesh = I.config3_mesh(250_000, seed=3)
    else:
        raise SystemExit(f"unknown workload {name}")
    U0 = I.initial_state(mesh, I.vortex, 4)
    return mesh, U0


def sample_patch(geo, n):
    """About n cells nearest to the vortex centre: a contiguous patch."""
    d = (geo["cx"] - 5.0) ** 2 + (geo["cy"] - 5.0) ** 2
    return np.argsort(d, kind="stable")[:n]


# ---------------------------------------------------------------- CPU oracle
# The oracle is timed on patches: a patch of n cells around a centre, with the
# two rings of neighbours its step reads, cut out as a mesh of its own; one
# oracle step of the patch cells costs the same per cell as on the whole mesh.
def oracle_patch(mesh, U0, centre, n, nbr=None, bary=None):
    """(local mesh, its state, local indices of the n patch cells); nbr and
    bary (neighbours, barycentres) may be passed in when cutting many patches."""
    from paper_2607_10809_b300 import partition as PT
    P = mesh.unwrapped().mean(axis=1) if bary is None else bary
    d = (P[:, 0] - centre[0]) ** 2 + (P[:, 1] - centre[1]) ** 2
    near = np.argpartition(d, n)[:n] if n < d.size else np.arange(d.size)
    patch = np.sort(near)
    nbr = PT.neighbours(mesh) if nbr is None else nbr
    ring1 = np.unique(nbr[patch].ravel()); ring1 = ring1[ring1 >= 0]
    ring2 = np.unique(nbr[ring1].ravel()); ring2 = ring2[ring2 >= 0]
    cells = np.union1d(patch, np.union1d(ring1, ring2))
    used = np.unique(mesh.tri[cells])
    remap = -np.ones(mesh.nv, dtype=np.int64); remap[used] = np.arange(used.size)
    local = I.Mesh(xy=mesh.xy[used].copy(), tri=remap[mesh.tri[cells]].astype(np.int32), Lx=mesh.Lx, Ly=mesh.Ly,
                   bc=1)
    return local, np.ascontiguousarray(U0[:, :, cells]), np.searchsorted(cells, patch)


def time_patch_steps(local, Ul, idx, seconds=None, steps=None, warmup=0):
    """Oracle patch steps (single thread): for `seconds`, or exactly `steps`
    after `warmup`.  Returns (steps, wall seconds)."""
    import oracle
    o = oracle.Oracle(local, "euler")
    dt = 0.5 * o.cfl_dt(Ul)
    for _ in range(warmup):
        o.step_cells(Ul, dt, idx)
    k, t0 = 0, time.perf_counter()
    while (steps is not None and k < steps) or (steps is None and time.perf_counter() - t0 < seconds):
        o.step_cells(Ul, dt, idx)
        k += 1
    return k, time.perf_counter() - t0


def _patch_worker(args):
    local, Ul, idx, seconds = args
    k, el = time_patch_steps(local, Ul, idx, seconds=seconds, warmup=1)
    return k * idx.size / el


def cpu_oracle_rates(mesh, U0, seconds, n=2000, max_workers=64):
    """The FP64 oracle as it stands on the host cores: one core, and every core
    (one single-threaded process per core, each on its own patch; the rates
    add).  Returns a dict for the bench line."""
    import multiprocessing as mpr
    from paper_2607_10809_b300 import partition as PT
    nbr, bary = PT.neighbours(mesh), mesh.unwrapped().mean(axis=1)
    single = _patch_worker((*oracle_patch(mesh, U0, (5.0, 5.0), n, nbr, bary), seconds))
    workers = max(1, min(os.cpu_count() or 1, max_workers))
    rng = np.random.default_rng(0)
    centres = [tuple(c) for c in rng.uniform(1.0, 9.0, size=(workers, 2))]
    jobs = [(*oracle_patch(mesh, U0, c, n, nbr, bary), seconds) for c in centres]
    with mpr.get_context("spawn").Pool(workers) as pool:
        rates = pool.map(_patch_worker, jobs)
    return {"single_core": single, "all_cores": float(sum(rates)), "workers": workers,
            "nproc": os.cpu_count(), "patch_cells": n, "seconds_per_worker": seconds}


# ---------------------------------------------------------------- our arm
# ---------------------------------------------------------------- replicas (N > 1)
# One independent replica per rank; the only collectives are the barriers
# around the timed region and the max over ranks of its duration.
def dist_barrier(world):
    if world > 1:
        import torch.distributed as tdist
        tdist.barrier()


def max_over_ranks_of(x, world, device):
    """max over ranks of a float (NCCL: device "cuda"; gloo: "cpu")."""
    if world == 1:
        return x
    import torch
    import torch.distributed as tdist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def replicas_value(cells, steps, ms_max, world):
    """Whole-job throughput: all ranks' triangle updates over the slowest
    rank's time (weak scaling)."""
    return world * cells * steps / (ms_max * 1e-3)


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2607_10809_b300 import build as B
    from paper_2607_10809_b300 import hweno

    torch.cuda.set_device(local_rank)
    B.build()
    hweno.load()
    if args.only in ("adjoint", "batched", "partition"):   # one leg alone (profiling runs)
        leg = {"adjoint": adjoint_leg, "batched": lambda a: batched_leg(a, world),
               "partition": partition_leg}[args.only](args)
        if rank == 0:
            print(json.dumps({"partial_run": True, args.only: leg}), flush=True)
        return
    mesh, U0 = workload(args.workload)
    N = mesh.nt
    hmesh = hweno.Mesh(mesh)

    def barrier():
        dist_barrier(world)

    def max_over_ranks(x):
        return max_over_ranks_of(x, world, "cuda")

    results = {}
    precs = ("fp32", "fp64") if args.only == "both" else (args.only,)
    for prec in precs:
        K = args.steps if prec == "fp32" else max(20, args.steps // args.fp64_divisor)
        s = hweno.Solver(hmesh, U0, eq="euler", precision=prec, time_rule=args.time_rule,
                         step_kernels=args.step_kernels)
        stream = s.stream
        for _ in range(args.warmup):
            s.step()
        torch.cuda.synchronize(); barrier(); torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        s.profile(True)
        with ClockSampler(local_rank) as clk:
            e0.record(stream)
            for _ in range(K):
                s.step()
            e1.record(stream)
            torch.cuda.synchronize()
        barrier(); torch.cuda.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1))
        prof = s.profile_read()
        s.profile(False)
        flags = s.status_flags()
        results[prec] = {"K": K, "ms": ms, "prof": prof, "clocks": clk.summary(), "flags": flags,
                         "kernels": s.step_kernels()}
        if args.only == "both":
            # accuracy of the FP32 form against the FP64 form: the same fixed
            # steps from the initial state (outside the timed region)
            s.set_state(U0, 0.0)
            dt_fix = 0.5 * s.time()[1]
            for _ in range(args.acc_steps):
                s.step(dt_fix)
            results.setdefault("acc", {})[prec] = (s.get_state()[0], dt_fix)
        if prec == "fp32" and not args.no_e2e:
            # end to end through the C ABI with host buffers: every step copies
            # its state in (pinned host -> device), steps, and copies the new
            # state out (device -> pinned host).  Serial: one solver, each
            # step waits for the last.  Pipelined: two solvers on two streams
            # take the steps in turn, so that one step's copy out overlaps the
            # next step's copy in and kernels (the two copy directions use
            # separate copy engines).
            Upin = [torch.empty((3, 4, N), dtype=torch.float64, pin_memory=True).numpy() for _ in range(2)]
            Uout = [torch.empty((3, 4, N), dtype=torch.float64, pin_memory=True).numpy() for _ in range(2)]
            for u in Upin:
                u[...] = U0
            Ke = max(3, min(K, args.e2e_steps))
            s.set_state(Upin[0]); s.step(); s.get_state(out=Uout[0])
            torch.cuda.synchronize(); barrier()
            t0 = time.perf_counter()
            for _ in range(Ke):
                s.set_state(Upin[0])
                s.step()
                s.get_state(out=Uout[0])
            el_serial = max_over_ranks(time.perf_counter() - t0)
            pair = [hweno.Solver(hmesh, U0, eq="euler", precision=prec, stream=torch.cuda.Stream(),
                                 time_rule=args.time_rule, step_kernels=args.step_kernels) for _ in range(2)]

            def pipelined(n):
                prev = None
                for k in range(n):
                    cur = pair[k % 2]
                    cur.set_state(Upin[k % 2])
                    cur.step()
                    if prev is not None:
                        prev[0].get_state(out=prev[1])
                    prev = (cur, Uout[k % 2])
                prev[0].get_state(out=prev[1])

            pipelined(4)
            torch.cuda.synchronize(); barrier()
            t0 = time.perf_counter()
            pipelined(Ke)
            el = max_over_ranks(time.perf_counter() - t0)
            for q in pair:
                q.close()
            del pair
            results["e2e"] = {"steps": Ke, "s": el, "s_serial": el_serial, "bytes": 3 * 4 * N * 8}
        s.close()
        del s
        torch.cuda.empty_cache()

    fused_line = None
    if args.only == "both" and args.step_kernels == "default":
        # the fused reconstruct-and-flux kernel (option step_kernels = 2) on the same workload
        sf = hweno.Solver(hmesh, U0, eq="euler", precision="fp32", step_kernels="fused")
        for _ in range(args.warmup):
            sf.step()
        sf.profile(True)
        for _ in range(min(200, args.steps)):
            sf.step()
        pf = sf.profile_read()
        sf.profile(False)
        sf.close()
        ms_f = pf["recon_ms"] / max(1, pf["steps"])
        fused_line = {"kernel": "k_fused", "ms_per_step": ms_f, "steps": pf["steps"], "value": N / (ms_f * 1e-3),
                 "alg_bytes_per_cell": alg_bytes("fused", 4),
                 "achieved_gbs": alg_bytes("fused", 4) * N / (ms_f * 1e-3) / 1e9}
    batched = None
    if args.only == "both" and not args.no_batch and world > 1:
        batched = batched_leg(args, world)   # every rank takes part
    if rank != 0:
        return
    if args.only != "both" or args.no_e2e or args.time_rule != "lobatto":
        print(json.dumps({"partial_run": True, "N": N, **{k: v for k, v in results.items() if k != "acc"}}), flush=True)
        return
    hbm, peak_kind = measured_peaks()
    r32 = results["fp32"]
    K = r32["K"]
    value = replicas_value(N, K, r32["ms"], world)
    rec_ms = r32["prof"]["recon_ms"] / max(1, r32["prof"]["steps"])
    edge_ms = r32["prof"]["edge_ms"] / max(1, r32["prof"]["steps"])
    fused = r32["kernels"] == "fused"
    if fused:
        dom, dom_ms = "fused", rec_ms
        kernel_ms = {"k_fused": rec_ms}
    else:
        dom = "recon" if rec_ms >= edge_ms else "edge"
        dom_ms = max(rec_ms, edge_ms)
        kernel_ms = {"k_recon": rec_ms, "k_edge": edge_ms}
    achieved = alg_bytes(dom, 4) * N / (dom_ms * 1e-3) / 1e9
    sha = kernel_sources_sha()
    tr = TRAFFIC["per_cell"].get(f"{dom}_fp32") if TRAFFIC["sources_sha"] == sha else None
    r64 = results["fp64"]
    rec64 = r64["prof"]["recon_ms"] / max(1, r64["prof"]["steps"])
    edge64 = r64["prof"]["edge_ms"] / max(1, r64["prof"]["steps"])
    e2e = results["e2e"]
    acc = None
    if "acc" in results and len(results["acc"]) == 2:
        (U32, dt32), (U64, dt64) = results["acc"]["fp32"], results["acc"]["fp64"]
        if abs(dt32 - dt64) <= 1e-6 * dt64:
            area = I.cell_areas(mesh)
            d = np.abs(U32[0] - U64[0])
            acc = {"steps": args.acc_steps, "what": "cell averages, FP32 - FP64 after the same fixed steps",
                   "l1": ((d * area).sum(axis=1) / area.sum()).tolist(), "linf": d.max(axis=1).tolist()}
    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": K,
        "warmup": args.warmup,
        "ms_per_step": r32["ms"] / K,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"euler-isentropic-vortex, periodic [0,10]^2, Poisson-disk Delaunay, {N} triangles",
                   "triangles": N, "equation": "euler", "precision": "fp32 state/arithmetic, fp64 precompute",
                   "l2": "inputs larger than L2 (working set %.2f GB)" % (
                       (86 * 4 + 16 + 2 * 48 + 288) * N / 1e9),
                   "parallelism": "replicas" if world > 1 else "single-gpu"},
        "roofline": {"bound": "hbm", "kernel": f"k_{dom}", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "peak_kind": peak_kind, "alg_bytes_per_cell": alg_bytes(dom, 4),
                     "traffic": (tr * N) if tr else None,
                     "kernel_ms": kernel_ms, "step_kernels": r32["kernels"]},
        "e2e": {"value": replicas_value(N, e2e["steps"], e2e["s"] * 1e3, world), "unit": UNIT,
                "h2d_bytes_per_step": e2e["bytes"], "d2h_bytes_per_step": e2e["bytes"],
                "how": "two solvers on two streams take the steps in turn (copy out of one step overlaps "
                       "the copy in and kernels of the next)",
                "serial_value": replicas_value(N, e2e["steps"], e2e["s_serial"] * 1e3, world)},
        "gpu_launches": (1 if fused else 2) * K,
        "clocks": r32["clocks"],
        "fp64": {"value": replicas_value(N, r64["K"], r64["ms"], world), "steps": r64["K"],
                 "ms_per_step": r64["ms"] / r64["K"], "step_kernels": r64["kernels"],
                 "kernel_ms": {"k_recon": rec64,
                               ("k_edge_flux+k_edge_update" if r64["kernels"] == "edge_once" else "k_edge"): edge64},
                 "clocks": r64["clocks"], "roofline": fp64_roofline(N, rec64, edge64, r64["clocks"], sha)},
        "status_flags": {"fp32": r32["flags"], "fp64": r64["flags"]},
        "fp32_vs_fp64": acc,
        "fused_step": fused_line,
    }
    if not args.no_batch:
        line["batched"] = batched if batched is not None else batched_leg(args, world)
    if not args.no_adjoint:
        line["adjoint"] = adjoint_leg(args)
    if args.partition:
        line["partition"] = partition_leg(args)
    if not args.no_cpu:
        r = cpu_oracle_rates(mesh, U0, args.cpu_seconds)
        line["cpu_baseline"] = {
            "value": r["all_cores"], "unit": UNIT, "cores": r["workers"], "kind": "oracle",
            "single_core_value": r["single_core"], "nproc": r["nproc"],
            "sample": (f"FP64 oracle steps of {r['patch_cells']}-cell patches of the {N}-cell mesh, "
                       f"{r['seconds_per_worker']:.0f} s per process, one single-threaded process per core "
                       f"({r['workers']} processes; rates added); single_core_value: one process")}
    print(json.dumps(line), flush=True)


def fp64_roofline(N, rec_ms, edge_ms, clocks, sha):
    """The FP64 form is bound by the FP64 pipe: achieved FLOP/s of its dominant
    kernel against the probe's FP64 rate at the sampled SM clock."""
    if TRAFFIC["sources_sha"] != sha:
        return None
    dom, ms = ("recon", rec_ms) if rec_ms >= edge_ms else ("edge", edge_ms)
    achieved = FLOPS[f"{dom}_fp64"] * N / (ms * 1e-3) / 1e12
    peak = FP64_FLOP_PER_CLOCK * clocks["sm_mhz"] * 1e6 / 1e12 if clocks.get("sm_mhz") else None
    return {"bound": "alu", "kernel": f"k_{dom}", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak if peak else None, "flop_per_cell": FLOPS[f"{dom}_fp64"],
            "peak_kind": "2 FP64 FMA per SM per clock (nominal 1.25 TFLOP/s at 2032 MHz) at the sampled SM clock"}


# ---------------------------------------------------------------- batched leg
def batched_leg_dealt(args, world, meshes, states, T):
    """N ranks: the solves dealt to ranks by size (no communication on the data
    path); whole-job rate = all ranks' triangle updates / the slowest rank's
    time.  Every rank runs this; rank 0 reports."""
    import torch
    import torch.distributed as tdist
    from paper_2607_10809_b300 import hweno
    from paper_2607_10809_b300 import partition as PT
    rank = tdist.get_rank()
    mine = PT.deal_solves([m.nt for m in meshes], world)[rank]
    b = hweno.Batch([meshes[k] for k in mine], [states[k] for k in mine], eq="euler", precision="fp32",
                    positivity=True)
    b.autotune(trial_steps=6)
    b.reset()
    dist_barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    try:
        cells = b.run_to(T)
    except hweno.HwError:
        cells = sum(b.get_state(k)[2] * meshes[mine[k]].nt for k in range(len(mine)))
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    failed = sum(1 for k in range(len(mine)) if b.get_state(k)[3])
    b.close()
    v = torch.tensor([el, float(cells), float(failed)], dtype=torch.float64, device="cuda")
    tmax = v[:1].clone(); tdist.all_reduce(tmax, op=tdist.ReduceOp.MAX)
    tsum = v[1:].clone(); tdist.all_reduce(tsum, op=tdist.ReduceOp.SUM)
    return {"workload": f"{len(meshes)} four-quadrant Riemann solves dealt to {world} ranks by size",
            "value": float(tsum[0]) / float(tmax[0]), "unit": UNIT, "seconds": float(tmax[0]),
            "cell_steps": int(tsum[0]), "failed_solves": int(tsum[1]), "scaling": "strong"}


def batched_leg(args, world):
    """256 four-quadrant Riemann solves (2k-40k triangles each, FP32, scale
    limiter) advanced to T = 0.25 in one persistent launch with the autotuned
    schedule, against the same solves run one after another through the
    single-solve path, and against the plain FP64 single-solve form on a
    sample of the solves (its throughput, and the batched FP32 states'
    relative L1 difference to it, per solve that both forms carried to T)."""
    import torch
    from paper_2607_10809_b300 import hweno
    meshes, states = I.config4_batch(args.batch_solves)
    T = args.batch_T
    if world > 1:
        return batched_leg_dealt(args, world, meshes, states, T)
    b = hweno.Batch(meshes, states, eq="euler", precision="fp32", positivity=True)
    best = b.autotune(trial_steps=6)
    b.reset()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    try:
        cell_steps = b.run_to(T)
        status = "ok"
    except hweno.HwError as e:
        status = str(e).split(":")[0]
        cell_steps = sum(b.get_state(k)[2] * m.nt for k, m in enumerate(meshes))
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    failed = sum(1 for k in range(len(meshes)) if b.get_state(k)[3])
    steps = [b.get_state(k)[2] for k in range(len(meshes))]
    # a sample of the solves (spread over the sizes) for the FP64 reference below
    nref = min(args.batch_fp64_solves, len(meshes))
    order = np.argsort([m.nt for m in meshes], kind="stable")
    sample = [int(order[int(round(k * (len(meshes) - 1) / max(1, nref - 1)))]) for k in range(nref)]
    batched_states = {k: b.get_state(k) for k in sample}
    b.close()
    # the same solves one by one through the single-solve path (graph-captured run_to)
    seq_cells, seq_time = 0, 0.0
    for mesh, U0 in zip(meshes, states):
        s = hweno.Solver(mesh, U0, eq="euler", precision="fp32", positivity=True)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        try:
            n = s.run_to(T)
        except hweno.HwError:
            n = s.time()[2]
        torch.cuda.synchronize()
        seq_time += time.perf_counter() - t1
        seq_cells += n * mesh.nt
        s.close()
    # the plain FP64 single-solve form on the sample: its throughput, and the
    # batched FP32 states against it
    ref_cells, ref_time, errs = 0, 0.0, []
    for k in sample:
        s = hweno.Solver(meshes[k], states[k], eq="euler", precision="fp64", positivity=True)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        try:
            n = s.run_to(T)
            ok = True
        except hweno.HwError:
            n, ok = s.time()[2], False
        torch.cuda.synchronize()
        ref_time += time.perf_counter() - t1
        ref_cells += n * meshes[k].nt
        Ub, tb, _, fb = batched_states[k]
        if ok and not fb:
            U64 = s.get_state()[0]
            area = I.cell_areas(meshes[k])
            d = np.abs(Ub[0] - U64[0])
            errs.append(float(((d * area).sum(axis=1) / area.sum() / np.abs(U64[0]).max(axis=1)).max()))
        s.close()
    fp64_ref = {"solves": sample, "value": ref_cells / ref_time, "unit": UNIT, "seconds": ref_time,
                "fp32_batched_vs_fp64_rel_l1": {"median": float(np.median(errs)) if errs else None,
                                                 "max": float(np.max(errs)) if errs else None,
                                                 "solves_compared": len(errs)}}
    return {"workload": f"{len(meshes)} four-quadrant Riemann solves on [0,1]^2, "
                        f"{sum(m.nt for m in meshes)} triangles, FP32 + scale limiter, T={T}",
            "value": cell_steps / el, "unit": UNIT, "seconds": el, "cell_steps": int(cell_steps),
            "steps_min_max": [int(min(steps)), int(max(steps))], "failed_solves": failed, "status": status,
            "schedule": best, "single_solve_sequential_value": seq_cells / seq_time,
            "single_solve_sequential_seconds": seq_time, "fp64_single_solve": fp64_ref}


# ---------------------------------------------------------------- adjoint leg
def adjoint_leg(args):
    """Gradient of the density misfit J = 1/2 sum_K |K| (rho_K(T) - rho*_K)^2
    with respect to the initial state (W, W_x, W_y averages), rho* the exact
    unperturbed vortex at T, through `adj_steps` FP32 steps on the 199,712-cell
    jittered periodic mesh of [0, 10]^2 (vortex + 8 density bumps), checkpoints
    every 10 steps.  Reported: the wall time of the backward pass (recompute
    and adjoint steps) over that of the plain forward run, the wall time of
    the whole gradient (checkpointed forward + backward) over the same (all
    from host arrays to host arrays, outputs into pinned memory), and the
    FP32 gradient's relative L-infinity difference to the FP64 gradient."""
    import torch
    from paper_2607_10809_b300 import hweno
    from paper_2607_10809_b300.adjoint import cfl_steps, rollout
    mesh = I.config5_mesh()
    U0 = I.config5_state(mesh)
    area = torch.from_numpy(I.cell_areas(mesh))
    every = 10
    out, grads = {}, {}
    dts = None
    for prec in ("fp32", "fp64"):
        s = hweno.Solver(mesh, U0, eq="euler", precision=prec)
        if dts is None:
            dts = cfl_steps(s, U0, args.adj_steps)
            T = float(np.sum(dts))
            rho_star = torch.from_numpy(I.cell_averages(mesh, lambda x, y: I.vortex(x, y, T), 4)[0])

        Uout = torch.empty(U0.shape, dtype=torch.float64, pin_memory=True).numpy()

        def forward():
            s.set_state(U0, 0.0)
            for dt in dts:
                s.step(dt)
            return s.get_state(out=Uout)[0]

        def gradient():
            """(seconds of the checkpointed forward pass, of the backward pass), dJ/dU0, J"""
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            x = torch.from_numpy(U0.copy()).requires_grad_(True)
            UT = rollout(x, s, dts, every)
            J = 0.5 * (area * (UT[0, 0] - rho_star) ** 2).sum()
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            J.backward()
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            return (t1 - t0, t2 - t1), x.grad.numpy(), float(J.detach())

        def timed(fn, reps):
            ts = []
            for _ in range(reps):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                r = fn()
                torch.cuda.synchronize()
                ts.append(time.perf_counter() - t0)
            return statistics.median(ts), r

        reps = 3 if prec == "fp32" else 1
        forward(); gradient()                       # warm-up (graph/allocator/first-touch)
        t_fwd, _ = timed(forward, reps)
        runs = [gradient() for _ in range(reps)]
        t_ck = statistics.median(r[0][0] for r in runs)
        t_bwd = statistics.median(r[0][1] for r in runs)
        t_adj = statistics.median(r[0][0] + r[0][1] for r in runs)
        _, g, J = runs[-1]
        grads[prec] = g
        out[prec] = {"forward_s": t_fwd, "checkpointed_forward_s": t_ck, "backward_s": t_bwd,
                     "forward_backward_s": t_adj, "ratio": t_bwd / t_fwd, "gradient_ratio": t_adj / t_fwd,
                     "J": J}
        s.close()
        del s
        torch.cuda.empty_cache()
    err = float(np.abs(grads["fp32"] - grads["fp64"]).max() / np.abs(grads["fp64"]).max())
    return {"workload": f"euler vortex + 8 density bumps, jittered periodic [0,10]^2, {mesh.nt} triangles, "
                        f"{len(dts)} steps, checkpoint every {every}",
            "metric": "adjoint/forward wall time", "value": out["fp32"]["ratio"], "unit": "x",
            "what": "value: the backward pass (recomputation of the checkpoint segments and the adjoint steps) "
                    "over the plain forward run; gradient_ratio: checkpointed forward + backward over the plain "
                    "forward run",
            "higher_is_better": False, "fp32": out["fp32"], "fp64": out["fp64"],
            "grad_fp32_vs_fp64_rel_linf": err}


# ---------------------------------------------------------------- partition leg
def partition_leg(args):
    """One mesh cut into P parts (Hilbert ranges + two halo rings), the parts
    advanced one after another on this one GPU with the device-resident halo
    exchange: the partitioned step's cost on one GPU, split into the parts'
    step kernels (CUDA events) and the rest (dt minimum over the parts, halo
    rows out and in, CFL refresh, host calls).  On P GPUs the parts' steps would run side by side; this measures
    the redundant halo work and the exchange's device-side cost, not a
    scaling curve."""
    import torch
    from paper_2607_10809_b300 import hweno
    from paper_2607_10809_b300 import partition as PT
    mesh, U0 = workload(args.workload)
    N = mesh.nt
    perm = hweno.Mesh(mesh).permutation()
    out = {"workload": f"{args.workload}: {N} triangles, FP32", "parts": {}}
    K = args.partition_steps
    for P in [int(x) for x in (args.partition or "2,4").split(",")]:
        parts = PT.build(mesh, perm, P)
        steppers = [PT.DeviceStepper(hweno.Solver(p.mesh, PT.scatter_state(U0, p), eq="euler", precision="fp32"), p)
                    for p in parts]
        PT.run_local_device(parts, steppers, 3)
        torch.cuda.synchronize()
        for st in steppers:
            st.s.profile(True)      # the parts' step kernels, timed with CUDA events
        t0 = time.perf_counter()
        PT.run_local_device(parts, steppers, K)
        torch.cuda.synchronize()
        total = (time.perf_counter() - t0) / K
        steps_only = 0.0
        for st in steppers:
            pr = st.s.profile_read()
            st.s.profile(False)
            steps_only += (pr["recon_ms"] + pr["edge_ms"]) * 1e-3 / pr["steps"]
        local = int(sum(p.cells.size for p in parts))
        out["parts"][str(P)] = {"ms_per_step": total * 1e3, "parts_steps_ms": steps_only * 1e3,
                                "exchange_ms": (total - steps_only) * 1e3, "local_cells": local,
                                "halo_fraction": local / N - 1.0, "steps": K}
        for st in steppers:
            st.s.close()
        del steppers
        torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    """The FP64 CPU oracle as the reference arm, on one host core: each step is
    one oracle step of a patch of the same workload (the cpu_baseline's
    single-core measurement, with --steps / --warmup)."""
    if rank != 0:
        return
    mesh, U0 = workload(args.workload)
    n = args.ref_cells
    local, Ul, idx = oracle_patch(mesh, U0, (5.0, 5.0), n)
    k, el = time_patch_steps(local, Ul, idx, steps=args.steps, warmup=args.warmup)
    value = n * k / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / k * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"euler-isentropic-vortex, periodic [0,10]^2, Poisson-disk Delaunay, {mesh.nt} triangles",
                       "triangles": mesh.nt},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"each step: one FP64 oracle step of a {n}-cell patch of the {mesh.nt}-cell mesh"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="vortex2m", choices=["vortex2m", "vortex500k"])
    ap.add_argument("--fp64-divisor", type=int, default=20, help="FP64 timed steps = steps / divisor")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end measurement")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched (many solves) leg")
    ap.add_argument("--batch-solves", type=int, default=256)
    ap.add_argument("--batch-T", type=float, default=0.25, help="final time of the batched solves")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint (gradient) leg")
    ap.add_argument("--adj-steps", type=int, default=200)
    ap.add_argument("--partition", default="", help="comma-separated part counts of the partition leg (off if empty)")
    ap.add_argument("--partition-steps", type=int, default=50)
    ap.add_argument("--only", default="both", choices=["both", "fp32", "fp64", "adjoint", "batched", "partition"],
                    help="precisions to run, or one leg alone")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--acc-steps", type=int, default=50, help="fixed steps of the FP32-vs-FP64 accuracy check")
    ap.add_argument("--time-rule", default="lobatto", choices=["lobatto", "gauss"],
                    help="time rule of the edge flux in the single-solve legs (gauss: ablation runs only)")
    ap.add_argument("--batch-fp64-solves", type=int, default=16,
                    help="solves of the batch re-run one by one in FP64 (accuracy and FP64 throughput)")
    ap.add_argument("--ref-cells", type=int, default=2000)
    ap.add_argument("--step-kernels", default="default", choices=["default", "separate", "fused", "edge_once"],
                    help="kernels of the single-solve step (default: the two-sided flux kernel in FP32, the edge-once flux phase in FP64)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(local_rank)
        tdist.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as tdist
        tdist.destroy_process_group()


if __name__ == "__main__":
    main()
