#!/usr/bin/env python
"""Throughput of the GB300 lattice Boltzmann hot path (arXiv 2512.12213).

Headline (value): D3Q19 flow past a sphere, 256 x 128 x 128 nodes, periodic
box, body force, populations stored as shifted binary16 (FP32 arithmetic);
one step = the fused collide-stream kernel plus the FP64 momentum-exchange
drag on the sphere (link kernel + fixed-order reduction), every step.
Reported beside it on the same workload: FP64, FP32 and bfloat16 storage
with their drag error against FP64; the FP32 D3Q19 lid-driven LES cavity;
adjoint throughput on the 2-D cylinder; an end-to-end run through host
buffers; the roofline of the fused step kernel; the CPU oracle.

    python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]

N > 1 runs N independent replicas (one per rank, launched by torchrun) and
reports their summed throughput.
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
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "D3Q19 MLUPS & % HBM roofline, mixed vs FP64 at stated drag error; adjoint MLUPS"
WORKLOAD = ("D3Q19 sphere r=12 in 256x128x128 periodic box, Re 20 configuration (tau 0.68, calibrated body force; steady Re 19.9), started from rest, model [e], halfway bounce-back")
FALLBACK_HBM = 6800.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--repeats", type=int, default=5, help="timed blocks of --steps steps; the median is reported")
    p.add_argument("--study", default=None, choices=["steady"],
                   help="instead of the benchmark: run the sphere to steady state in every storage (long)")
    p.add_argument("--study-out", default=None,
                   help="also write the study's JSON line to this file (profiles/steady_sphere.json keeps the record)")
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--drag-steps", type=int, default=2000)
    p.add_argument("--no-extras", action="store_true", help="headline only")
    p.add_argument("--storage", default="f16s", choices=["f64", "f32", "f16s", "bf16s"],
                   help="storage of the headline run (profiling)")
    p.add_argument("--rounding", default="stochastic", choices=["nearest", "stochastic"],
                   help="rounding of 16-bit stores in the headline run")
    p.add_argument("--size", type=int, default=256, help="edge of the cavity workload (profiling)")
    p.add_argument("--step-kernel", default="auto", choices=["auto", "register", "staged"],
                   help="ask the context for one step kernel (comparisons; the default lets the library choose)")
    p.add_argument("--workload", default="sphere", choices=["sphere", "cavity"] + list(EXTENSIONS),
                   help="headline workload (profiling): sphere 256x128x128, cavity 256^3 LES, or the "
                        "sphere box with one extension (curved walls, insulating walls, Brinkman, induced field)")
    return p.parse_args()


# ------------------------------------------------------------------ helpers
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(torch, dist, ws, value, device):
    """The largest of every rank's value (the slowest replica's time); the
    value itself on one rank.  Barrier first, so no rank reads a time that
    another rank has not finished."""
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if ws > 1:
        dist.barrier()
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(ws, nodes, steps, total_ms):
    """Node updates of all replicas per second (weak scaling: every rank
    advances its own box of `nodes` nodes `steps` times), in millions."""
    return ws * nodes * steps / (total_ms * 1e-3) / 1e6


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


# sources that compile into the step kernel (host code, the adjoint and the
# allocation-free wall force are left out)
STEP_SOURCES = ("lbm_device.cuh", "lbm_kernels.cuh", "lbm_staged.cuh", "lbm_internal.h",
                "inst_f64.cu", "inst_f32.cu", "inst_f16.cu", "inst_bf16.cu")


def source_hash():
    """Hash of the step kernel's sources, to match committed ncu figures."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2512_12213_gb300", "csrc")
    for f in STEP_SOURCES:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def traffic_for(key):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel sources; else None."""
    try:
        d = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
        e = d.get(key)
        if e and e.get("source_sha") == source_hash():
            return float(e["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


class Clocks:
    """Samples SM clock and throttle reasons with nvidia-smi while running."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.samples, self.proc, self.active = index, [], None, False

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            if self.active:
                self.samples.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if len(s) > 3 + i and s[3 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


# --------------------------------------------------------------- our arm
def bytes_per_node(Q, storage, induced=False):
    """Algorithmic bytes of one node update: read + write every population
    plus the node-class byte; with the induced field also read + write the
    3 x 7 field distributions (compute precision)."""
    s = {"f64": 8, "f32": 4, "f16s": 2, "bf16s": 2}[storage]
    b = 2 * Q * s + 1
    if induced:
        b += 2 * 3 * (5 if Q == 9 else 7) * (8 if storage == "f64" else 4)
    return b


# the sphere box with each extension of the core step: workload builder,
# step kernel(s) timed, and a description
EXTENSIONS = {
    "curved": ("sphere_curved", "k_step<19,S,EXT=0,FULL=1> (interpolated bounce-back in boundary chunks)",
               "true sphere r=12.4 as the wall, linear interpolated bounce-back from the signed distance"),
    "insulating": ("sphere_insulating", "k_step<19,S,EXT=1,FULL=1> + k_ins_update",
                   "imposed field (0, 0.02, 0), sigma_e = 1, Lorentz force, insulating walls E = -<v> x B"),
    "brinkman": ("sphere_brinkman", "k_step<19,S,EXT=1>",
                 "linear (Stokes) equilibrium, Darcy resistance 1e-4 (Brinkman)"),
    "induced": ("sphere_induced", "k_mhd_step<19,S> (fluid D3Q19 + field D3Q7, one node per thread)",
                "external field (0, 0.02, 0), induced field on D3Q7, eta = 0.05, Maxwell equilibrium at the local field"),
}


def make_workload(workloads, name, storage, size=256):
    """(cfg, mask, phi or None) of a named workload."""
    if name == "sphere":
        c, m = workloads.sphere(storage=storage)
        return c, m, None
    if name == "cavity":
        c, m = workloads.cavity(n=size, storage=storage)
        return c, m, None
    out = getattr(workloads, EXTENSIONS[name][0])(storage=storage)
    return out if len(out) == 3 else (out[0], out[1], None)


def timed_run(torch, lbm, sim, steps, warmup, wall=1, events=True, repeats=1):
    """Warm up, then time `repeats` blocks of exactly `steps` steps with CUDA
    events on the launching stream.  A step is the fused collide-stream
    kernel plus the FP64 wall force of the interval it advances over.  With
    the staged kernel both are one call (lbm_step_force: the force summed
    inside the step kernel, then its fixed-order pass; the step-kernel time
    then includes the force).  Otherwise the force reads the stored state
    that the step only reads, so it runs on a second stream beside the step
    (it waits for the previous step, and the next step waits for it).
    Returns (median block ms, every block's ms, mean step-kernel ms of the
    extra block whose launches carry events)."""
    st = sim.stream
    cs = torch.cuda.current_stream()
    side = torch.cuda.Stream(device=cs.device)
    hist = torch.zeros((max(steps, warmup, 1), 3), dtype=torch.float64, device=sim.device)
    # lbm_step_force sums the drag inside the staged step in boxes periodic
    # on every axis with the plain node code; elsewhere it is two calls
    c = sim.cfg
    ext = c.lorentz or c.maxwell or c.les or c.stokes or c.darcy > 0
    periodic = c.periodic[0] and c.periodic[1] and (c.lattice == 9 or c.periodic[2])
    fused = sim.step_kernel == "staged" and periodic and not ext

    def one(i, a=None, b=None):
        if fused:
            # the staged kernel sums the wall force inside the step (one
            # launch, plus the fixed-order pass of its block rows)
            if a is not None:
                a.record(cs)
            lbm.lbm_step_force(sim.ctx, wall, 0, 1.0, hist[i], 0, st)
            if b is not None:
                b.record(cs)
            return
        side.wait_stream(cs)
        lbm.lbm_wall_force(sim.ctx, wall, 0, 1.0, hist[i], 0, side.cuda_stream)
        if a is not None:
            a.record(cs)
        lbm.lbm_step(sim.ctx, 1, st)
        if b is not None:
            b.record(cs)
        cs.wait_stream(side)

    lbm.lbm_step(sim.ctx, 1, st)         # the wall force needs one step taken
    for i in range(warmup):
        one(i)
    torch.cuda.synchronize()

    def block(a, b):
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record(cs)
        for i in range(steps):
            one(i, a[i], b[i])
        t1.record(cs)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1)

    # the value blocks carry no per-step events (an event between two steps
    # opens a gap of a few microseconds); one more block times every
    # step-kernel launch for the roofline
    blocks = [block([None] * steps, [None] * steps) for _ in range(repeats)]
    kern = None
    if events and fused:
        # one launch per step: the launches run back to back, so the average
        # launch duration is the block's time over its launches (events
        # around every launch would add their own gaps)
        kern = statistics.median(blocks) / steps
    elif events:
        a = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        b = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        block(a, b)
        kern = sum(x.elapsed_time(y) for x, y in zip(a, b)) / steps
    return statistics.median(blocks), blocks, kern


def run_ours(args):
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2512_12213_gb300 import build, lbm, workloads
    build.build()
    lbm.load()

    clocks = Clocks(local)
    clocks.start()
    hbm, peak_kind = peaks()
    out = {}

    # ---- headline: sphere, shifted binary16 storage
    cfg, mask, phi = make_workload(workloads, args.workload, args.storage, args.size)
    hwall = 2 if args.workload == "cavity" else 1
    sr = args.storage in ("f16s", "bf16s") and args.rounding == "stochastic"
    if sr:
        cfg = dict(cfg, rounding="stochastic", seed=2024)
    if args.step_kernel != "auto":
        cfg = dict(cfg, step_kernel=args.step_kernel)
    sim = lbm.Sim(cfg, mask)
    if phi is not None:
        sim.set_wall_distance(phi)
    sim.rest()
    step_kernel = sim.step_kernel
    N = cfg["nx"] * cfg["ny"] * cfg["nz"]
    fluid = int((mask == 0).sum())
    bpn = bytes_per_node(19, args.storage, induced=bool(cfg.get("induced")))
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.active = True
    total_ms, blocks_ms, kern_ms = timed_run(torch, lbm, sim, args.steps, args.warmup, wall=hwall,
                                             repeats=args.repeats)
    clocks.active = False
    total_ms = max_over_ranks(torch, dist, ws, total_ms, "cuda")
    ms_step = total_ms / args.steps
    value = whole_job_mlups(ws, N, args.steps, total_ms)
    achieved = N * bpn / (kern_ms * 1e-3) / 1e9
    kname = {"f64": "StoreF64", "f32": "StoreF32", "f16s": "StoreF16", "bf16s": "StoreBF16"}[args.storage]
    if args.workload in EXTENSIONS:
        kernel = EXTENSIONS[args.workload][1].replace(",S", "," + kname)
    elif step_kernel == "staged":
        kernel = f"k_step_staged<19,{kname},SR={int(sr)}>"
    else:
        kernel = f"k_step<19,{kname},EXT={int(bool(cfg.get('les')))},SR={int(sr)}>"
    roof = {"kernel": kernel, "bound": "hbm", "achieved": round(achieved, 1),
            "peak": hbm, "unit": "GB/s", "frac": round(achieved / hbm, 4), "peak_source": peak_kind,
            "bytes_per_node": bpn, "step_kernel_ms": round(kern_ms, 5),
            "kernel_mlups": round(N / (kern_ms * 1e-3) / 1e6, 1),
            "traffic": traffic_for(f"{args.workload}256_{args.storage}{'_sr' if sr else ''}_{step_kernel}")}
    sim.close()
    del sim
    torch.cuda.empty_cache()

    if rank == 0 and not args.no_extras and args.workload == "sphere" and args.storage == "f16s" and sr:
        # ---- the same workload in the other storage formats, and drag error vs FP64
        variants = {}
        for key, steps in (("f32", args.steps), ("f16s", args.steps), ("bf16s_sr", args.steps),
                           ("f64", max(args.steps // 4, 50))):
            storage = key.split("_")[0]
            c, m = workloads.sphere(storage=storage)
            if key.endswith("_sr"):
                c = dict(c, rounding="stochastic", seed=2024)
            s = lbm.Sim(c, m)
            s.rest()
            clocks.active = True
            t, _, k = timed_run(torch, lbm, s, steps, args.warmup)
            clocks.active = False
            bp = bytes_per_node(19, storage)
            ach = N * bp / (k * 1e-3) / 1e9
            variants[key] = {"mlups": round(N * steps / (t * 1e-3) / 1e6, 1),
                                 "kernel_mlups": round(N / (k * 1e-3) / 1e6, 1),
                                 "achieved_gbs": round(ach, 1), "frac": round(ach / hbm, 4)}
            s.close()
            del s
            torch.cuda.empty_cache()
        variants["f16s_sr"] = {"mlups": round(value / ws, 1), "kernel_mlups": roof["kernel_mlups"],
                               "achieved_gbs": roof["achieved"], "frac": roof["frac"]}
        out["storage_variants"] = variants
        out["drag_error_vs_f64"] = drag_errors(torch, lbm, workloads, args.drag_steps)
        out["momentum_defect"] = momentum_defect(torch, lbm, workloads)
        out["near_steady_vs_f64"] = {f"re{re}": near_steady(torch, lbm, workloads, re) for re in (20, 100)}
        out["steady_state_study"] = steady_record()
        out["cavity_les_f32"] = cavity_bench(torch, lbm, workloads, hbm, args)
        out["cavity_sweep"] = cavity_sweep(torch, lbm, workloads, hbm, args)
        out["extensions_f32"] = extensions_bench(torch, lbm, workloads, hbm, args)
        out["adjoint"] = adjoint_bench(torch, lbm, workloads, hbm)
        e2e = e2e_bench(torch, lbm, workloads, args)
        cpu = cpu_baseline()
    else:
        e2e, cpu = None, None

    clocks.stop()
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_step, 5), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": {"sphere": WORKLOAD, "cavity": f"D3Q19 LES cavity {args.size}^3"}.get(
                           args.workload, WORKLOAD + "; " + EXTENSIONS.get(args.workload, ("", "", ""))[2]),
                       "nodes": N, "fluid_nodes": fluid,
                       "storage": args.storage + (" (shifted x2^12, stochastic rounding)" if sr and args.storage == "f16s"
                                                  else (" (stochastic rounding)" if sr else "")),
                       "compute": "f32",
                       "step": ("collide-stream with the FP64 drag summed in the step kernel + its fixed-order "
                                "reduction" if step_kernel == "staged" else
                                "fused collide-stream + FP64 drag reduction (on a second stream beside the step)"),
                       "l2": f"inputs larger than L2: {N * (bpn - 1) / 2 / 1e6:.0f} MB of populations read and the same "
                  "written per step",
                       "parallelism": f"{ws} independent replica(s)"},
            "roofline": roof, "gpu_launches": (1 if step_kernel == "staged" else 3) * args.steps,
            "clocks": clocks.summary(),
            "repeats": {"blocks": args.repeats, "block_ms": [round(b, 4) for b in blocks_ms],
                        "value_from": "median block (no per-step events); the roofline's kernel time is the "
                                      "median block over its launches where a step is one launch (staged "
                                      "kernel, drag fused), else an event pair around every step launch in "
                                      "one more block; gpu_launches counts one block"},
            "step_kernel": step_kernel,
        }
        if e2e:
            line["e2e"] = e2e
        if cpu:
            line["cpu_baseline"] = cpu
        line.update(out)
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


def sphere_measure(s, mask, cfg, radius=12):
    """(drag F_x on the sphere, mean fluid velocity U, C_d, Re) of a sphere
    context after a step: F from the FP64 momentum exchange of the last step,
    U = M_x / mass, C_d = F / (rho U^2 pi r^2 / 2), Re = U 2r / nu."""
    F = s.wall_force(1)[0]
    mass, mom, _ = s.balance()
    fluid = int((mask == 0).sum())
    U = mom[0] / mass
    rho = mass / fluid
    nu = (cfg["tau"] - 0.5) / 3
    return F, U, F / (0.5 * rho * U * U * np.pi * radius ** 2), U * 2 * radius / nu


PRECISIONS = ("f64", "f32", "f16s", "bf16s", "f16s_sr", "bf16s_sr")


def _sphere_sim(lbm, workloads, key, Re=20):
    storage = key.split("_")[0]
    c, m = workloads.sphere(storage=storage, Re=Re)
    if key.endswith("_sr"):
        c = dict(c, rounding="stochastic", seed=2024)
    return c, m, lbm.Sim(c, m)


def momentum_defect(torch, lbm, workloads, keys=("f32", "f16s_sr", "bf16s_sr"), warm=1000, steps=2000):
    """The per-step momentum balance of the step in each FP32-compute storage
    on the sphere box (Re 20 configuration) from a uniform stream at
    U = 0.05: after `warm` steps, over `steps` more, the defect
    (M(T) - M(0) + sum_t F_wall(t)) / (T sum rho a) - 1, which every force
    model makes exactly zero in exact arithmetic (the discrete form of
    Eq. 32).  The wall force is summed on the device step by step."""
    out = {"workload": "sphere 256x128x128, Re 20 configuration, from a uniform stream at U = 0.05",
           "warm_steps": warm, "steps": steps}
    for key in keys:
        c, m, s = _sphere_sim(lbm, workloads, key)
        nz, ny, nx = m.shape
        u = np.zeros((3, nz, ny, nx))
        u[0] = 0.05 * (m == 0)
        s.init_equilibrium(np.ones((nz, ny, nx)), u)
        s.step(warm)
        _, M0, ra = s.balance()
        st = s.stream
        F = torch.zeros(3, dtype=torch.float64, device=s.device)
        for _ in range(steps):
            lbm.lbm_step(s.ctx, 1, st)
            lbm.lbm_wall_force(s.ctx, 1, lbm.ACCUMULATE, 1.0, F, 0, st)
        _, M1, _ = s.balance()
        out[key] = float((M1[0] - M0[0] + F[0].item()) / (steps * ra[0]) - 1)
        s.close()
        del s
        torch.cuda.empty_cache()
    return out


def drag_errors(torch, lbm, workloads, steps, checkpoints=(1000, 5000, 20000), radius=12):
    """Drag on the sphere (Re 20 configuration) from rest in each storage
    format, relative to FP64: at fixed steps of the start-up transient
    (`checkpoints`), averaged over the first `steps` steps, and as the drag
    coefficient C_d = F / (rho U^2 pi r^2 / 2) at the last checkpoint, U the
    mean fluid velocity there (the flow is still accelerating: see the
    near-steady block for the calibrated Reynolds number)."""
    T = max(max(checkpoints), steps)
    res = {}
    for key in PRECISIONS:
        c, m, s = _sphere_sim(lbm, workloads, key)
        s.rest()
        st = s.stream
        acc = torch.zeros(3, dtype=torch.float64, device=s.device)
        at = torch.zeros((len(checkpoints), 3), dtype=torch.float64, device=s.device)
        for i in range(T):
            lbm.lbm_step(s.ctx, 1, st)
            if i < steps:
                lbm.lbm_wall_force(s.ctx, 1, lbm.ACCUMULATE, 1.0 / steps, acc, 0, st)
            if i + 1 in checkpoints:
                lbm.lbm_wall_force(s.ctx, 1, 0, 1.0, at[checkpoints.index(i + 1)], 0, st)
        F, U, cd, re = sphere_measure(s, m, c, radius)
        Fx = at[:, 0].cpu().numpy()
        res[key] = {"at": Fx, "mean": float(acc[0].item()), "cd": cd, "re": re}
        s.close()
        del s
        torch.cuda.empty_cache()
    ref = res["f64"]
    out = {"workload": "sphere 256x128x128 from rest, Re 20 configuration (tau 0.68, calibrated g)",
           "checkpoints": list(checkpoints), "mean_window": steps,
           "f64_drag_at": [float(v) for v in ref["at"]], "f64_drag_mean": ref["mean"],
           "f64_cd_at_last": ref["cd"], "re_at_last": ref["re"]}
    for k in PRECISIONS[1:]:
        out[k] = {"rel_err_at": [float(abs(a / b - 1)) for a, b in zip(res[k]["at"], ref["at"])],
                  "rel_err_mean": abs(res[k]["mean"] / ref["mean"] - 1),
                  "cd_rel_err": abs(res[k]["cd"] / ref["cd"] - 1)}
    return out


def near_steady(torch, lbm, workloads, Re, checkpoints=(2000, 5000, 10000), radius=12):
    """The sphere at the calibrated Reynolds number: every storage format
    starts from the same uniform stream at the target speed (U0 of the
    workload) and runs 10,000 steps; at each checkpoint the drag, the mean
    velocity U, C_d and Re are compared with FP64, and at the last one the
    S2 shear stress field too (max |sigma - sigma_FP64| / max |sigma_FP64|
    over the fluid nodes)."""
    U0 = workloads.SPHERE_RE[Re]["U0"]
    res, sig64 = {}, None
    for key in PRECISIONS:
        c, m, s = _sphere_sim(lbm, workloads, key, Re)
        nz, ny, nx = m.shape
        u = torch.zeros((3, nz, ny, nx), dtype=torch.float64, device=s.device)
        u[0] = U0 * torch.from_numpy(m == 0).to(s.device)
        s.init_equilibrium(torch.ones((nz, ny, nx), dtype=torch.float64, device=s.device), u)
        rows, done = [], 0
        for cp in checkpoints:
            s.step(cp - done)
            done = cp
            rows.append(sphere_measure(s, m, c, radius))
        sig = s.stress(lbm.S2)[0].double()
        if key == "f64":
            sig64 = sig
            sig_err = 0.0
        else:
            sig_err = float((sig - sig64).abs().max() / sig64.abs().max())
        res[key] = {"rows": rows, "sigma_rel_err": sig_err}
        s.close()
        del s, sig
        torch.cuda.empty_cache()
    del sig64
    torch.cuda.empty_cache()
    ref = res["f64"]["rows"]
    out = {"workload": f"sphere 256x128x128, Re {Re} configuration (tau {workloads.SPHERE_RE[Re]['tau']}, "
                       f"g {workloads.SPHERE_RE[Re]['g']:.5g}), from a uniform stream at U0 = {U0}",
           "checkpoints": list(checkpoints),
           "f64": {"drag": [r[0] for r in ref], "U": [r[1] for r in ref], "cd": [r[2] for r in ref],
                   "re": [r[3] for r in ref]}}
    for k in PRECISIONS[1:]:
        rows = res[k]["rows"]
        out[k] = {"drag_rel_err": [abs(a[0] / b[0] - 1) for a, b in zip(rows, ref)],
                  "U_rel_err": [abs(a[1] / b[1] - 1) for a, b in zip(rows, ref)],
                  "cd_rel_err": [abs(a[2] / b[2] - 1) for a, b in zip(rows, ref)],
                  "sigma_s2_rel_err_at_last": res[k]["sigma_rel_err"]}
    return out


def steady_record():
    """The steady-state study as last recorded (profiles/steady_sphere.json,
    written by `python bench.py --study steady`), or None."""
    try:
        d = json.load(open(os.path.join(ROOT, "profiles", "steady_sphere.json")))
        d["source"] = "profiles/steady_sphere.json (python bench.py --study steady)"
        return d
    except Exception:
        return None


def cavity_bench(torch, lbm, workloads, hbm, args):
    n = 256
    c, m = workloads.cavity(n=n, storage="f32")
    s = lbm.Sim(c, m)
    s.rest()
    N = n ** 3
    steps = max(args.steps // 4, 50)
    t, _, k = timed_run(torch, lbm, s, steps, args.warmup, wall=2)
    bp = bytes_per_node(19, "f32")
    ach = N * bp / (k * 1e-3) / 1e9
    s.close()
    del s
    torch.cuda.empty_cache()
    return {"workload": "D3Q19 lid-driven cavity 256^3, lid u=0.1, tau=0.55, Smagorinsky Cs=0.1, FP32",
            "mlups": round(N * steps / (t * 1e-3) / 1e6, 1), "kernel_mlups": round(N / (k * 1e-3) / 1e6, 1),
            "achieved_gbs": round(ach, 1), "frac": round(ach / hbm, 4), "steps": steps}


def cavity_sweep(torch, lbm, workloads, hbm, args, sizes=(128, 256, 512), steps=20):
    """The LES lid-driven cavity (lid u = 0.1, tau = 0.55, Cs = 0.1) at 128^3,
    256^3 and 512^3 in FP64, FP32 and FP32 compute with binary16 storage
    (stochastic rounding): mean step-kernel rate and achieved HBM bandwidth
    against the measured peak.  Initial state from device tensors (no host
    staging buffer for the 512^3 boxes)."""
    res = {}
    for n in sizes:
        row = {}
        for storage in ("f64", "f32", "f16s"):
            c, m = workloads.cavity(n=n, storage=storage)
            if storage == "f16s":
                c = dict(c, rounding="stochastic", seed=2024)
            s = lbm.Sim(c, m, stage=False)
            N = n ** 3
            s.init_equilibrium(torch.full((n, n, n), 1.0, dtype=torch.float64, device=s.device),
                               torch.zeros((3, n, n, n), dtype=torch.float64, device=s.device))
            t, _, k = timed_run(torch, lbm, s, steps, 3, wall=2)
            bp = bytes_per_node(19, storage)
            ach = N * bp / (k * 1e-3) / 1e9
            row[storage] = {"mlups": round(N * steps / (t * 1e-3) / 1e6, 1),
                            "kernel_mlups": round(N / (k * 1e-3) / 1e6, 1),
                            "achieved_gbs": round(ach, 1), "frac": round(ach / hbm, 4)}
            s.close()
            del s
            torch.cuda.empty_cache()
        res[f"{n}^3"] = row
    return res


def extensions_bench(torch, lbm, workloads, hbm, args):
    """Each extension of the core step on the sphere box in FP32 storage:
    throughput, the step's mean duration and its HBM roofline fraction
    (algorithmic bytes: populations, class byte, and the field distributions
    of the induced field)."""
    res = {}
    steps = max(args.steps // 4, 50)
    for name, (_, kernel, desc) in EXTENSIONS.items():
        c, m, phi = make_workload(workloads, name, "f32")
        s = lbm.Sim(c, m)
        if phi is not None:
            s.set_wall_distance(phi)
        s.rest()
        N = c["nx"] * c["ny"] * c["nz"]
        t, _, k = timed_run(torch, lbm, s, steps, args.warmup)
        bp = bytes_per_node(19, "f32", induced=bool(c.get("induced")))
        ach = N * bp / (k * 1e-3) / 1e9
        res[name] = {"workload": desc, "kernel": kernel.replace(",S", ",StoreF32"), "steps": steps,
                     "mlups": round(N * steps / (t * 1e-3) / 1e6, 1), "step_ms": round(k, 5),
                     "kernel_mlups": round(N / (k * 1e-3) / 1e6, 1), "bytes_per_node": bp,
                     "achieved_gbs": round(ach, 1), "frac": round(ach / hbm, 4)}
        s.close()
        del s
        torch.cuda.empty_cache()
    return res


def adjoint_case(torch, lbm, adjoint, c, m, T, hbm):
    """Forward (with checkpoints), backward (with recomputation) and the
    reverse-step kernel alone, on one configuration."""
    s = lbm.Sim(c, m)
    prob = adjoint.DragProblem(s, T, 1)
    theta = list(c["g"]) + [0.0, 0.0, 0.0]
    prob.forward(theta)
    prob.backward()                      # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    prob.forward(theta)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    g = prob.backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    N = c["nx"] * c["ny"] * c["nz"]
    Q = c["lattice"]
    st = s.stream
    cs = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(cs)
    phi_n, cur = None, 0
    for i in range(T):
        lbm.lbm_adjoint_step(s.ctx, prob.ckpt[0], phi_n, prob.phi[cur], 1, prob.d, 1.0 / T, st)
        phi_n, cur = prob.phi[cur], 1 - cur
    e1.record(cs)
    torch.cuda.synchronize()
    ka = e0.elapsed_time(e1) / T
    s.close()
    bpn = 3 * Q * 4 + 1           # FP32 state, phi_{t+1} and phi_t per node, plus the class byte
    gbs = N * bpn / (ka * 1e-3) / 1e9
    return {"adjoint_kernel_mlups": round(N / (ka * 1e-3) / 1e6, 1),
            "adjoint_kernel_gbs": round(gbs, 1), "adjoint_kernel_frac": round(gbs / hbm, 4),
            "bytes_per_node": bpn,
            "backward_mlups_with_recompute": round(N * T / (t2 - t1) / 1e6, 1),
            "forward_mlups": round(N * T / (t1 - t0) / 1e6, 1), "grad": [float(x) for x in g]}


def adjoint_bench(torch, lbm, workloads, hbm):
    from paper_2512_12213_gb300 import adjoint
    out = {}
    c, m = workloads.cylinder(storage="f32")
    T = 2000
    out["cylinder_2d"] = dict(workload=f"D2Q9 cylinder r=20 in 512x256, T={T} (sqrt(T) checkpoints), FP32",
                              **adjoint_case(torch, lbm, adjoint, c, m, T, hbm))
    c, m = workloads.sphere_small(storage="f32")
    T = 2000
    out["sphere_3d"] = dict(workload=f"D3Q19 sphere r=10 in 128^3, T={T} (sqrt(T) checkpoints), FP32",
                            **adjoint_case(torch, lbm, adjoint, c, m, T, hbm))
    return out


def e2e_bench(torch, lbm, workloads, args):
    """Through the C ABI with host buffers: the initial canonical state is
    copied from pinned host memory, every step's drag is copied to pinned host
    memory (asynchronously, by the library, on a second stream beside the
    next step), and the final state is copied back to the host."""
    c, m = workloads.sphere(storage="f16s")
    c = dict(c, rounding="stochastic", seed=2024)
    s = lbm.Sim(c, m)
    N = c["nx"] * c["ny"] * c["nz"]
    s.rest()
    f_host = torch.empty((19, N), dtype=torch.float32, pin_memory=True)
    lbm.lbm_export_f(s.ctx, f_host, 1, 1, s.stream)
    steps = args.steps
    drag = torch.zeros((steps, 3), dtype=torch.float64, pin_memory=True)
    st = s.stream
    cs = torch.cuda.current_stream()
    side = torch.cuda.Stream(device=cs.device)
    for i in range(args.warmup):
        lbm.lbm_step(s.ctx, 1, st)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lbm.lbm_import_f(s.ctx, f_host, 1, 1, st)
    for i in range(steps):
        if i > 0:       # drag of step i-1 -> i, from the state step i reads
            side.wait_stream(cs)
            lbm.lbm_wall_force(s.ctx, 1, 0, 1.0, drag[i - 1], lbm.OUT_HOST_ASYNC, side.cuda_stream)
        lbm.lbm_step(s.ctx, 1, st)
        if i > 0:
            cs.wait_stream(side)
    lbm.lbm_wall_force(s.ctx, 1, 0, 1.0, drag[steps - 1], lbm.OUT_HOST_ASYNC, st)
    lbm.lbm_export_f(s.ctx, f_host, 1, 1, st)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    s.close()
    if not bool(torch.isfinite(drag).all()) or float(drag[-1, 0]) == 0.0:
        raise RuntimeError("end-to-end run returned no drag")
    state_bytes = 19 * N * 4
    return {"value": round(N * steps / (t1 - t0) / 1e6, 1), "unit": "MLUPS",
            "h2d_bytes_per_step": round(state_bytes / steps, 1),
            "d2h_bytes_per_step": round((state_bytes + 24 * steps) / steps, 1),
            "note": (f"per run: the canonical FP32 state ({state_bytes} B) in from pinned host memory and out "
                     f"again; per step: the 24-byte drag out (asynchronous, beside the next step); the byte "
                     f"counts above spread the state copies over the {steps} steps")}


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=20).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def _oracle_mlups(orc, ocfg, mask, f, budget_s, max_steps, omp):
    """Oracle steps within a time budget, as one call after a one-step probe
    (the per-call copy of the state is then paid once); (MLUPS, steps, s)."""
    t0 = time.perf_counter()
    f = orc.run(ocfg, mask, f, 1, omp=omp)
    probe = time.perf_counter() - t0
    n = int(max(1, min(max_steps, budget_s / max(probe, 1e-9))))
    t0 = time.perf_counter()
    orc.run(ocfg, mask, f, n, omp=omp)
    t = time.perf_counter() - t0
    return mask.size * n / t / 1e6, n, t


def cpu_baseline(budget_s=10.0):
    """The FP64 oracle as it stands on the host: its OpenMP timing build on
    every core (the parallel node loops of a step; results identical to the
    single-threaded parity build) and the parity build on one thread, each on
    a bounded sample of the headline workload (steps of the full
    256x128x128 sphere box); plus the two small 2-D configurations run in
    full: the Poiseuille channel (64x32, 10,000 steps) and the Hartmann channel
    (256x128, 50,000 steps, all cores, if it fits in about a minute and a half)."""
    cores = host_cores()
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    from oracle import oracle as orc
    from paper_2512_12213_gb300 import workloads
    orc.build()
    orc.build(omp=True)
    threads = orc.threads(omp=True)
    cfg, mask = workloads.sphere(storage="f64")
    ocfg = orc.make_cfg(**workloads.oracle_kwargs(cfg))
    nz, ny, nx = mask.shape
    f = orc.init(ocfg, mask, np.ones((nz, ny, nx)), np.zeros((3, nz, ny, nx)))
    v_all, s_all, t_all = _oracle_mlups(orc, ocfg, mask, f, budget_s, 200, True)
    v_one, s_one, t_one = _oracle_mlups(orc, ocfg, mask, f, budget_s, 20, False)
    out = {"value": round(v_all, 3), "unit": "MLUPS", "cores": threads, "kind": "oracle",
           "sample": f"{s_all} FP64 step(s) of the full 256x128x128 sphere box, OpenMP timing build on "
                     f"{threads} thread(s)",
           "cpu_model": cpu_model(), "host_cores": cores,
           "single_thread": {"value": round(v_one, 3), "unit": "MLUPS", "cores": 1,
                             "sample": f"{s_one} FP64 step(s) of the same box, parity build"}}
    # C1 in full, single thread
    c1, m1 = workloads.poiseuille(storage="f64")
    o1 = orc.make_cfg(**workloads.oracle_kwargs(c1))
    f1 = orc.init(o1, m1, np.ones(m1.shape), np.zeros((3,) + m1.shape))
    t0 = time.perf_counter()
    orc.run(o1, m1, f1, 10000)
    t1 = time.perf_counter() - t0
    out["poiseuille_64x32_10000_steps"] = {"seconds": round(t1, 3), "mlups": round(m1.size * 1e4 / t1 / 1e6, 3),
                                            "cores": 1}
    # C2 in full on every core, if the first 2,000 steps project it within ~90 s
    c2, m2 = workloads.hartmann(storage="f64")
    o2 = orc.make_cfg(**workloads.oracle_kwargs(c2))
    f2 = orc.init(o2, m2, np.ones(m2.shape), np.zeros((3,) + m2.shape))
    t0 = time.perf_counter()
    f2 = orc.run(o2, m2, f2, 2000, omp=True)
    tp = time.perf_counter() - t0
    if tp * 25 <= 90.0:
        orc.run(o2, m2, f2, 48000, omp=True)
        t2 = time.perf_counter() - t0
        out["hartmann_256x128_50000_steps"] = {"seconds": round(t2, 3),
                                                "mlups": round(m2.size * 5e4 / t2 / 1e6, 3), "cores": threads}
    else:
        out["hartmann_256x128_50000_steps"] = {"projected_seconds": round(tp * 25, 1),
                                                "mlups": round(m2.size * 2000 / tp / 1e6, 3), "cores": threads,
                                                "note": "first 2,000 steps timed; the full run would exceed 90 s"}
    return out


# ------------------------------------------------------ steady-state study
def _shift_mean_flow(torch, lbm, sim, fluid, dU):
    """Re-initialise the state at equilibrium with the node's density and
    flow velocity (from the library's residual and stress outputs) plus dU
    along x at the fluid nodes: a new initial condition for the same
    dynamics, which moves the slow mean-flow mode toward its steady value
    (the steady state reached afterwards does not depend on it)."""
    v = sim.velocity_buffer()
    sim.residual(v)
    rho = sim.stress(lbm.S2)[2].double()
    v[0] += dU * fluid
    sim.init_equilibrium(rho, v)


def _aitken(u0, u1, u2):
    """Limit of a geometric sequence from three equally spaced samples."""
    d1, d2 = u1 - u0, u2 - u1
    if d1 == 0.0 or not (0.0 < d2 / d1 < 0.98):
        return u2            # not a converging geometric approach: no correction
    return u2 - d2 * d2 / (d2 - d1)


def _series(torch, lbm, sim, mask, cfg, steps, every, vref=None):
    """Run `steps` steps sampling (step, F, U, C_d, Re, r) every `every` steps;
    r is the residual over `every` steps when vref is given."""
    out = []
    for i in range(steps // every):
        sim.step(every)
        r = sim.residual(vref)[2] if vref is not None else None
        out.append((every * (i + 1),) + sphere_measure(sim, mask, cfg) + (r,))
    return out


def _window(rows, frac=0.25):
    """Means of F, U, C_d, Re over the last `frac` of a series, and the
    spread (max - min) / mean of F there."""
    w = rows[-max(2, int(len(rows) * frac)):]
    F = [r[1] for r in w]
    return {"F": float(np.mean(F)), "U": float(np.mean([r[2] for r in w])), "cd": float(np.mean([r[3] for r in w])),
            "re": float(np.mean([r[4] for r in w])), "F_spread": float((max(F) - min(F)) / abs(np.mean(F)))}


def steady_study(torch, lbm, workloads, budget_f64=300_000):
    """The sphere (256x128x128, r = 12) at Re 20 and Re 100 run toward steady
    state, FP64 first, then every reduced storage from the FP64 state.

    FP64 is slow on GB300 (its arithmetic, not HBM, limits it), so the FP64
    run starts from an FP32 run: a uniform stream at the target speed, two
    mean-flow corrections (Aitken extrapolation of the mean velocity over
    three equally spaced samples), then FP32 until its residual stops
    falling; the FP32 state is exported in FP64, imported into the FP64
    context and run with one more correction until the residual over 100
    steps, r = sum |v(t) - v(t-100)| / sum |v(t)|, is below 1e-9 or the step
    budget is spent.  At steady state the momentum-exchange drag equals the
    body force on the fluid (the steady form of Eq. 32), which F / (g m)
    checks.  Each reduced storage then starts from the FP64 state and runs
    400,000 steps (Re 20) or 300,000 (Re 100); its drag, U and C_d are the
    means over the last quarter of the run, against the FP64 values."""
    out = {}
    for Re in (20, 100):
        res = {}
        t0 = time.perf_counter()
        c32, m, s32 = _sphere_sim(lbm, workloads, "f32", Re)
        nz, ny, nx = m.shape
        fluid = torch.from_numpy(m == 0).to(s32.device)
        U0 = workloads.SPHERE_RE[Re]["U0"]
        u = torch.zeros((3, nz, ny, nx), dtype=torch.float64, device=s32.device)
        u[0] = U0 * fluid
        s32.init_equilibrium(torch.ones((nz, ny, nx), dtype=torch.float64, device=s32.device), u)
        warm = []
        for cyc in range(3):
            rows = _series(torch, lbm, s32, m, c32, 60_000, 2_000)
            warm.extend(rows)
            Us = [r[2] for r in rows]
            U_inf = _aitken(np.mean(Us[6:10]), np.mean(Us[16:20]), np.mean(Us[26:30]))
            if cyc < 2:
                _shift_mean_flow(torch, lbm, s32, fluid, U_inf - Us[-1])
        v32 = s32.velocity_buffer()
        s32.residual(v32)
        tail32 = _series(torch, lbm, s32, m, c32, 100_000, 2_000, v32)
        res["f32_warmup"] = {"steps": 280_000, "last": tail32[-1][1:], "window": _window(tail32)}
        f = s32.export_f()
        s32.close()
        del s32, v32
        torch.cuda.empty_cache()
        # FP64 from the FP32 state
        c64, _, s64 = _sphere_sim(lbm, workloads, "f64", Re)
        s64.import_f(f)
        del f
        rows = _series(torch, lbm, s64, m, c64, 30_000, 1_000)
        Us = [r[2] for r in rows]
        _shift_mean_flow(torch, lbm, s64, fluid, _aitken(np.mean(Us[3:7]), np.mean(Us[13:17]),
                                                         np.mean(Us[23:27])) - Us[-1])
        v64 = s64.velocity_buffer()
        s64.residual(v64)
        series64, steps64, r = [], 30_000, None
        while steps64 < budget_f64:
            chunk = _series(torch, lbm, s64, m, c64, 10_000, 100, v64)
            series64.extend(chunk[-1:])
            steps64 += 10_000
            r = chunk[-1][5]
            if r is not None and r < 1e-9:
                break
        mass, _, rho_a = s64.balance()
        F, U, cd, re = sphere_measure(s64, m, c64)
        g = c64["g"][0]
        res["f64"] = {"steps": steps64, "r_100": r, "F": F, "U": U, "cd": cd, "re": re,
                      "F_over_body_force": F / (g * mass), "F_over_sum_rho_a": F / rho_a[0],
                      "series": [list(x) for x in series64], "window": _window(series64),
                      "seconds": round(time.perf_counter() - t0, 1)}
        ref = res["f64"]["window"] if (r is None or r >= 1e-9) else {"F": F, "U": U, "cd": cd, "re": re}
        f64state = s64.export_f()
        s64.close()
        del s64, v64
        torch.cuda.empty_cache()
        steps = 400_000 if Re == 20 else 300_000
        for key in PRECISIONS[1:]:
            c, _, s = _sphere_sim(lbm, workloads, key, Re)
            s.import_f(f64state)
            rows = _series(torch, lbm, s, m, c, steps, 5_000)
            w = _window(rows)
            mass, _, _ = s.balance()
            res[key] = {"steps": steps, "window": w, "F_over_body_force": w["F"] / (c["g"][0] * mass),
                        "drag_rel_err": abs(w["F"] / ref["F"] - 1), "U_rel_err": abs(w["U"] / ref["U"] - 1),
                        "cd_rel_err": abs(w["cd"] / ref["cd"] - 1),
                        "series_U": [r[2] for r in rows[::8]]}
            s.close()
            del s
            torch.cuda.empty_cache()
        del f64state
        torch.cuda.empty_cache()
        res["reference"] = "f64 final state" if (r is not None and r < 1e-9) else "f64 last-quarter means"
        out[f"re{Re}"] = res
    return out


def run_study(args):
    import torch
    torch.cuda.set_device(0)
    from paper_2512_12213_gb300 import build, lbm, workloads
    build.build()
    lbm.load()
    clocks = Clocks(0)
    clocks.start()
    clocks.active = True
    t0 = time.perf_counter()
    res = steady_study(torch, lbm, workloads)
    clocks.active = False
    clocks.stop()
    res["seconds"] = round(time.perf_counter() - t0, 1)
    res["clocks"] = clocks.summary()
    res["command"] = "python bench.py --study steady"
    line = json.dumps(res, default=float)
    print(line, flush=True)
    if args.study_out:
        os.makedirs(os.path.dirname(os.path.abspath(args.study_out)), exist_ok=True)
        with open(args.study_out, "w") as fh:
            fh.write(line + "\n")


# --------------------------------------------------------- reference arm
def run_reference(args):
    """The FP64 CPU oracle as it stands on the headline workload's metric, on
    the host's cores (its OpenMP timing build; the per-node arithmetic of the
    parity build): each step is one oracle step on a z-slab of the sphere box
    (periodic), sized so the whole run stays within a few minutes."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    cores = host_cores()
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    from oracle import oracle as orc
    from paper_2512_12213_gb300 import workloads
    orc.build(omp=True)
    threads = orc.threads(omp=True)
    cfg, mask = workloads.sphere(storage="f64")
    total_steps = args.steps + args.warmup

    def slab(nzs):
        m = mask[64 - nzs // 2: 64 - nzs // 2 + nzs].copy()
        c = dict(cfg, nz=nzs)
        oc = orc.make_cfg(**workloads.oracle_kwargs(c))
        f = orc.init(oc, m, np.ones(m.shape), np.zeros((3,) + m.shape))
        return oc, m, f
    # pick the slab thickness from an 8-layer probe: ~120 s for the whole run
    oc, m, f = slab(8)
    t0 = time.perf_counter()
    f = orc.run(oc, m, f, 2, omp=True)
    per_layer = (time.perf_counter() - t0) / 2 / 8
    nzs = int(max(1, min(128, 120.0 / max(total_steps * per_layer, 1e-9))))
    oc, m, f = slab(nzs)
    f = orc.run(oc, m, f, args.warmup, omp=True)
    t0 = time.perf_counter()
    f = orc.run(oc, m, f, args.steps, omp=True)
    t = time.perf_counter() - t0
    N = m.size
    value = N * args.steps / t / 1e6
    sample = (f"each step: one FP64 oracle step on a 256x128x{nzs} z-slab through the sphere (periodic), "
              f"OpenMP timing build on {threads} thread(s)")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "MLUPS", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * t / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_nodes": N},
            "cpu_baseline": {"value": round(value, 3), "unit": "MLUPS", "cores": threads, "kind": "oracle",
                             "sample": sample, "cpu_model": cpu_model()},
            "e2e": {"value": round(value, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.study:
        run_study(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
