"""Benchmark of the MEMD hot path on GB300.

A step is one MEMD time step of the whole hot path (half kick, plaquette
update, drift with charge transfer, link update, transfer application,
dipole sum, force gather with corrections and Langevin force, half kick) on
the workload's synthetic system.  The default workload is the 32^3 slab with
1000 charges and FP32 fields.  It fits in L2, so L2 is flushed (a 256 MiB
write) before every timed step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...   (the FP64 CPU oracle on the same workload)

Under torchrun (N > 1) every rank runs its own replica (seed + rank, weak
scaling, no collective on the data path); timings are max-reduced over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "lattice link-updates/s + particle-steps/s (HBM % of peak); served p50/p99"
L2_FLUSH_BYTES = 256 << 20


def workload(name, rank=0):
    from paper_1309_7859_gb300 import inputs
    if name == "slab-32":
        return inputs.slab_32(seed=1001 + 7919 * rank)
    if name == "plain-8":
        s = inputs.plain_8(seed=1000 + 7919 * rank)
        return s
    if name == "salt-64":
        return inputs.salt_64(seed=1002 + 7919 * rank)
    if name.startswith("bigslab-"):
        N = int(name.split("-")[1])
        return inputs.big_slab(N=N, seed=1005 + 7919 * rank)
    raise SystemExit(f"unknown workload {name}")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_rank{gpu_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
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
            self.fh.close()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        try:
            rows = [l.split(",") for l in open(self.path).read().strip().splitlines() if l.strip()]
        except Exception:
            return out
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except Exception:
                continue
            for nm, val in zip(names, r[5:9]):
                if "Active" in val and "Not" not in val:
                    reasons.add(nm)
        if sm:
            out.update(sm_mhz=statistics.median(sm), sm_max_mhz=max(mx), samples=len(sm))
        out["reasons"] = sorted(reasons)
        return out


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "memd" else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def allmax(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------------ oracle arm
def oracle_rate(sysc, budget_s, cores_note=1):
    """Time the FP64 CPU oracle on a bounded sample of steps of the workload."""
    from oracle import oracle as O
    kinds = {"const": O.EPS_CONST, "links": O.EPS_LINKS, "vertices": O.EPS_VERTICES,
             "tanh": O.EPS_TANH, "sin": O.EPS_SIN}
    e = dict(kind=kinds[sysc.eps.kind], axis=sysc.eps.axis, params=sysc.eps.params)
    if sysc.eps.values is not None:
        e["values"] = sysc.eps.values
    o = O.OracleSystem(sysc.mesh, sysc.box, eps=e, c_light=sysc.c_light, dt=sysc.dt,
                       seed=sysc.seed)
    o.set_particles(sysc.x, sysc.q, sysc.m, sysc.v)
    o.init_field()
    steps, t0 = 0, time.perf_counter()
    while True:
        o.step(1, thermostat=sysc.thermostat)
        steps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or steps >= sysc.steps:
            break
    links = 3 * sysc.sites
    return {"value": links * steps / el, "unit": "link-updates/s", "cores": 1,
            "kind": "oracle", "particle_steps_per_s": sysc.n * steps / el,
            "sample": f"{steps} steps of {sysc.name} (FP64 oracle, single thread, "
                      f"{el:.1f} s after an untimed init)"}


def run_reference(args, world, rank):
    """The oracle on this workload: one untimed create + init, W warm-up steps,
    then K steps timed one by one on the host cores."""
    if rank != 0:
        return 0
    from oracle import oracle as O
    sysc = workload(args.workload)
    kinds = {"const": O.EPS_CONST, "links": O.EPS_LINKS, "vertices": O.EPS_VERTICES,
             "tanh": O.EPS_TANH, "sin": O.EPS_SIN}
    e = dict(kind=kinds[sysc.eps.kind], axis=sysc.eps.axis, params=sysc.eps.params)
    if sysc.eps.values is not None:
        e["values"] = sysc.eps.values
    o = O.OracleSystem(sysc.mesh, sysc.box, eps=e, c_light=sysc.c_light, dt=sysc.dt,
                       seed=sysc.seed)
    o.set_particles(sysc.x, sysc.q, sysc.m, sysc.v)
    o.init_field()
    o.step(args.warmup, thermostat=sysc.thermostat)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(1, thermostat=sysc.thermostat)
    el = time.perf_counter() - t0
    links = 3 * sysc.sites
    v = links * args.steps / el
    sample = f"{args.steps} steps of {sysc.name} (FP64 oracle, single thread, untimed init)"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "link-updates/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": sysc.name, "mesh": list(sysc.mesh), "charges": sysc.n,
                       "fields": "fp64 (oracle)"},
            "particle_steps_per_s": sysc.n * args.steps / el,
            "cpu_baseline": {"value": v, "unit": "link-updates/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "link-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------- GPU arm
def run_memd(args, world, rank, local):
    import torch
    from paper_1309_7859_gb300.memd import Memd

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    sysc = workload(args.workload, rank)
    g = Memd(sysc.mesh, sysc.box, sysc.eps, c_light=sysc.c_light, dt=sysc.dt,
             precision=sysc.precision, seed=sysc.seed, time_kernels=True, stream=stream)
    g.init_field(sysc.x, sysc.q, sysc.m, sysc.v)
    th = sysc.thermostat
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    links = 3 * sysc.sites
    with torch.cuda.stream(stream):
        g.step(args.warmup, thermostat=th)
        g.synchronize()
        g.reset_kernel_stats()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        barrier(world)
        torch.cuda.synchronize()
        with ClockSampler(local) as clk:
            for i in range(args.steps):
                flush.fill_(float(i))           # evict the system from L2
                evs[i][0].record(stream)
                g.step(1, thermostat=th)
                evs[i][1].record(stream)
            torch.cuda.synchronize()
        barrier(world)
    step_ms = [a.elapsed_time(b) for a, b in evs]
    tot_ms = allmax(sum(step_ms), world, dev)
    ks = g.kernel_stats()
    field_ms_per_launch = ks.field_ms / max(1, ks.field_launches)
    e = g.energy()

    # end to end through the C ABI with pinned host buffers, copies inside
    n = sysc.n
    hx = torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
    hv = torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
    hi = torch.empty((n, 3), dtype=torch.int32, pin_memory=True).numpy()
    hf = torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
    g.get_particles_into(hx, hv, hi)
    e2e_steps = max(1, args.steps)
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        g.set_particles(hx, hv, hi)
        g.step(1, thermostat=th)
        g.get_particles_into(hx, hv, hi)
        g.forces(hf)
    e2e_s = allmax(time.perf_counter() - t0, world, dev)
    h2d = n * (24 + 24 + 12)
    d2h = n * (24 + 24 + 12 + 24)

    hbm, peak_kind = peaks()
    achieved = ks.field_bytes / (field_ms_per_launch * 1e-3) / 1e9
    value = world * links * args.steps / (tot_ms * 1e-3)
    out = None
    if rank == 0:
        traffic = None
        prof = os.path.join(ROOT, "profiles", "traffic.json")
        if os.path.exists(prof):
            try:
                traffic = json.load(open(prof)).get(sysc.name)
            except Exception:
                traffic = None
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cpu = oracle_rate(sysc, args.cpu_seconds)
        out = {
            "metric": METRIC, "value": value, "unit": "link-updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if sysc.precision == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": sysc.name, "mesh": list(sysc.mesh), "charges": sysc.n,
                       "fields": sysc.precision, "dt": sysc.dt,
                       "thermostat": "langevin gamma=1 kT=1" if th else "none",
                       "l2": "flushed (256 MiB write) before every timed step",
                       "parallelism": f"replicas x{world}" if world > 1 else "single system"},
            "particle_steps_per_s": world * n * args.steps / (tot_ms * 1e-3),
            "roofline": {"bound": "hbm", "kernel": "k_fused_curl (B then D update, one pass)",
                         "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "peak_kind": peak_kind, "traffic": traffic,
                         "bytes_per_launch": ks.field_bytes,
                         "ms_per_launch": field_ms_per_launch},
            "cpu_baseline": cpu,
            "e2e": {"value": world * links * e2e_steps / e2e_s, "unit": "link-updates/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "api": "memd_set_particles + memd_step(1) + memd_get_particles + memd_forces"},
            "clocks": clk.summary(),
            "gpu_launches": int(ks.launches_per_step * args.steps),
            "gauss_exact": bool(e["gauss_exact"]),
        }
    g.close()
    if rank == 0 and out is not None and args.large > 0:
        out["large_mesh"] = large_mesh(args.large, dev, stream, args)
    return out


def large_mesh(N, dev, stream, args):
    """The same step on an N^3 system whose fields exceed L2 (no flush needed):
    shows the field stencil against HBM bandwidth."""
    import torch
    from paper_1309_7859_gb300.memd import Memd
    sysc = workload(f"bigslab-{N}")
    g = Memd(sysc.mesh, sysc.box, sysc.eps, c_light=sysc.c_light, dt=sysc.dt,
             precision=sysc.precision, seed=sysc.seed, time_kernels=True, stream=stream)
    g.init_field(sysc.x, sysc.q, sysc.m, sysc.v)
    th = sysc.thermostat
    steps = max(10, min(args.steps, 50))
    with torch.cuda.stream(stream):
        g.step(3, thermostat=th)
        g.synchronize()
        g.reset_kernel_stats()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            g.step(1, thermostat=th)
        b.record(stream)
        torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    ks = g.kernel_stats()
    per = ks.field_ms / max(1, ks.field_launches)
    hbm, kind = peaks()
    ach = ks.field_bytes / (per * 1e-3) / 1e9
    e = g.energy()
    g.close()
    links = 3 * sysc.sites
    return {"workload": sysc.name, "steps": steps, "ms_per_step": ms / steps,
            "link_updates_per_s": links * steps / (ms * 1e-3),
            "particle_steps_per_s": sysc.n * steps / (ms * 1e-3),
            "l2": "fields (1 GB) larger than L2, no flush",
            "roofline": {"bound": "hbm", "kernel": "k_fused_curl", "achieved": ach, "peak": hbm,
                         "unit": "GB/s", "frac": ach / hbm, "peak_kind": kind,
                         "bytes_per_launch": ks.field_bytes, "ms_per_launch": per},
            "gauss_exact": bool(e["gauss_exact"])}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="memd", choices=["memd", "reference"])
    ap.add_argument("--workload", default="slab-32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--large", type=int, default=256,
                    help="edge of the extra larger-than-L2 system (0: skip)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        rc = run_reference(args, world, rank)
    else:
        out = run_memd(args, world, rank, local)
        if rank == 0 and out is not None:
            print(json.dumps(out), flush=True)
        rc = 0
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
