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
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "lattice link-updates/s + particle-steps/s (HBM % of peak); served p50/p99"
L2_FLUSH_BYTES = 256 << 20
L2_BYTES = 129e6


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
    if name.startswith("colloid-"):
        return inputs.colloid(N=int(name.split("-")[1]), seed=1006 + 7919 * rank)
    if name.startswith("cloud-wall-"):
        return inputs.cloud_wall(N=int(name.split("-")[2]), seed=1007 + 7919 * rank)
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
        self.path = os.path.join(tempfile.gettempdir(), f"memd_clocks_{os.getpid()}_{gpu_index}.csv")

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
    # the timed steps run as a user runs them: no timing events inside the
    # step graph (each event node adds a few microseconds to a step)
    g = Memd(sysc.mesh, sysc.box, sysc.eps, c_light=sysc.c_light, dt=sysc.dt,
             precision=sysc.precision, seed=sysc.seed, time_kernels=False, stream=stream,
             field_kernel=args.field_kernel, step_engine=args.step_engine,
             apply_mode=args.apply)
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
    if ks.single:
        # one launch a step: the per-step event time bounds the kernel's
        # duration from above (it includes the launch)
        field_ms_per_launch = sum(step_ms) / args.steps
    else:
        field_ms_per_launch = field_kernel_ms(sysc, args, dev, stream, flush)
    e = g.energy()

    # end to end through the C ABI with the library's page-locked I/O block,
    # copies inside: each step loads positions, images and velocities from
    # host memory and reads state and forces back
    n = sysc.n
    io = g.io_buffers()
    g.step_io(0, thermostat=th, load=False)   # the present state into the buffers
    e2e_steps = max(1, min(args.steps, 1000))
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        g.step_io(1, thermostat=th, load=True)
    e2e_s = allmax(time.perf_counter() - t0, world, dev)
    assert np.all(np.isfinite(io["f"]))
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
            "roofline": {"bound": "hbm",
                         "kernel": ks.field_kernel if ks.single
                         else ks.field_kernel + " (B then D update, one pass)",
                         "note": ("the whole step in one launch: latency bound at this size, "
                                  "bytes are the step's field and particle state; duration "
                                  "= the step's CUDA-event time (launch included)")
                         if ks.single else "field update of the step; duration from CUDA "
                                           "events around it in an instrumented step graph",
                         "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "peak_kind": peak_kind, "traffic": traffic,
                         "bytes_per_launch": ks.field_bytes,
                         "ms_per_launch": field_ms_per_launch},
            "cpu_baseline": cpu,
            "e2e": {"value": world * links * e2e_steps / e2e_s, "unit": "link-updates/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "api": "memd_step_io: one copy in (positions, images, velocities), one step, one copy out (state and forces), one sync"},
            "clocks": clk.summary(),
            "gpu_launches": int(ks.launches_per_step * args.steps),
            "gauss_exact": bool(e["gauss_exact"]),
        }
    g.close()
    if rank == 0 and out is not None and args.large > 0:
        out["large_mesh"] = large_mesh(args.large, dev, stream, args)
    if rank == 0 and out is not None and args.salt:
        out["salt"] = stepped_systems(("salt-64",), dev, stream, args)["salt-64"]
    if rank == 0 and out is not None and args.validation:
        out["validation"] = validation_systems(dev, stream, args)
    if rank == 0 and out is not None and args.batch > 0:
        out["batched"] = batched(args.batch, dev, args)
    if rank == 0 and out is not None and args.serve > 0:
        out["served"] = served(args.serve, args)
    if rank == 0 and out is not None and not args.no_cpu_baseline:
        out["precision_report"] = precision_report(sysc)
    return out


def field_kernel_ms(sysc, args, dev, stream, flush, steps=None):
    """Average duration of the field kernel inside the step (CUDA events
    around it in the step graph) on a second, instrumented context of the
    same system, stepped with the same L2 flush before every step."""
    import torch
    from paper_1309_7859_gb300.memd import Memd
    g = Memd(sysc.mesh, sysc.box, sysc.eps, c_light=sysc.c_light, dt=sysc.dt,
             precision=sysc.precision, seed=sysc.seed, time_kernels=True, stream=stream,
             field_kernel=args.field_kernel, step_engine=args.step_engine,
             apply_mode=args.apply)
    g.init_field(sysc.x, sysc.q, sysc.m, sysc.v)
    th = sysc.thermostat
    steps = steps or max(10, min(args.steps, 500))
    with torch.cuda.stream(stream):
        g.step(args.warmup, thermostat=th)
        g.synchronize()
        g.reset_kernel_stats()
        for i in range(steps):
            if flush is not None:
                flush.fill_(float(i))
            g.step(1, thermostat=th)
        g.synchronize()
    ks = g.kernel_stats()
    g.close()
    return ks.field_ms / max(1, ks.field_launches)


def precision_report(sysc):
    """Each observable's error of the FP32-field GPU path against the FP64
    oracle after 10 steps from the same state (relative RMS; energies and
    the dipole moment as relative differences)."""
    from oracle import oracle as O
    from paper_1309_7859_gb300.memd import Memd
    kinds = {"const": O.EPS_CONST, "links": O.EPS_LINKS, "vertices": O.EPS_VERTICES,
             "tanh": O.EPS_TANH, "sin": O.EPS_SIN}
    o = O.OracleSystem(sysc.mesh, sysc.box, eps=dict(kind=kinds[sysc.eps.kind], axis=sysc.eps.axis,
                                                     params=sysc.eps.params),
                       c_light=sysc.c_light, dt=sysc.dt, seed=sysc.seed)
    o.set_particles(sysc.x, sysc.q, sysc.m, sysc.v)
    o.init_field()
    g = Memd(sysc.mesh, sysc.box, sysc.eps, c_light=sysc.c_light, dt=sysc.dt, precision="fp32",
             seed=sysc.seed)
    g.init_field(sysc.x, sysc.q, sysc.m, sysc.v)
    g.set_fields(D=o.field("D"), B=o.field("B"), Lg=o.field("Lg"))
    g.set_particles(x=o.particles("x"), v=o.particles("v"), img=o.particles("img"))
    g.compute_forces()
    o.step(10, thermostat=sysc.thermostat)
    g.step(10, thermostat=sysc.thermostat)
    D, B, Lg = g.fields()
    x, v, img = g.particles()
    rel = lambda a, b: float(np.sqrt(np.sum((a - b) ** 2) / max(np.sum(b * b), 1e-300)))
    eg, eo = g.energy(), o.energy()
    rep = {"steps": 10, "workload": sysc.name, "D": rel(D, o.field("D")), "B": rel(B, o.field("B")),
           "forces": rel(g.forces(), o.particles("F")), "velocities": rel(v, o.particles("v")),
           "positions_max_abs": float(np.max(np.abs(x - o.particles("x")))),
           "ledger_mismatches": int(np.sum(Lg != o.field("Lg"))),
           "gauss_exact": bool(eg["gauss_exact"])}
    for k in ("electric", "magnetic", "kinetic", "total", "P0", "P1", "P2"):
        rep[k] = abs(eg[k] - eo[k]) / max(abs(eo[k]), 1e-300)
    g.close()
    return rep


def served(count, args):
    """A served stream: `count` requests (meshes 16-96, 100-50000 charges,
    smooth random eps, 200-5000 steps, FP32) with Poisson arrivals, admitted
    by device-memory footprint into a continuous batch; p50/p99 latency and
    aggregate throughput.  Beside it, the plain single-replica FP64 GPU path
    on the first requests (one at a time, short runs)."""
    import torch
    from paper_1309_7859_gb300 import inputs
    from paper_1309_7859_gb300.memd import Memd, Server, serve
    reqs = inputs.served_stream(count=count, smax=args.serve_max_steps)
    rng = np.random.default_rng(4242)
    arrivals = np.cumsum(rng.exponential(1.0 / args.serve_rate, size=count)).tolist()
    srv = Server(precision="fp32", budget_bytes=args.serve_budget << 30, max_slots=128,
                 quantum=50, thermostat=(1.0, 1.0), admission_workers=args.serve_workers)
    t0 = time.perf_counter()
    rec = serve(srv, reqs, arrivals)
    wall = time.perf_counter() - t0
    lat = np.array([r["latency"] for r in rec])
    links = sum(3 * r.sites * r.steps for r in reqs)
    parts = sum(r.n * r.steps for r in reqs)
    st = srv.stats()
    srv.close()
    # plain single-replica FP64 path, requests one at a time
    k, t_single, l_single = 0, 0.0, 0
    for r in reqs[:8]:
        steps = min(r.steps, 200)
        g = Memd(r.mesh, r.box, r.eps, c_light=r.c_light, dt=r.dt, precision="fp64", seed=r.seed)
        g.init_field(r.x, r.q, r.m, r.v)
        g.step(5, thermostat=(1.0, 1.0))
        g.synchronize()
        a = time.perf_counter()
        g.step(steps, thermostat=(1.0, 1.0))
        g.synchronize()
        t_single += time.perf_counter() - a
        l_single += 3 * r.sites * steps
        g.close()
        k += 1
    return {"requests": count, "arrival_rate_per_s": args.serve_rate,
            "budget_gib": args.serve_budget, "max_slots": 128, "quantum": 50,
            "max_steps": args.serve_max_steps, "wall_s": wall,
            "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)),
            "link_updates_per_s": links / wall, "particle_steps_per_s": parts / wall,
            "setup_s_summed": st["setup_s"], "admission_workers": args.serve_workers,
            "step_gpu_s": st["step_gpu_s"],
            "stepping_link_updates_per_s": links / max(st["step_gpu_s"], 1e-9),
            "mean_budget_use": st["budget_use_sum"] / max(1, st["rounds"]),
            "rounds": st["rounds"], "batch_rebuilds": st["rebuilds"],
            "single_fp64_link_updates_per_s": l_single / max(t_single, 1e-9),
            "single_fp64_sample": f"first {k} requests one at a time, up to 200 steps each, FP64 fields",
            "note": "wall time includes every request's setup (eps, Green's table, "
                    "eps_eff and initial solve; run by admission workers beside the "
                    "stepping) and the arrival gaps; stepping rate = link updates over "
                    "the device time of the batch steps"}


def batched(count, dev, args):
    """The batched-replica workload: `count` independent systems (meshes from
    {16,24,32,48}^3, 200-8000 charges, random slabs, FP32) stepped together,
    four launches per step for all of them."""
    import torch
    from paper_1309_7859_gb300 import inputs
    from paper_1309_7859_gb300.memd import Batch, Memd
    systems = inputs.batch_replicas(count=count)
    stream = torch.cuda.Stream(device=dev)
    t0 = time.perf_counter()
    members = []
    for i, s in enumerate(systems):
        g = Memd(s.mesh, s.box, s.eps, c_light=s.c_light, dt=s.dt, precision=s.precision,
                 seed=s.seed, stream=stream, time_kernels=False, field_kernel="ldg",
                 apply_mode=args.apply)
        g.init_field(s.x, s.q, s.m, s.v)
        members.append(g)
    setup_s = time.perf_counter() - t0
    b = Batch(members, field_kernel=args.batch_kernel)
    th = systems[0].thermostat
    steps = max(20, min(args.steps, 200))
    with torch.cuda.stream(stream):
        b.step(5, thermostat=th)
        b.synchronize()
        b.kernel_stats()  # reset
        ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        ev[0].record(stream)
        b.step(steps, thermostat=th)
        ev[1].record(stream)
        b.synchronize()
    ms = ev[0].elapsed_time(ev[1])
    # the field kernel's duration: the same batch (same kernel) with CUDA
    # events around its field update in the step graph
    b.set_timing(True)
    with torch.cuda.stream(stream):
        b.step(3, thermostat=th)
        b.synchronize()
        b.kernel_stats()  # reset
        b.step(steps, thermostat=th)
        b.synchronize()
    ks = b.kernel_stats()
    kernel = ks.field_kernel
    per = ks.field_ms / max(1, ks.field_launches)
    b.close()
    hbm, kind = peaks()
    ach = ks.field_bytes / (per * 1e-3) / 1e9
    sites = sum(s.sites for s in systems)
    parts = sum(s.n for s in systems)
    exact = all(g.energy()["gauss_exact"] == 1.0 for g in members)
    for g in members:
        g.close()
    return {"workload": f"batch-{count} replicas (meshes {{16,24,32,48}}^3, 200-8000 charges, "
                        f"random slabs, FP32)", "replicas": count, "sites": sites,
            "charges": parts, "steps": steps, "ms_per_step": ms / steps,
            "link_updates_per_s": 3 * sites * steps / (ms * 1e-3),
            "particle_steps_per_s": parts * steps / (ms * 1e-3),
            "launches_per_step": ks.launches_per_step, "setup_s": setup_s,
            "l2": f"fields {sites * 60 / 1e6:.0f} MB, larger than L2, no flush",
            "roofline": {"bound": "hbm", "kernel": kernel, "achieved": ach, "peak": hbm,
                         "unit": "GB/s", "frac": ach / hbm, "peak_kind": kind,
                         "bytes_per_launch": ks.field_bytes, "ms_per_launch": per},
            "gauss_exact": exact}


def large_mesh(N, dev, stream, args):
    """The same step on an N^3 system whose fields exceed L2 (no flush needed):
    shows the field stencil against HBM bandwidth."""
    import torch
    from paper_1309_7859_gb300.memd import Memd
    sysc = workload(f"bigslab-{N}")
    g = Memd(sysc.mesh, sysc.box, sysc.eps, c_light=sysc.c_light, dt=sysc.dt,
             precision=sysc.precision, seed=sysc.seed, time_kernels=False, stream=stream,
             field_kernel=args.field_kernel, step_engine=args.step_engine,
             apply_mode=args.apply)
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
    e = g.energy()
    g.close()
    per = field_kernel_ms(sysc, args, dev, stream, None, steps=steps)
    hbm, kind = peaks()
    ach = ks.field_bytes / (per * 1e-3) / 1e9
    links = 3 * sysc.sites
    return {"workload": sysc.name, "steps": steps, "ms_per_step": ms / steps,
            "link_updates_per_s": links * steps / (ms * 1e-3),
            "particle_steps_per_s": sysc.n * steps / (ms * 1e-3),
            "l2": f"fields ({ks.field_bytes / 1e9:.1f} GB a pass) larger than L2, no flush",
            "roofline": {"bound": "hbm", "kernel": ks.field_kernel, "achieved": ach, "peak": hbm,
                         "unit": "GB/s", "frac": ach / hbm, "peak_kind": kind,
                         "bytes_per_launch": ks.field_bytes, "ms_per_launch": per},
            "gauss_exact": bool(e["gauss_exact"])}


def validation_systems(dev, stream, args):
    """The paper's validation systems as synthetic workloads (our own
    parameters): the dielectric colloid in salt water and the cloud-wall
    system."""
    return stepped_systems(("colloid-64", "cloud-wall-32"), dev, stream, args)


def stepped_systems(names, dev, stream, args):
    """Single systems beside the default line, each stepped as that line is
    (L2 flushed before every step, CUDA events on the library's stream), up
    to 2000 steps; field-kernel duration from an instrumented context when
    the step is not one launch."""
    import torch
    from paper_1309_7859_gb300.memd import Memd
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    out = {}
    for name in names:
        sysc = workload(name)
        g = Memd(sysc.mesh, sysc.box, sysc.eps, c_light=sysc.c_light, dt=sysc.dt,
                 precision=sysc.precision, seed=sysc.seed, time_kernels=False, stream=stream,
                 field_kernel=args.field_kernel, step_engine=args.step_engine,
                 apply_mode=args.apply)
        g.init_field(sysc.x, sysc.q, sysc.m, sysc.v)
        th = sysc.thermostat
        steps = max(10, min(args.steps, 2000))
        x0 = g.particles()[0]
        with torch.cuda.stream(stream):
            g.step(args.warmup, thermostat=th)
            g.synchronize()
            g.reset_kernel_stats()
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(steps)]
            for i in range(steps):
                flush.fill_(float(i))
                evs[i][0].record(stream)
                g.step(1, thermostat=th)
                evs[i][1].record(stream)
            torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in evs)
        ks = g.kernel_stats()
        per = (ms / steps if ks.single else
               field_kernel_ms(sysc, args, dev, stream, flush, steps=min(steps, 500)))
        hbm, kind = peaks()
        ach = ks.field_bytes / (per * 1e-3) / 1e9
        e = g.energy()
        x1 = g.particles()[0]
        nh = sysc.extra.get("heavy", 0)
        drift = float(np.max(np.abs(x1[:nh] - x0[:nh]))) if nh else 0.0
        g.close()
        out[name] = {"workload": sysc.name, "steps": steps, "ms_per_step": ms / steps,
                     "link_updates_per_s": 3 * sysc.sites * steps / (ms * 1e-3),
                     "particle_steps_per_s": sysc.n * steps / (ms * 1e-3),
                     "eps": sysc.eps.kind, "engine": "single" if ks.single else "graph",
                     "roofline": {"bound": "hbm", "kernel": ks.field_kernel, "achieved": ach,
                                  "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                                  "peak_kind": kind, "bytes_per_launch": ks.field_bytes,
                                  "ms_per_launch": per,
                                  **({"note": f"fields of {ks.field_bytes / 1e6:.0f} MB a pass fit "
                                              "in L2 (129 MB): not an HBM-bound figure; the "
                                              "step is bound by its particle kernels"}
                                     if ks.field_bytes < L2_BYTES else {})},
                     "fixed_charges_max_move": drift if nh else None,
                     "dipole": [e["P0"], e["P1"], e["P2"]],
                     "gauss_exact": bool(e["gauss_exact"])}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="memd", choices=["memd", "reference"])
    ap.add_argument("--workload", default="slab-32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--field-kernel", default="auto", choices=["auto", "ldg", "tma", "site"])
    ap.add_argument("--step-engine", default="auto", choices=["auto", "graph", "single"])
    ap.add_argument("--apply", default="auto", choices=["auto", "sparse", "dense"],
                    help="how graph steps and batches apply the charge transfers")
    ap.add_argument("--batch", type=int, default=64,
                    help="replicas of the extra batched measurement (0: skip)")
    ap.add_argument("--serve", type=int, default=512,
                    help="requests of the extra served-stream measurement (0: skip)")
    ap.add_argument("--serve-rate", type=float, default=40.0)
    ap.add_argument("--serve-budget", type=int, default=8, help="GiB")
    ap.add_argument("--serve-max-steps", type=int, default=5000)
    ap.add_argument("--serve-workers", type=int, default=3,
                    help="admission threads of the server (request setup beside stepping)")
    ap.add_argument("--large", type=int, default=256,
                    help="edge of the extra larger-than-L2 system (0: skip)")
    ap.add_argument("--batch-kernel", default="auto", choices=["auto", "site", "rows"],
                    help="field kernel of the batched replicas (auto: timed choice)")
    ap.add_argument("--salt", type=int, default=1,
                    help="1: also step the 64^3 salt system (32768 charges, eps from salt density)")
    ap.add_argument("--validation", type=int, default=1,
                    help="1: also step the colloid and cloud-wall systems (0: skip)")
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
