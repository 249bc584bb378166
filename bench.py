"""Benchmark of the MEMD hot path on GB300.

A step is one MEMD time step of the whole hot path (half kick, plaquette
update, drift with charge transfer, link update, transfer application,
dipole sum, force gather with corrections and Langevin force, half kick).
The default workload is the batched one: 64 independent replicas (meshes
from {16,24,32,48}^3, 200-8000 charges, random dielectric slabs, FP32 fields)
stepped together; a step advances every replica by one time step.  Their
fields (177 MB) exceed L2 (129 MB), so no flush is needed between steps.
Single-system workloads (--workload slab-32, salt-64, ...) flush L2 (a 256 MiB
write) before every timed step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...   (the FP64 CPU oracle on the same workload)

Under torchrun (N > 1) every rank runs its own batch (seed + rank, weak
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


def is_batch(name):
    return name.startswith("batch-")


def batch_systems(name, rank=0):
    from paper_1309_7859_gb300 import inputs
    count = int(name.split("-")[1])
    return inputs.batch_replicas(seed=1003 + 7919 * rank, count=count)


def batch_name(count):
    return (f"batch-{count} replicas (meshes {{16,24,32,48}}^3, 200-8000 charges, "
            f"random slabs, FP32)")


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
def host_cpu():
    """Core count and CPU model of the host the oracle runs on."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return {"nproc": os.cpu_count(), "model": model}


def oracle_system(sysc):
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
    return o


class OracleBatchModel:
    """The FP64 oracle on a bounded sample of a batch: the first replica of
    each mesh size, created and initialised untimed, then stepped one step at
    a time (timed).  A linear cost model t = a V + b n (sites, charges) is fitted
    to the samples' mean step times (non-negative least squares) and summed
    over every replica of the batch: the extrapolated single-core time of one
    batch step."""

    def __init__(self, systems):
        self.systems = systems
        self.samples = []
        seen = set()
        for s in systems:
            if s.mesh[0] in seen:
                continue
            seen.add(s.mesh[0])
            self.samples.append((s, oracle_system(s)))
        self.times = [[] for _ in self.samples]

    def step(self, k=1):
        for i, (s, o) in enumerate(self.samples):
            for _ in range(k):
                t0 = time.perf_counter()
                o.step(1, thermostat=s.thermostat)
                self.times[i].append(time.perf_counter() - t0)

    def batch_step_seconds(self):
        from scipy.optimize import nnls
        A = np.array([[s.sites, s.n] for s, _ in self.samples], dtype=np.float64)
        t = np.array([np.mean(ts) for ts in self.times])
        scale = A.max(axis=0)
        coef, _ = nnls(A / scale, t)
        coef = coef / scale
        per = [coef[0] * s.sites + coef[1] * s.n for s in self.systems]
        return float(np.sum(per)), coef, t

    def describe(self):
        steps = len(self.times[0]) if self.times else 0
        names = ", ".join(s.name for s, _ in self.samples)
        return (f"extrapolated: {steps} timed steps of each of {len(self.samples)} sample "
                f"replicas ({names}; FP64 oracle, single thread, untimed create and init); "
                f"cost per step fitted as a*sites + b*charges and summed over all "
                f"{len(self.systems)} replicas")


def oracle_batch_baseline(systems, steps=10):
    m = OracleBatchModel(systems)
    m.step(steps)
    t, coef, tm = m.batch_step_seconds()
    sites = sum(s.sites for s in systems)
    parts = sum(s.n for s in systems)
    cpu = host_cpu()
    v = 3 * sites / t
    return {"value": v, "unit": "link-updates/s", "cores": 1, "kind": "oracle",
            "sample": m.describe(), "particle_steps_per_s": parts / t,
            "ms_per_batch_step": t * 1e3,
            "fit_s_per_site": float(coef[0]), "fit_s_per_charge": float(coef[1]),
            "sample_ms_per_step": [float(x * 1e3) for x in tm],
            "host_cpu": cpu["model"], "host_nproc": cpu["nproc"],
            "all_cores_extrapolated": {"value": v * (cpu["nproc"] or 1),
                                       "note": "single-core rate x nproc (independent "
                                               "replicas, one per core; not measured)"}}


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


def run_reference_batch(args):
    """The oracle on the batched workload: its sample replicas (one per mesh
    size) created and initialised untimed, W warm-up steps each, then K timed
    steps each; the batch step time extrapolated by the fitted cost model."""
    systems = batch_systems(args.workload)
    m = OracleBatchModel(systems)
    for (s, o) in m.samples:
        o.step(args.warmup, thermostat=s.thermostat)
    m.step(args.steps)
    t, coef, tm = m.batch_step_seconds()
    sites = sum(s.sites for s in systems)
    parts = sum(s.n for s in systems)
    v = 3 * sites / t
    cpu = host_cpu()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "link-updates/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": batch_name(len(systems)), "replicas": len(systems),
                       "sites": sites, "charges": parts, "fields": "fp64 (oracle)"},
            "particle_steps_per_s": parts / t,
            "cpu_baseline": {"value": v, "unit": "link-updates/s", "cores": 1, "kind": "oracle",
                             "sample": m.describe(), "host_cpu": cpu["model"],
                             "host_nproc": cpu["nproc"],
                             "sample_ms_per_step": [float(x * 1e3) for x in tm]},
            "e2e": {"value": v, "unit": "link-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_reference(args, world, rank):
    """The oracle on this workload: one untimed create + init, W warm-up steps,
    then K steps timed one by one on the host cores."""
    if rank != 0:
        return 0
    if is_batch(args.workload):
        return run_reference_batch(args)
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
# Algorithmic bytes of the particle kernels per charge (FP32 fields; each word
# counted once, the cell's links at their minimum): deposition 96 B of state
# read (x, v, Ft, h, img, q), 84 B written (x, v, img, move record) and 12
# transfer words added (8 B each); application 24 B of move record and 12
# links' transfer word (read and cleared), ledger word and D (read and
# written); gather 84 B read (x, q, v, m, h, sig), 72 B written (F, Ft, v) and
# D and 1/eps of 12 links.
def particle_bytes(esz):
    return {"deposit": 96 + 84 + 12 * 8,
            "apply": 24 + 12 * (8 + 8 + 8 + 8 + 2 * esz),
            "gather": 84 + 72 + 12 * 2 * esz}


def clock_preroll(step_fn, sync, seconds=1.0, max_steps=20000):
    """Untimed steps for about `seconds` so that the nvidia-smi sampler (200 ms
    period) sees the GPU under this load just before the timed steps."""
    t0 = time.perf_counter()
    k = 1
    done = 0
    while time.perf_counter() - t0 < seconds and done < max_steps:
        step_fn(k)
        sync()
        done += k
        k = min(2 * k, 1024)
    return done


def batch_line(args, world, rank, local):
    """The headline: the batched replicas, every replica advanced one step per
    step, device time of exactly K steps between a barrier and a synchronise
    on both sides, max over ranks."""
    import torch
    from paper_1309_7859_gb300.memd import Batch, Memd

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    systems = batch_systems(args.workload, rank)
    t0 = time.perf_counter()
    members = []
    # --batch-rows-nt N: members fix the row kernel at N threads a CTA, which
    # the batch then takes untimed (for captures whose own timing would skew
    # the choice)
    fixed = dict(field_kernel="rows", field_shape=(0, 0, 0, args.batch_rows_nt)) \
        if args.batch_rows_nt else dict(field_kernel="ldg")
    for s in systems:
        g = Memd(s.mesh, s.box, s.eps, c_light=s.c_light, dt=s.dt, precision=s.precision,
                 seed=s.seed, stream=stream, time_kernels=False, apply_mode=args.apply,
                 **fixed)
        g.init_field(s.x, s.q, s.m, s.v)
        members.append(g)
    setup_s = time.perf_counter() - t0
    b = Batch(members, field_kernel=args.batch_kernel)
    th = systems[0].thermostat
    sites = sum(s.sites for s in systems)
    parts = sum(s.n for s in systems)
    links = 3 * sites
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    with torch.cuda.stream(stream):
        b.step(args.warmup, thermostat=th)
        b.synchronize()
        with ClockSampler(local) as clk:
            pre = clock_preroll(lambda k: b.step(k, thermostat=th), b.synchronize)
            barrier(world)
            torch.cuda.synchronize()
            ev[0].record(stream)
            b.step(args.steps, thermostat=th)
            ev[1].record(stream)
            torch.cuda.synchronize()
            barrier(world)
    tot_ms = allmax(ev[0].elapsed_time(ev[1]), world, dev)
    ks0 = b.kernel_stats()
    esz = 4 if systems[0].precision == "fp32" else 8
    pb = particle_bytes(esz)

    def instrumented():
        """Kernel durations inside the step: the same batch stepped again with
        an event pair around each of its launches."""
        b.set_timing(True)
        tsteps = max(20, min(args.steps, 200))
        with torch.cuda.stream(stream):
            b.step(3, thermostat=th)
            b.synchronize()
            b.kernel_stats()  # reset
            b.step(tsteps, thermostat=th)
            b.synchronize()
        k = b.kernel_stats()
        b.set_timing(False)
        n = max(1, k.field_launches)
        if k.single:
            # one launch a step: its bytes are the field pass and every
            # charge's particle work
            return k, {k.field_kernel: (k.field_bytes + sum(pb.values()) * parts,
                                        k.field_ms / n)}
        return k, {k.field_kernel: (k.field_bytes, k.field_ms / n),
                   "k_deposit_batch": (pb["deposit"] * parts, k.phase_ms[0] / n),
                   "k_apply_batch": (pb["apply"] * parts, k.phase_ms[1] / n),
                   "k_gather_batch": (pb["gather"] * parts, k.phase_ms[2] / n)}

    ks, kern = instrumented()
    graph_kern = None
    if ks.single:
        # the same batch as a graph of four kernels, for the breakdown
        b.set_engine("graph")
        gks, graph_kern = instrumented()
        b.set_engine("auto")
    else:
        gks = ks
    nl = max(1, gks.field_launches)
    inst_ms = sum(v[1] for v in kern.values())
    dom = max(kern, key=lambda k: kern[k][1])
    dbytes, dms = kern[dom]

    def table(kk):
        tot = sum(v[1] for v in kk.values())
        return {k: {"ms_per_launch": v[1], "share": v[1] / tot, "bytes_per_launch": v[0],
                    "GBps": v[0] / (v[1] * 1e-3) / 1e9 if v[1] > 0 else None}
                for k, v in kk.items()}
    # end to end through the C ABI: one page-locked block for all replicas,
    # each step copies every replica's positions, image counters and velocities
    # in and their state and forces out, with one synchronisation
    io = b.io_buffers()
    b.step_io(0, thermostat=th, load=False)
    e2e_steps = max(1, min(args.steps, 1000))
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        b.step_io(1, thermostat=th, load=True)
    e2e_s = allmax(time.perf_counter() - t0, world, dev)
    assert np.all(np.isfinite(io["f"]))
    h2d = parts * (24 + 24 + 12)
    d2h = parts * (24 + 24 + 12 + 24) + 4 * len(systems)
    exact = all(g.energy()["gauss_exact"] == 1.0 for g in members)
    b.close()
    for g in members:
        g.close()
    hbm, peak_kind = peaks()
    ach = dbytes / (dms * 1e-3) / 1e9
    field_ach = gks.field_bytes / (gks.field_ms / nl * 1e-3) / 1e9
    out = None
    if rank == 0:
        traffic = None
        prof = os.path.join(ROOT, "profiles", "traffic.json")
        if os.path.exists(prof):
            try:
                traffic = json.load(open(prof)).get(dom.split("<")[0] + "@" + args.workload)
            except Exception:
                traffic = None
        out = {
            "metric": METRIC, "value": world * links * args.steps / (tot_ms * 1e-3),
            "unit": "link-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if esz == 4 else "f64", "data": "synthetic",
            "config": {"workload": batch_name(len(systems)), "replicas": len(systems),
                       "sites": sites, "charges": parts, "fields": systems[0].precision,
                       "dt": systems[0].dt,
                       "thermostat": "langevin gamma=1 kT=1" if th else "none",
                       "l2": f"inputs larger than L2: fields {ks.field_bytes / 1e6:.0f} MB a "
                             "step (L2 129 MB), no flush",
                       "parallelism": f"replicas x{world}" if world > 1 else "one batch",
                       "clock_window": f"{pre} untimed steps (~1 s) just before the timed "
                                       "steps, sampled with them"},
            "particle_steps_per_s": world * parts * args.steps / (tot_ms * 1e-3),
            "roofline": {"bound": "hbm", "kernel": dom,
                         "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                         "peak_kind": peak_kind, "traffic": traffic,
                         "bytes_per_launch": dbytes, "ms_per_launch": dms,
                         "note": ("the whole step is one launch: bytes are the field pass "
                                  "(60 B a site) and every charge's particle work "
                                  f"({sum(pb.values())} B a charge); duration from a CUDA-event "
                                  "pair around the launch in an instrumented run")
                         if ks.single else
                                 "dominant kernel of the step by CUDA-event time in an "
                                 "instrumented run of the same batch (event pair around "
                                 "each launch)"},
            "engine": "single launch" if ks.single else "graph of four kernels",
            "kernels": table(kern),
            "graph_kernels": table(graph_kern) if graph_kern else None,
            "field_roofline": {"kernel": gks.field_kernel, "achieved": field_ach, "peak": hbm,
                               "frac": field_ach / hbm, "bytes_per_launch": gks.field_bytes,
                               "ms_per_launch": gks.field_ms / nl,
                               "note": "the batch's field kernel in the graph of four "
                                       "kernels (event pair around it)"},
            "launches_per_step": ks0.launches_per_step,
            "cpu_baseline": None,
            "e2e": {"value": world * links * e2e_steps / e2e_s, "unit": "link-updates/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "api": "memd_batch_step_io: one copy in (every replica's positions, "
                           "images, velocities) beside the field update, one batch step, "
                           "positions and images copied out beside the transfer "
                           "application and gather, velocities, forces and error words "
                           "after it, one sync"},
            "clocks": clk.summary(),
            "gpu_launches": int(ks0.launches_per_step * args.steps),
            "setup_s": setup_s,
            "gauss_exact": bool(exact),
        }
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = oracle_batch_baseline(systems, steps=args.cpu_steps)
    return out


def run_memd(args, world, rank, local):
    if is_batch(args.workload):
        out = batch_line(args, world, rank, local)
        extras = ("slab32", "large", "salt", "validation", "serve", "precision")
    else:
        out = single_line(args, world, rank, local, args.workload)
        extras = ("large", "salt", "validation", "batch", "serve", "precision")
    if rank != 0 or out is None:
        return out
    import torch
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    if "slab32" in extras and args.slab32:
        out["slab32"] = single_line(args, 1, 0, local, "slab-32", steps=args.single_steps)
    if "large" in extras and args.large > 0:
        out["large_mesh"] = large_mesh(args.large, dev, stream, args)
    if "salt" in extras and args.salt:
        out["salt"] = stepped_systems(("salt-64",), dev, stream, args)["salt-64"]
    if "validation" in extras and args.validation:
        out["validation"] = validation_systems(dev, stream, args)
    if "batch" in extras and args.batch > 0:
        out["batched"] = batched(args.batch, dev, args)
    if "serve" in extras and args.serve > 0:
        out["served"] = served(args.serve, args)
    if "precision" in extras and not args.no_cpu_baseline:
        out["precision_report"] = precision_report(workload("slab-32"))
    return out


def single_line(args, world, rank, local, name, steps=None):
    """One system stepped alone (L2 flushed before every timed step)."""
    import torch
    from paper_1309_7859_gb300.memd import Memd

    steps = steps or args.steps
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    sysc = workload(name, rank)
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
               for _ in range(steps)]
        barrier(world)
        torch.cuda.synchronize()
        with ClockSampler(local) as clk:
            for i in range(steps):
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
        field_ms_per_launch = sum(step_ms) / steps
    else:
        field_ms_per_launch = field_kernel_ms(sysc, args, dev, stream, flush)
    e = g.energy()

    # end to end through the C ABI with the library's page-locked I/O block,
    # copies inside: each step loads positions, images and velocities from
    # host memory and reads state and forces back
    n = sysc.n
    io = g.io_buffers()
    g.step_io(0, thermostat=th, load=False)   # the present state into the buffers
    e2e_steps = max(1, min(steps, 1000))
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
    value = world * links * steps / (tot_ms * 1e-3)
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
            "steps": steps, "warmup": args.warmup, "ms_per_step": tot_ms / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if sysc.precision == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": sysc.name, "mesh": list(sysc.mesh), "charges": sysc.n,
                       "fields": sysc.precision, "dt": sysc.dt,
                       "thermostat": "langevin gamma=1 kT=1" if th else "none",
                       "l2": "flushed (256 MiB write) before every timed step",
                       "parallelism": f"replicas x{world}" if world > 1 else "single system"},
            "particle_steps_per_s": world * n * steps / (tot_ms * 1e-3),
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
            "gpu_launches": int(ks.launches_per_step * steps),
            "gauss_exact": bool(e["gauss_exact"]),
        }
    g.close()
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
    ap.add_argument("--workload", default="batch-64",
                    help="batch-<count> (the default line: 64 replicas), or one system: "
                         "slab-32, plain-8, salt-64, bigslab-<N>, colloid-64, cloud-wall-32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="oracle time budget of a single system's cpu_baseline")
    ap.add_argument("--cpu-steps", type=int, default=10,
                    help="timed oracle steps of each sample replica of a batch's cpu_baseline")
    ap.add_argument("--slab32", type=int, default=1,
                    help="1: beside a batch line, also the single 32^3 slab system (slab32)")
    ap.add_argument("--single-steps", type=int, default=2000,
                    help="timed steps of the slab32 object")
    ap.add_argument("--field-kernel", default="auto", choices=["auto", "ldg", "tma", "site"])
    ap.add_argument("--step-engine", default="auto", choices=["auto", "graph", "single"])
    ap.add_argument("--apply", default="auto", choices=["auto", "sparse", "dense"],
                    help="how graph steps and batches apply the charge transfers")
    ap.add_argument("--batch", type=int, default=64,
                    help="beside a single-system line: replicas of the extra batched "
                         "measurement (0: skip)")
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
    ap.add_argument("--batch-rows-nt", type=int, default=0, choices=[0, 256, 512],
                    help="fix the batch's row kernel at this many threads a CTA (0: timed)")
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
