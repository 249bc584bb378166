"""Serving: the request server admits systems of uneven sizes by device-memory
footprint, steps the resident ones together and retires them; every request
must get exactly the result it gets when run alone, whatever it was mixed
with, and the admission ledger must stay inside the budget."""
import time

import numpy as np
import pytest

from paper_1309_7859_gb300 import inputs
from paper_1309_7859_gb300.inputs import EpsSpec, System

pytestmark = pytest.mark.gpu

TH = (1.0, 1.0)


def requests(count=8, seed=11):
    rng = np.random.default_rng(seed)
    out = []
    for r in range(count):
        N = int(rng.choice([8, 12, 16, 20, 24]))
        mesh = (N, N, int(rng.choice([N, N // 2 + 4])))
        box = tuple(float(n) for n in mesh)
        n = int(rng.integers(1, 40)) * 2
        vals = inputs.smooth_random_vertices(np.random.default_rng(seed * 100 + r), mesh, 2.0)
        out.append(System(name=f"req{r}", mesh=mesh, box=box, eps=EpsSpec("vertices", 0, (), vals),
                          c_light=1.0, dt=0.005, precision="fp32",
                          x=inputs.uniform_positions(rng, n, box), q=inputs.neutral_charges(rng, n),
                          m=np.ones(n), v=inputs.thermal_velocities(rng, n),
                          # long enough (8-20 rounds of 8 steps) that admissions
                          # finishing on the worker threads overlap running requests
                          steps=int(rng.integers(64, 160)), thermostat=TH, seed=500 + r))
    return out


def alone(sysc):
    from paper_1309_7859_gb300.memd import Memd
    g = Memd(sysc.mesh, sysc.box, sysc.eps, c_light=sysc.c_light, dt=sysc.dt, precision="fp32",
             seed=sysc.seed, field_kernel="ldg")
    g.init_field(sysc.x, sysc.q, sysc.m, sysc.v)
    g.step(sysc.steps, thermostat=TH)
    x, v, img = g.particles()
    f = g.forces()
    e = g.energy()
    g.close()
    return x, v, img, f, e


def check_same(res, ref):
    x, v, img, f, e = res
    xr, vr, ir, fr, er = ref
    assert np.array_equal(x, xr) and np.array_equal(v, vr) and np.array_equal(img, ir)
    assert np.array_equal(f, fr)
    for k in ("kinetic", "electric", "magnetic", "total", "P0", "P1", "P2"):
        assert e[k] == er[k], k
    assert e["step"] == er["step"]


def test_server_results_match_alone_with_queuing():
    from paper_1309_7859_gb300.memd import Server
    reqs = requests()
    srv = Server(precision="fp32", budget_bytes=64 << 20, max_slots=3, quantum=8, thermostat=TH)
    ids = [srv.submit(s) for s in reqs]
    seen_active = 0
    for _ in range(500):
        a, q, d = srv.pump()
        seen_active = max(seen_active, a)
        assert srv.used_bytes() <= 64 << 20
        assert a <= 3
        if d == len(reqs):
            break
        if seen_active < 2:
            # a quantum of these small systems is shorter than a request's
            # setup on the admission threads: give them time to finish one
            time.sleep(0.005)
    assert d == len(reqs) and seen_active >= 2
    for s, rid in zip(reqs, ids):
        assert srv.status(rid) == 2
        check_same(srv.result(rid), alone(s))
    srv.close()


def test_server_continuous_arrivals_and_oversize():
    from paper_1309_7859_gb300.memd import MemdError, Server
    reqs = requests(6, seed=12)
    srv = Server(precision="fp32", budget_bytes=256 << 20, max_slots=16, quantum=5, thermostat=TH)
    ids = [srv.submit(s) for s in reqs[:3]]
    srv.pump()
    srv.pump()
    ids += [srv.submit(s) for s in reqs[3:]]          # arrive while the first run
    big = requests(1, seed=13)[0]
    big.mesh, big.box = (96, 96, 96), (96.0, 96.0, 96.0)
    big.eps = EpsSpec("const", 0, (2.0,))
    big_id = srv.submit(big)                           # larger than the budget
    for _ in range(500):
        a, q, d = srv.pump()
        if d == len(reqs) + 1:
            break
    assert srv.status(big_id) == 3
    with pytest.raises(MemdError):
        srv.result(big_id)
    for s, rid in zip(reqs, ids):
        check_same(srv.result(rid), alone(s))
        srv.release(rid)
    srv.close()


def test_serve_driver_records_latency():
    from paper_1309_7859_gb300.memd import Server, serve
    reqs = requests(5, seed=14)
    srv = Server(precision="fp32", budget_bytes=1 << 30, max_slots=8, quantum=10, thermostat=TH)
    arrivals = [0.0, 0.0, 0.05, 0.1, 0.1]
    rec = serve(srv, reqs, arrivals)
    assert len(rec) == 5
    for r in rec:
        assert r["done"] is not None and r["latency"] > 0
    srv.close()


def test_served_stream_sample_matches_alone():
    # requests drawn from the bench's served stream itself (meshes 16-96,
    # 100-50000 charges, smooth random eps), run through the server with the
    # bench's options and arrivals while others run, each against its solo run
    # (step counts shortened to keep the solo runs quick)
    from paper_1309_7859_gb300.memd import Server, serve
    reqs = inputs.served_stream(count=10, smin=40, smax=120)
    srv = Server(precision="fp32", budget_bytes=8 << 30, max_slots=128, quantum=50,
                 thermostat=TH)
    rng = np.random.default_rng(4)
    arrivals = np.cumsum(rng.exponential(1.0 / 40.0, size=len(reqs))).tolist()
    rec = serve(srv, reqs, arrivals)
    assert len(rec) == len(reqs)
    for s, r in zip(reqs, rec):
        check_same(srv.result(r["id"]), alone(s))
    srv.close()
