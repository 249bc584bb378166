"""Batched replicas: many independent systems stepped by one graph of four
launches must give, for every member, exactly what that member gives when
stepped alone with the same field kernel, and alone must match the oracle
(checked in test_gpu_parity)."""
import numpy as np
import pytest

from paper_1309_7859_gb300 import inputs
from paper_1309_7859_gb300.inputs import EpsSpec

pytestmark = pytest.mark.gpu

SPECS = [((16, 16, 16), 200, EpsSpec("tanh", 2, (41.0, 39.0, 8.0, 3.0, 1.5))),
         ((24, 24, 24), 600, EpsSpec("sin", 0, (60.0, -20.0, 0.0))),
         ((20, 12, 28), 150, EpsSpec("const", 0, (3.0,))),
         ((33, 9, 7), 40, EpsSpec("tanh", 1, (20.0, 15.0, 2.0, 2.0, 1.0))),
         ((8, 8, 8), 16, EpsSpec("const", 0, (1.0,))),
         ((48, 16, 16), 0, EpsSpec("tanh", 0, (41.0, 39.0, 24.0, 8.0, 1.5)))]


def systems(precision):
    out = []
    for i, (mesh, n, eps) in enumerate(SPECS):
        rng = np.random.default_rng(100 + i)
        box = tuple(float(N) for N in mesh)
        q = inputs.neutral_charges(rng, n)
        x = inputs.uniform_positions(rng, n, box)
        v = inputs.thermal_velocities(rng, n)
        out.append(dict(mesh=mesh, box=box, eps=eps, q=q, x=x, v=v, seed=7 + i,
                        precision=precision))
    return out


def make(s, stream=None, apply_mode="auto"):
    from paper_1309_7859_gb300.memd import Memd
    g = Memd(s["mesh"], s["box"], s["eps"], c_light=1.0, dt=0.005, precision=s["precision"],
             seed=s["seed"], field_kernel="ldg", stream=stream, apply_mode=apply_mode)
    g.init_field(s["x"], s["q"], None, s["v"])
    return g


def state(g):
    D, B, Lg = g.fields()
    x, v, img = g.particles()
    f = g.forces() if g.n else np.zeros((0, 3))
    e = g.energy()
    return D, B, Lg, x, v, img, f, (e["P0"], e["P1"], e["P2"], e["step"])


def assert_same(a, b):
    for u, w in zip(a[:7], b[:7]):
        assert np.array_equal(u, w)
    assert a[7] == b[7]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_members_match_alone(precision):
    import torch
    from paper_1309_7859_gb300.memd import Batch
    sys_ = systems(precision)
    stream = torch.cuda.Stream()
    members = [make(s, stream) for s in sys_]
    alone = [make(s) for s in sys_]
    batch = Batch(members)
    batch.step(4)                              # NVE
    batch.step(6, thermostat=(1.0, 1.0))       # then Langevin
    batch.synchronize()
    for g in alone:
        g.step(4)
        g.step(6, thermostat=(1.0, 1.0))
    for gm, ga in zip(members, alone):
        assert_same(state(gm), state(ga))
        assert gm.energy()["gauss_exact"] == 1.0


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_apply_modes_match(precision):
    # a batch applies its transfers per charge or by a dense pass over
    # (replica, chunk) pairs, following member 0's mode; the members end
    # identical either way (one member has an odd word count over two chunks)
    import torch
    from paper_1309_7859_gb300.memd import Batch
    sys_ = systems(precision)
    res = []
    for mode in ("sparse", "dense"):
        stream = torch.cuda.Stream()
        members = [make(s, stream, apply_mode=mode) for s in sys_]
        batch = Batch(members)
        batch.step(3)
        batch.step(7, thermostat=(1.0, 1.0))
        batch.synchronize()
        res.append([state(g) for g in members])
        for g in members:
            assert g.energy()["gauss_exact"] == 1.0
    for a, b in zip(res[0], res[1]):
        assert_same(a, b)


def test_batch_follows_members_stepped_alone():
    # a member stepped on its own between batch steps flips its buffers; the
    # batch notices and keeps every member consistent
    import torch
    from paper_1309_7859_gb300.memd import Batch
    sys_ = systems("fp32")[:3]
    stream = torch.cuda.Stream()
    members = [make(s, stream) for s in sys_]
    alone = [make(s) for s in sys_]
    batch = Batch(members)
    batch.step(3, thermostat=(1.0, 1.0))
    members[1].step(1, thermostat=(1.0, 1.0))
    batch.step(2, thermostat=(1.0, 1.0))
    batch.synchronize()
    for i, ga in enumerate(alone):
        ga.step(6 if i == 1 else 5, thermostat=(1.0, 1.0))
    for gm, ga in zip(members, alone):
        assert_same(state(gm), state(ga))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_row_kernel_members_match_alone(precision):
    # the row kernel (whole rows of 16-byte vectors, persistent balanced grid)
    # does the field arithmetic of the site kernels term for term
    import torch
    from paper_1309_7859_gb300.memd import Batch
    sys_ = [s for s in systems(precision) if s["mesh"][0] % 4 == 0]
    stream = torch.cuda.Stream()
    members = [make(s, stream) for s in sys_]
    alone = [make(s) for s in sys_]
    batch = Batch(members, field_kernel="rows")
    batch.set_engine("graph")                  # the row kernel of the four-kernel step
    batch.step(3)
    batch.step(5, thermostat=(1.0, 1.0))
    batch.synchronize()
    assert batch.kernel_stats().field_kernel.startswith("k_rows_batch")
    for g in alone:
        g.step(3)
        g.step(5, thermostat=(1.0, 1.0))
    for gm, ga in zip(members, alone):
        assert_same(state(gm), state(ga))
        assert gm.energy()["gauss_exact"] == 1.0


@pytest.mark.parametrize("nt", [256, 512])
def test_members_fixing_the_row_width_fix_the_batch(nt):
    # members created with the row kernel at one fixed width: the batch takes
    # that width untimed, and its members still match the members alone
    import torch
    from paper_1309_7859_gb300.memd import Batch, Memd
    sys_ = [s for s in systems("fp32") if s["mesh"][0] % 4 == 0]
    stream = torch.cuda.Stream()

    def fixed(s, stream=None):
        g = Memd(s["mesh"], s["box"], s["eps"], c_light=1.0, dt=0.005,
                 precision=s["precision"], seed=s["seed"], field_kernel="rows",
                 field_shape=(0, 0, 0, nt), stream=stream)
        g.init_field(s["x"], s["q"], None, s["v"])
        return g
    members = [fixed(s, stream) for s in sys_]
    alone = [make(s) for s in sys_]
    batch = Batch(members)
    batch.step(4, thermostat=(1.0, 1.0))
    batch.synchronize()
    assert batch.kernel_stats().field_kernel == f"k_rows_batch<nt={nt}>"
    for g in alone:
        g.step(4, thermostat=(1.0, 1.0))
    for gm, ga in zip(members, alone):
        assert_same(state(gm), state(ga))
    batch.close()


@pytest.mark.parametrize("nsteps,wide", [(1, False), (2, False), (1, True)])
def test_batch_step_io_equals_the_separate_calls(nsteps, wide):
    # every member's state through the batch's host block (one step a call:
    # the copies run beside the step; two steps: around it), against the
    # same edits made member by member and batch steps, with the quad and
    # the one-thread-per-charge particle kernels (more than 16384 charges);
    # the members include one without charges
    import torch
    from paper_1309_7859_gb300.memd import Batch
    sys_ = systems("fp32")
    if wide:
        counts = [4000, 6000, 3002, 2000, 1500, 0]
        assert sum(counts) > 16384
        for i, (s, n) in enumerate(zip(sys_, counts)):
            rng = np.random.default_rng(300 + i)
            s["q"] = inputs.neutral_charges(rng, n)
            s["x"] = inputs.uniform_positions(rng, n, s["box"])
            s["v"] = inputs.thermal_velocities(rng, n)
        # one particle without charge: an odd total, so the image counters
        # end off an 8-byte boundary
        s0 = sys_[0]
        s0["q"] = np.concatenate([s0["q"], [0]]).astype(np.int32)
        s0["x"] = np.concatenate([s0["x"], [[3.3, 4.4, 5.5]]])
        s0["v"] = np.concatenate([s0["v"], [[0.1, -0.2, 0.3]]])
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    A = [make(s, sa) for s in sys_]
    Bm = [make(s, sb) for s in sys_]
    ba, bb = Batch(A), Batch(Bm)
    io = ba.io_buffers()
    off = io["offsets"]
    ba.step_io(0, load=False)
    th = (1.0, 1.0)
    for it in range(4):
        io["vel"] *= 0.999                  # the host edits the state between calls
        ba.step_io(nsteps, thermostat=th, load=True)
        for g in Bm:
            x, v, img = g.particles()
            g.set_particles(x, v * 0.999, img)
        bb.step(nsteps, thermostat=th)
        bb.synchronize()
        for r, g in enumerate(Bm):
            x, v, img = g.particles()
            sl = slice(off[r], off[r + 1])
            assert np.array_equal(io["pos"][sl], x) and np.array_equal(io["vel"][sl], v)
            assert np.array_equal(io["img"][sl], img)
            if g.n:
                assert np.array_equal(io["f"][sl], g.forces())
    for ga, gb in zip(A, Bm):
        assert_same(state(ga), state(gb))
        assert ga.energy()["gauss_exact"] == 1.0
    ba.close()
    bb.close()


def test_row_kernel_falls_back_to_site_tiles():
    # a member whose x extent is not a multiple of 4 sites keeps the batch on
    # site tiles, with the same results
    import torch
    from paper_1309_7859_gb300.memd import Batch
    sys_ = systems("fp32")[2:5]       # includes the 33-wide mesh
    assert any(s["mesh"][0] % 4 for s in sys_)
    stream = torch.cuda.Stream()
    members = [make(s, stream) for s in sys_]
    alone = [make(s) for s in sys_]
    batch = Batch(members, field_kernel="rows")
    batch.step(4, thermostat=(1.0, 1.0))
    batch.synchronize()
    assert batch.kernel_stats().field_kernel.startswith("k_fused_site_batch")
    for g in alone:
        g.step(4, thermostat=(1.0, 1.0))
    for gm, ga in zip(members, alone):
        assert_same(state(gm), state(ga))


def test_batch_of_64_at_bench_size_matches_alone_and_the_oracle():
    # the bench's batched workload itself (64 replicas, meshes 16-48^3,
    # 200-8000 charges, FP32) in the launch configuration it times (the
    # autotuned field kernel): every member keeps Gauss's law exact, sampled
    # members are bit identical to their solo runs, and one small member's
    # forces are recomputed by the oracle from its batched state
    import torch
    from oracle import oracle as O
    from paper_1309_7859_gb300.memd import Batch, Memd
    from tests.test_gpu_parity import oracle_eps, rel
    systems = inputs.batch_replicas(count=64)
    stream = torch.cuda.Stream()

    def mk(s, st=None):
        g = Memd(s.mesh, s.box, s.eps, c_light=s.c_light, dt=s.dt, precision=s.precision,
                 seed=s.seed, stream=st, field_kernel="ldg")
        g.init_field(s.x, s.q, s.m, s.v)
        return g
    members = [mk(s, stream) for s in systems]
    batch = Batch(members)
    batch.step(4, thermostat=systems[0].thermostat)
    batch.synchronize()
    for g in members:
        assert g.energy()["gauss_exact"] == 1.0
    for i in (0, 17, 40, 63):
        ga = mk(systems[i])
        ga.step(4, thermostat=systems[i].thermostat)
        assert_same(state(members[i]), state(ga))
        ga.close()
    i = min(range(64), key=lambda k: systems[k].sites)
    s = systems[i]
    D, B, Lg = members[i].fields()
    x, v, img = members[i].particles()
    o = O.OracleSystem(s.mesh, s.box, eps=oracle_eps(s.eps), c_light=s.c_light, dt=s.dt,
                       seed=s.seed)
    o.set_particles(x, s.q, s.m, v, img)
    o.field("D")[...] = D
    o.field("Lg")[...] = Lg
    o.gather()
    assert rel(members[i].forces(), o.particles("F")) < 1e-5
    batch.close()


# ------------------------------------------------ single-launch batch step
ROW_SPECS = [((16, 16, 16), 200, EpsSpec("tanh", 2, (41.0, 39.0, 8.0, 3.0, 1.5))),
             ((24, 13, 11), 300, EpsSpec("sin", 0, (60.0, -20.0, 0.0))),   # ragged tiles
             ((48, 16, 16), 0, EpsSpec("tanh", 0, (41.0, 39.0, 24.0, 8.0, 1.5))),
             ((32, 32, 20), 900, EpsSpec("const", 0, (3.0,))),
             ((8, 8, 8), 16, EpsSpec("const", 0, (1.0,))),
             ((20, 22, 18), 70, EpsSpec("tanh", 1, (20.0, 15.0, 2.0, 2.0, 1.0)))]


def row_systems(precision):
    out = []
    for i, (mesh, n, eps) in enumerate(ROW_SPECS):
        rng = np.random.default_rng(300 + i)
        box = tuple(float(N) for N in mesh)
        out.append(dict(mesh=mesh, box=box, eps=eps, q=inputs.neutral_charges(rng, n),
                        x=inputs.uniform_positions(rng, n, box),
                        v=inputs.thermal_velocities(rng, n), seed=40 + i, precision=precision))
    return out


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_single_launch_step_matches_graph_and_alone(precision):
    # the whole step of every member in one cooperative launch (work queues,
    # per-member readiness counts) against the graph of four kernels and the
    # members stepped alone: bit identical, over many launches (the queue
    # bases and launch count carry from one launch to the next)
    import torch
    from paper_1309_7859_gb300.memd import Batch
    sys_ = row_systems(precision)
    res = {}
    for engine in ("single", "graph"):
        stream = torch.cuda.Stream()
        members = [make(s, stream) for s in sys_]
        batch = Batch(members)
        batch.set_engine(engine)
        batch.step(4)
        batch.step(9, thermostat=(1.0, 1.0))
        batch.synchronize()
        ks = batch.kernel_stats()
        assert ks.single == (engine == "single")
        assert ks.launches_per_step == (1 if engine == "single" else 4)
        res[engine] = [state(g) for g in members]
        for g in members:
            assert g.energy()["gauss_exact"] == 1.0
        batch.close()
    for s, a, b in zip(sys_, res["single"], res["graph"]):
        assert_same(a, b)
        ga = make(s)
        ga.step(4)
        ga.step(9, thermostat=(1.0, 1.0))
        assert_same(a, state(ga))


def test_single_launch_scheduling_variants_agree():
    # every CTA starting with deposition, every CTA starting with field work,
    # and field segments of two planes: the schedule changes, the results do not
    import torch
    from paper_1309_7859_gb300.memd import Batch
    sys_ = row_systems("fp32")
    res = []
    for field_ctas, planes in ((-1, 0), (0, 0), (100000, 0), (-1, 2)):
        stream = torch.cuda.Stream()
        members = [make(s, stream) for s in sys_]
        batch = Batch(members)
        batch.set_engine("single", field_ctas=field_ctas, item_planes=planes)
        batch.step(6, thermostat=(1.0, 1.0))
        batch.synchronize()
        res.append([state(g) for g in members])
        batch.close()
    for other in res[1:]:
        for a, b in zip(res[0], other):
            assert_same(a, b)


def test_engines_switch_mid_run():
    # single launch, then the graph, then the single launch again (and a
    # member stepped alone in between): the members end as when stepped alone
    import torch
    from paper_1309_7859_gb300.memd import Batch
    sys_ = row_systems("fp32")
    stream = torch.cuda.Stream()
    members = [make(s, stream) for s in sys_]
    batch = Batch(members)
    batch.set_engine("single")
    batch.step(3, thermostat=(1.0, 1.0))
    batch.set_engine("graph")
    batch.step(2, thermostat=(1.0, 1.0))
    members[3].step(1, thermostat=(1.0, 1.0))
    batch.set_engine("single")
    batch.step(4, thermostat=(1.0, 1.0))
    batch.set_timing(True)                     # an event pair around the launch
    batch.step(2, thermostat=(1.0, 1.0))
    batch.synchronize()
    assert batch.kernel_stats().field_launches == 2
    for i, s in enumerate(sys_):
        ga = make(s)
        ga.step(12 if i == 3 else 11, thermostat=(1.0, 1.0))
        assert_same(state(members[i]), state(ga))


def test_single_launch_refused_for_site_tile_members():
    # a member whose x extent is not a multiple of 4 sites cannot run in row
    # tiles: the single launch is refused, the automatic choice is the graph
    import torch
    from paper_1309_7859_gb300.memd import Batch, MemdError
    sys_ = systems("fp32")[2:5]
    stream = torch.cuda.Stream()
    members = [make(s, stream) for s in sys_]
    batch = Batch(members)
    assert not batch.kernel_stats().single
    with pytest.raises(MemdError):
        batch.set_engine("single")
    batch.set_engine("auto")
    batch.step(2, thermostat=(1.0, 1.0))
    batch.synchronize()
    for s, g in zip(sys_, members):
        ga = make(s)
        ga.step(2, thermostat=(1.0, 1.0))
        assert_same(state(g), state(ga))
