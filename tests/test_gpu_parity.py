"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle,
element by element on the same seeded inputs.

Tolerances (relative RMS over all elements unless stated):
  * integer work (ledger, image counters, cell indices): bit exact;
  * FP64 fields and forces over 10 steps from the same state: 1e-12;
  * FP32 fields and forces over 10 steps from the same state: 1e-5;
  * the relaxed initial field: 1e-9.  Both sides stop at a circulation
    residual of 1e-12 max|E|; the field error behind such a residual is up to
    the condition number of the plaquette operator (about N^2 times the eps
    contrast, 1e3-1e4 here) larger, so two independent solvers can differ by
    ~1e-9 and no less;
  * create-time 1/eps: 1e-15, Green's table: 1e-13 absolute, eps_eff^-1: 1e-10.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1309_7859_gb300 import inputs
from paper_1309_7859_gb300.inputs import EpsSpec, System
from tests import refs

pytestmark = pytest.mark.gpu

OKIND = {"const": O.EPS_CONST, "links": O.EPS_LINKS, "vertices": O.EPS_VERTICES,
         "tanh": O.EPS_TANH, "sin": O.EPS_SIN, "planes": O.EPS_PLANES,
         "sphere": O.EPS_SPHERE, "cut": O.EPS_CUT}


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.sqrt(np.sum(b * b))
    return float(np.sqrt(np.sum((a - b) ** 2)) / (den if den > 0 else 1.0))


def oracle_eps(e):
    d = dict(kind=OKIND[e.kind], axis=e.axis, params=e.params)
    if e.values is not None:
        d["values"] = e.values
    return d


# (step engine, field kernel) pairs: the graph of four kernels with each
# field kernel, and the single cooperative launch (its own field tiles)
ENGINES = [("graph", "ldg"), ("graph", "site"), ("graph", "tma"), ("graph", "rows"),
           ("single", "auto")]


def make_pair(sysc, self_mode=1, dipole_corr=1, precision=None, init=True, field_kernel="auto",
              step_engine="auto"):
    from paper_1309_7859_gb300.memd import Memd
    prec = precision or sysc.precision
    g = Memd(sysc.mesh, sysc.box, sysc.eps, c_light=sysc.c_light, dt=sysc.dt, precision=prec,
             self_mode=self_mode, dipole_corr=dipole_corr, seed=sysc.seed,
             field_kernel=field_kernel, step_engine=step_engine)
    o = O.OracleSystem(sysc.mesh, sysc.box, eps=oracle_eps(sysc.eps), c_light=sysc.c_light,
                       dt=sysc.dt, self_mode=self_mode, dipole_corr=dipole_corr, seed=sysc.seed)
    if init:
        o.set_particles(sysc.x, sysc.q, sysc.m, sysc.v)
        o.init_field()
        g.init_field(sysc.x, sysc.q, sysc.m, sysc.v)
    return g, o


def small_system(mesh, n, eps, precision="fp64", seed=7, dt=0.01, thermostat=(1.0, 1.0)):
    rng = np.random.default_rng(seed)
    box = tuple(float(N) for N in mesh)
    q = inputs.neutral_charges(rng, n)
    x = inputs.uniform_positions(rng, n, box)
    v = inputs.thermal_velocities(rng, n)
    return System(name="test", mesh=tuple(mesh), box=box, eps=eps, c_light=1.0, dt=dt,
                  precision=precision, x=x, q=q, m=np.ones(n), v=v, steps=10,
                  thermostat=thermostat, seed=seed)


SLAB = EpsSpec("tanh", 2, (41.0, 39.0, 6.0, 3.0, 1.5))
SINX = EpsSpec("sin", 0, (60.0, -20.0, 0.0))

# meshes spanning several 32 x 8 tiles with ragged tails, plus tiny ones
MESHES = [(8, 8, 8), (40, 20, 12), (33, 9, 7), (4, 4, 4), (2, 3, 2)]


# ------------------------------------------------------------ create time
@pytest.mark.parametrize("mesh", MESHES[:3])
@pytest.mark.parametrize("eps", [EpsSpec("const", 0, (2.5,)), SLAB, SINX, "vertices", "links"])
def test_setup_matches_oracle(mesh, eps):
    from paper_1309_7859_gb300.memd import Memd
    rng = np.random.default_rng(3)
    V = mesh[0] * mesh[1] * mesh[2]
    if eps == "vertices":
        eps = EpsSpec("vertices", 0, (), rng.uniform(2, 80, size=V))
    elif eps == "links":
        eps = EpsSpec("links", 0, (), rng.uniform(2, 80, size=3 * V))
    sysc = small_system(mesh, 0, eps)
    g, o = make_pair(sysc, init=False)
    ie, G, M = g.setup()
    assert rel(ie, o.field("ie")) < 1e-15
    assert np.max(np.abs(G - o.G)) < 1e-13
    assert np.max(np.abs(M - o.Minv)) < 1e-10 * np.max(np.abs(o.Minv))


# ------------------------------------------------------- initial solution
@pytest.mark.parametrize("mesh,n,eps", [((8, 8, 8), 16, EpsSpec("const", 0, (1.0,))),
                                        ((40, 20, 12), 200, SLAB),
                                        ((33, 9, 7), 50, SINX),
                                        ((4, 4, 4), 6, EpsSpec("const", 0, (3.0,))),
                                        ((2, 3, 2), 2, EpsSpec("const", 0, (1.0,))),
                                        # multigrid levels with odd extents (aggregation)
                                        ((36, 20, 10), 150, "vertices"),
                                        ((45, 12, 14), 100, SLAB)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_initial_solution_matches_oracle(mesh, n, eps, precision):
    if eps == "vertices":
        vals = inputs.smooth_random_vertices(np.random.default_rng(8), mesh)
        eps = EpsSpec("vertices", 0, (), vals)
    sysc = small_system(mesh, n, eps, precision=precision)
    g, o = make_pair(sysc)
    D, B, Lg = g.fields()
    assert np.array_equal(Lg, o.field("Lg"))
    assert rel(D, o.field("D")) < (1e-9 if precision == "fp64" else 1e-6)
    assert np.all(B == 0)
    x, v, img = g.particles()
    assert np.array_equal(x, o.particles("x")) and np.array_equal(img, o.particles("img"))
    assert rel(g.forces(), o.particles("F")) < (1e-8 if precision == "fp64" else 1e-5)
    e = g.energy()
    assert e["gauss_exact"] == 1.0


def test_non_neutral_background_matches_oracle():
    sysc = small_system((8, 8, 8), 2, EpsSpec("const", 0, (2.0,)))
    sysc.q = np.array([1, 2], dtype=np.int32)   # 3 e over 512 vertices: exact background
    g, o = make_pair(sysc)
    D, _, Lg = g.fields()
    assert np.array_equal(Lg, o.field("Lg"))
    assert rel(D, o.field("D")) < 1e-9


# ------------------------------------------------- 10 steps from one state
def load_oracle_state(g, o):
    g.set_fields(D=o.field("D"), B=o.field("B"), Lg=o.field("Lg"))
    g.set_particles(x=o.particles("x"), v=o.particles("v"), img=o.particles("img"))
    g.compute_forces()


def compare_state(g, o, tol, ledger_exact=True):
    D, B, Lg = g.fields()
    x, v, img = g.particles()
    if ledger_exact:
        assert np.array_equal(Lg, o.field("Lg"))
    assert np.array_equal(img, o.particles("img"))
    assert rel(D, o.field("D")) < tol
    assert rel(B, o.field("B")) < tol
    assert rel(g.forces(), o.particles("F")) < tol
    assert rel(v, o.particles("v")) < tol
    assert np.max(np.abs(x - o.particles("x"))) < 1e-9


@pytest.mark.parametrize("mesh,n,eps", [((8, 8, 8), 16, EpsSpec("const", 0, (1.0,))),
                                        ((40, 20, 12), 300, SLAB),
                                        ((33, 9, 7), 60, SINX)])
@pytest.mark.parametrize("self_mode", [O.SELF_GF, O.SELF_DIRECT, O.SELF_NONE])
@pytest.mark.parametrize("engine,field_kernel", ENGINES)
def test_ten_steps_fp64(mesh, n, eps, self_mode, engine, field_kernel):
    sysc = small_system(mesh, n, eps, dt=0.01)
    g, o = make_pair(sysc, self_mode=self_mode, field_kernel=field_kernel, step_engine=engine)
    load_oracle_state(g, o)
    assert rel(g.forces(), o.particles("F")) < 1e-12
    o.step(10, thermostat=(1.0, 1.0))
    g.step(10, thermostat=(1.0, 1.0))
    compare_state(g, o, 1e-12)
    eg, eo = g.energy(), o.energy()
    for k in ("kinetic", "electric", "magnetic", "self", "dipole", "total", "P0", "P1", "P2"):
        assert abs(eg[k] - eo[k]) <= 1e-11 * max(1.0, abs(eo[k])), k
    assert eg["gauss_exact"] == 1.0 and eo["gauss_exact"] == 1.0


@pytest.mark.parametrize("mesh,n,eps", [((8, 8, 8), 16, EpsSpec("const", 0, (1.0,))),
                                        ((40, 20, 12), 300, SLAB),
                                        ((72, 20, 6), 200, SINX),
                                        ((4, 6, 2), 8, EpsSpec("const", 0, (2.0,)))])
@pytest.mark.parametrize("engine,field_kernel", ENGINES)
def test_ten_steps_fp32(mesh, n, eps, engine, field_kernel):
    sysc = small_system(mesh, n, eps, precision="fp32", dt=0.005)
    g, o = make_pair(sysc, field_kernel=field_kernel, step_engine=engine)
    load_oracle_state(g, o)
    o.step(10, thermostat=(1.0, 1.0))
    g.step(10, thermostat=(1.0, 1.0))
    # FP32 forces move the FP64 positions by ~1e-12; a sub-cell step can then
    # round the other way, so the ledger is compared in the replay test and
    # checked here through the exact Gauss identity
    compare_state(g, o, 1e-5, ledger_exact=False)
    assert g.energy()["gauss_exact"] == 1.0


def test_nve_without_thermostat_fp64():
    sysc = small_system((8, 8, 8), 16, EpsSpec("const", 0, (1.0,)), dt=0.01)
    g, o = make_pair(sysc)
    load_oracle_state(g, o)
    o.step(10)
    g.step(10)
    compare_state(g, o, 1e-12)


# ------------------------------------------------------ prescribed moves
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_replay_moves_ledger_bit_exact(precision):
    rng = np.random.default_rng(17)
    sysc = small_system((40, 20, 12), 400, SLAB, precision=precision)
    g, o = make_pair(sysc)
    load_oracle_state(g, o)
    L = np.array(sysc.box)
    x = o.particles("x").copy()
    img = o.particles("img").copy()
    for it in range(12):
        step = rng.uniform(-0.97, 0.97, size=x.shape)
        if it % 3 == 0:
            step[:, it % 3] = rng.choice([-0.999, 0.999], size=len(x))
        un = x + img * L + step
        img = np.floor(un / L).astype(np.int32)
        x = un - img * L
        o.move(x, img)
        g.move(x, img)
        D, _, Lg = g.fields()
        assert np.array_equal(Lg, o.field("Lg"))
        xg, _, ig = g.particles()
        assert np.array_equal(xg, o.particles("x")) and np.array_equal(ig, o.particles("img"))
        assert rel(D, o.field("D")) < (1e-13 if precision == "fp64" else 1e-6)
    assert g.energy()["gauss_exact"] == 1.0


def test_cell_jump_is_reported():
    from paper_1309_7859_gb300.memd import MemdError
    sysc = small_system((8, 8, 8), 4, EpsSpec("const", 0, (1.0,)))
    g, o = make_pair(sysc)
    x, _, img = g.particles()
    x2 = x.copy()
    x2[0, 0] = (x2[0, 0] + 2.5) % 8.0
    with pytest.raises(MemdError):
        g.move(x2, img)
    xa, _, _ = g.particles()
    assert np.array_equal(xa[0], x[0])   # the offending charge did not move
    assert g.energy()["gauss_exact"] == 1.0


# ------------------------------------------------ full-size configurations
def test_plain_8_full_run_matches_oracle():
    # the 8^3 FP64 Langevin system, all 100 steps from the same state
    sysc = inputs.plain_8()
    g, o = make_pair(sysc)
    load_oracle_state(g, o)
    o.step(sysc.steps, thermostat=sysc.thermostat)
    g.step(sysc.steps, thermostat=sysc.thermostat)
    compare_state(g, o, 1e-10)


@pytest.mark.parametrize("engine,field_kernel", ENGINES)
def test_slab_32_full_size_matches_oracle(engine, field_kernel):
    # 32^3 slab, 1000 charges, FP32 fields: init on both sides, then 10 steps
    sysc = inputs.slab_32()
    g, o = make_pair(sysc, field_kernel=field_kernel, step_engine=engine)
    _, _, Lg = g.fields()
    assert np.array_equal(Lg, o.field("Lg"))
    load_oracle_state(g, o)
    o.step(10, thermostat=sysc.thermostat)
    g.step(10, thermostat=sysc.thermostat)
    assert g.kernel_stats().single == (engine == "single")   # the engine is chosen at the first step
    compare_state(g, o, 1e-5, ledger_exact=False)


def test_salt_64_full_size_sampled_forces():
    # 64^3, 32768 charges: the GPU runs init + 10 steps; the oracle recomputes
    # every force from the GPU's own state (fields, positions) and the
    # invariants are checked at full size
    from paper_1309_7859_gb300.memd import Memd
    sysc = inputs.salt_64()
    g = Memd(sysc.mesh, sysc.box, sysc.eps, c_light=sysc.c_light, dt=sysc.dt,
             precision="fp32", seed=sysc.seed)
    g.init_field(sysc.x, sysc.q, sysc.m, sysc.v)
    g.step(10, thermostat=sysc.thermostat)
    e = g.energy()
    assert e["gauss_exact"] == 1.0
    D, B, Lg = g.fields()
    x, v, img = g.particles()
    Lg_sum = Lg.reshape(3, -1).sum(axis=1)
    P = refs.dipole_fixed(x, img, sysc.q, sysc.mesh, 1.0)
    assert np.allclose([e["P0"], e["P1"], e["P2"]], P, rtol=0, atol=1e-9)
    # eps varies along x only: eps_eff^-1 is the harmonic mean across the
    # layers for x and the arithmetic mean along them for y and z
    e_par = refs.eps_at("sin", sysc.eps.params, np.arange(64.0), 64.0)
    e_nrm = refs.eps_at("sin", sysc.eps.params, np.arange(64.0) + 0.5, 64.0)
    Mc = np.diag([np.mean(1 / e_nrm), 1 / np.mean(e_par), 1 / np.mean(e_par)])
    _, _, Mg = g.setup()
    assert np.max(np.abs(Mg - Mc)) < 1e-10 * np.max(Mc)
    o = O.OracleSystem(sysc.mesh, sysc.box, eps=oracle_eps(sysc.eps), c_light=sysc.c_light,
                       dt=sysc.dt, seed=sysc.seed, eps_eff_inv=Mc)
    o.set_particles(x, sysc.q, sysc.m, v, img)
    o.field("D")[...] = D
    o.field("Lg")[...] = Lg
    o.gather()
    assert rel(g.forces(), o.particles("F")) < 1e-5
    assert np.array_equal(refs.divergence(Lg), refs.cic(x, sysc.q, sysc.mesh, 1.0))
    assert Lg_sum.dtype == np.int64


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_field_kernels_agree_on_a_large_mesh(precision):
    # the field kernels against each other on a mesh of many tiles (ragged in
    # y and z): same state, 3 steps, fields equal to rounding
    from paper_1309_7859_gb300.memd import Memd
    sysc = small_system((96, 44, 37), 2000, SLAB, precision=precision, dt=0.005)
    out = []
    for fk in ("ldg", "tma", "site", "rows"):
        g = Memd(sysc.mesh, sysc.box, sysc.eps, c_light=1.0, dt=sysc.dt, precision=precision,
                 seed=3, field_kernel=fk)
        g.init_field(sysc.x, sysc.q, sysc.m, sysc.v)
        g.step(3, thermostat=(1.0, 1.0))
        if fk == "rows":
            assert g.kernel_stats().field_kernel.startswith("k_rows")
        D, B, Lg = g.fields()
        out.append((D, B, Lg, g.forces()))
    # FP32: B is the circulation of a nearly curl-free E, so the two kernels'
    # different rounding of E = D / eps shows up amplified by that cancellation;
    # the bound is the FP32 field tolerance used against the oracle
    tol = 1e-13 if precision == "fp64" else 1e-5
    for other in out[1:]:
        for a, b in zip(out[0][:2], other[:2]):
            assert rel(a, b) < tol
        assert rel(out[0][3], other[3]) < tol
    # the plain-load kernels (halo loops, one thread per site, whole rows)
    # share every operation: bit-identical
    for other in (out[2], out[3]):
        for a, b in zip(out[0], other):
            assert np.array_equal(a, b)


def test_automatic_field_kernel_choice():
    # left to choose, a system steps with the row kernel where its mesh fits
    # it (x extent a multiple of 4 sites with FP32 fields) and with a tile
    # kernel where it does not, with the results of the kernel asked for
    from paper_1309_7859_gb300.memd import Memd
    for mesh, rows in (((64, 40, 36), True), ((66, 40, 36), False)):
        sysc = small_system(mesh, 3000, SLAB, precision="fp32", dt=0.005)
        out = []
        for fk in ("auto", "rows" if rows else "site"):
            g = Memd(sysc.mesh, sysc.box, sysc.eps, c_light=1.0, dt=sysc.dt, precision="fp32",
                     seed=3, field_kernel=fk, step_engine="graph")
            g.init_field(sysc.x, sysc.q, sysc.m, sysc.v)
            g.step(4, thermostat=(1.0, 1.0))
            assert g.energy()["gauss_exact"] == 1.0
            out.append((g.kernel_stats().field_kernel, g.fields(), g.forces()))
            g.close()
        assert out[0][0].startswith("k_rows") == rows, out[0][0]
        if rows:
            # the row kernel at either width does the same arithmetic
            for a, b in zip(out[0][1], out[1][1]):
                assert np.array_equal(a, b)
            assert np.array_equal(out[0][2], out[1][2])
        else:
            # a tile kernel (the TMA one agrees to rounding)
            for a, b in zip(out[0][1][:2], out[1][1][:2]):
                assert rel(a, b) < 1e-5
            assert rel(out[0][2], out[1][2]) < 1e-5


@pytest.mark.parametrize("mesh,n,eps,precision", [((8, 8, 8), 16, EpsSpec("const", 0, (1.0,)), "fp64"),
                                                  ((40, 20, 12), 300, SLAB, "fp32"),
                                                  ((24, 24, 24), 5000, SLAB, "fp32"),
                                                  ((72, 20, 6), 200, SINX, "fp64"),
                                                  ((4, 6, 2), 8, EpsSpec("const", 0, (2.0,)), "fp32")])
def test_step_engines_bit_identical(mesh, n, eps, precision):
    # the single cooperative launch and the graph of four kernels run the same
    # device functions: 20 thermostatted steps give identical bits, also with
    # several particle passes per CTA (5000 charges) and ragged tiles
    from paper_1309_7859_gb300.memd import Memd
    sysc = small_system(mesh, n, eps, precision=precision, dt=0.005)
    out = []
    for engine in ("graph", "single"):
        g = Memd(sysc.mesh, sysc.box, sysc.eps, c_light=1.0, dt=sysc.dt, precision=precision,
                 seed=5, step_engine=engine, field_kernel="site")
        g.init_field(sysc.x, sysc.q, sysc.m, sysc.v)
        g.step(20, thermostat=(1.0, 1.0))
        assert g.kernel_stats().single == (engine == "single")
        D, B, Lg = g.fields()
        x, v, img = g.particles()
        e = g.energy()
        out.append((D, B, Lg, x, v, img, g.forces(), e["total"], e["P0"], e["step"]))
        g.close()
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(np.asarray(a), np.asarray(b))


@pytest.mark.parametrize("mesh,n,precision", [((15, 9, 7), 60, "fp32"),     # 3V odd
                                               ((16, 12, 10), 80, "fp64"),   # two chunks
                                               ((24, 24, 24), 5000, "fp32"),
                                               ((40, 8, 8), 10, "fp64")])    # 24 per charge
def test_apply_modes_bit_identical(mesh, n, precision):
    # the transfers of a step applied per charge (atomic exchanges on the
    # crossed links) or by one pass over every link's word: each word gets
    # one addition either way, so 20 thermostatted graph steps agree bit for bit
    from paper_1309_7859_gb300.memd import Memd
    sysc = small_system(mesh, n, SLAB, precision=precision, dt=0.005)
    out = []
    for mode in ("sparse", "dense"):
        g = Memd(sysc.mesh, sysc.box, sysc.eps, c_light=1.0, dt=sysc.dt, precision=precision,
                 seed=5, step_engine="graph", apply_mode=mode)
        g.init_field(sysc.x, sysc.q, sysc.m, sysc.v)
        g.step(20, thermostat=(1.0, 1.0))
        D, B, Lg = g.fields()
        x, v, img = g.particles()
        e = g.energy()
        assert e["gauss_exact"] == 1.0
        out.append((D, B, Lg, x, v, img, g.forces(), e["total"], e["P0"], e["step"]))
        g.close()
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(np.asarray(a), np.asarray(b))


@pytest.mark.parametrize("engine", ["graph", "single"])
def test_direct_launches_match_graphs_with_timing(engine):
    # the same steps launched directly (no CUDA graph) with kernel timing on
    # give the graph-replayed result bit for bit
    from paper_1309_7859_gb300.memd import Memd
    sysc = small_system((24, 16, 12), 120, SLAB, precision="fp32", dt=0.005)
    out = []
    for graphs in (True, False):
        g = Memd(sysc.mesh, sysc.box, sysc.eps, c_light=1.0, dt=sysc.dt, precision="fp32", seed=9,
                 step_engine=engine, use_graphs=graphs, time_kernels=True)
        g.init_field(sysc.x, sysc.q, sysc.m, sysc.v)
        g.step(12, thermostat=(1.0, 1.0))
        ks = g.kernel_stats()
        assert ks.field_launches >= 1 and ks.field_ms > 0
        D, B, Lg = g.fields()
        x, v, img = g.particles()
        out.append((D, B, Lg, x, v, img, g.forces()))
        g.close()
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("engine", ["graph", "single"])
def test_step_host_equals_the_separate_calls(engine):
    # memd_step_host (load, step, read back, one sync) against memd_set_particles
    # + memd_step + memd_get_particles + memd_forces, bit for bit
    import torch
    sysc = small_system((16, 12, 8), 60, SLAB, precision="fp32", dt=0.005)
    a, _ = make_pair(sysc, step_engine=engine)
    b, _ = make_pair(sysc, step_engine=engine)
    n = sysc.n
    pin = lambda dt: torch.empty((n, 3), dtype=dt, pin_memory=True).numpy()
    hx, hv, hi, hf = pin(torch.float64), pin(torch.float64), pin(torch.int32), pin(torch.float64)
    a.get_particles_into(hx, hv, hi)
    x2, v2, i2 = a.particles()
    for _ in range(6):
        a.step_host(1, thermostat=(1.0, 1.0), x_in=hx, v_in=hv, img_in=hi, x_out=hx, v_out=hv,
                    img_out=hi, f_out=hf)
        b.set_particles(x2, v2, i2)
        b.step(1, thermostat=(1.0, 1.0))
        x2, v2, i2 = b.particles()
        f2 = b.forces()
        assert np.array_equal(hx, x2) and np.array_equal(hv, v2) and np.array_equal(hi, i2)
        assert np.array_equal(hf, f2)
    a.step_host(3)                          # no load, no read-back
    b.step(3)
    assert np.array_equal(a.particles()[0], b.particles()[0])
    D1, B1, L1 = a.fields()
    D2, B2, L2 = b.fields()
    assert np.array_equal(D1, D2) and np.array_equal(L1, L2)


@pytest.mark.parametrize("engine", ["graph", "single"])
def test_step_io_equals_the_separate_calls(engine):
    # an odd particle count (the image counters end off an 8-byte boundary):
    # 60 charges and one neutral particle
    sysc = small_system((16, 12, 8), 60, SLAB, precision="fp32", dt=0.005)
    sysc.x = np.concatenate([sysc.x, [[3.3, 4.4, 5.5]]])
    sysc.v = np.concatenate([sysc.v, [[0.1, -0.2, 0.3]]])
    sysc.m = np.concatenate([sysc.m, [1.0]])
    sysc.q = np.concatenate([sysc.q, [0]]).astype(np.int32)
    a, _ = make_pair(sysc, step_engine=engine)
    b, _ = make_pair(sysc, step_engine=engine)
    io = a.io_buffers()
    a.step_io(0, load=False)
    x2, v2, i2 = b.particles()
    assert np.array_equal(io["pos"], x2) and np.array_equal(io["vel"], v2)
    for _ in range(5):
        io["vel"] *= 0.999                  # the host edits the state between steps
        a.step_io(1, thermostat=(1.0, 1.0), load=True)
        b.set_particles(x2, v2 * 0.999, i2)
        b.step(1, thermostat=(1.0, 1.0))
        x2, v2, i2 = b.particles()
        assert np.array_equal(io["pos"], x2) and np.array_equal(io["vel"], v2)
        assert np.array_equal(io["img"], i2) and np.array_equal(io["f"], b.forces())


@pytest.mark.parametrize("engine,precision", [("graph", "fp64"), ("single", "fp32"),
                                              ("graph", "fp32")])
def test_resume_from_a_saved_state_is_bit_identical(engine, precision):
    # run A: 7 steps, save, 9 more; run B: a fresh context, any initial state
    # of the same particle count, load A's saved state, 9 steps: identical
    sysc = small_system((16, 12, 10), 80, SLAB, precision=precision, dt=0.005)
    a, _ = make_pair(sysc, step_engine=engine)
    a.step(7, thermostat=(1.0, 1.0))
    saved = a.save_state()
    a.step(9, thermostat=(1.0, 1.0))
    b, _ = make_pair(sysc, step_engine=engine, init=False)
    b.init_field(sysc.x[::-1].copy(), sysc.q, sysc.m, None)
    b.load_state(saved)
    b.step(9, thermostat=(1.0, 1.0))
    for u, w in zip(a.fields(), b.fields()):
        assert np.array_equal(u, w)
    for u, w in zip(a.particles(), b.particles()):
        assert np.array_equal(u, w)
    assert np.array_equal(a.forces(), b.forces())
    ea, eb = a.energy(), b.energy()
    for k in ("total", "P0", "P1", "P2", "step"):
        assert ea[k] == eb[k], k
    # a state of another particle count is refused and changes nothing
    from paper_1309_7859_gb300.memd import MemdError
    c, _ = make_pair(small_system((16, 12, 10), 20, SLAB, precision=precision), init=True,
                     step_engine=engine)
    before = c.particles()[0].copy()
    with pytest.raises(MemdError):
        c.load_state(saved)
    assert np.array_equal(c.particles()[0], before)


@pytest.mark.parametrize("field", ["x_outside", "x_nan", "mass_zero", "valence"])
def test_corrupted_saved_state_is_refused(field):
    # a saved state ends with the particle arrays x, v, F, Ft (3n doubles
    # each), img (3n int32), q (n int32), m (n doubles); one corrupted entry
    # is refused before anything is copied
    from paper_1309_7859_gb300.memd import Memd, MemdError
    sysc = small_system((16, 12, 10), 40, SLAB, precision="fp32", dt=0.005)
    a = Memd(sysc.mesh, sysc.box, sysc.eps, c_light=sysc.c_light, dt=sysc.dt, precision="fp32",
             seed=sysc.seed)
    a.init_field(sysc.x, sysc.q, sysc.m, sysc.v)
    a.step(3, thermostat=(1.0, 1.0))
    saved = a.save_state()
    n, size = 40, saved.size
    bad = saved.copy()
    x = bad[size - 120 * n: size - 96 * n].view(np.float64)
    q = bad[size - 12 * n: size - 8 * n].view(np.int32)
    m = bad[size - 8 * n:].view(np.float64)
    assert np.array_equal(x.reshape(n, 3), a.particles()[0])   # the layout read above
    if field == "x_outside":
        x[7] = sysc.box[1] + 0.25
    elif field == "x_nan":
        x[11] = np.nan
    elif field == "mass_zero":
        m[5] = 0.0
    else:
        q[3] = 40000
    before = [u.copy() for u in a.fields()] + [u.copy() for u in a.particles()]
    with pytest.raises(MemdError) as err:
        a.load_state(bad)
    assert err.value.status == 1                                 # MEMD_ERR_INVALID
    after = list(a.fields()) + list(a.particles())
    for u, w in zip(before, after):
        assert np.array_equal(u, w)
    a.load_state(saved)                                          # the intact state loads
    a.step(2, thermostat=(1.0, 1.0))
    assert a.energy()["gauss_exact"] == 1.0
