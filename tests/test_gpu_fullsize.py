"""GPU parity at full size: the kernel instances the benchmark times, on the
meshes it times them on (or larger ragged ones), against the FP64 oracle.

The oracle cannot relax a 256^3 field in test time, and no oracle input may
come from the CUDA path, so every test starts both sides from one state made
on the CPU: the exact int64 Gauss scan of the charges (Fig. 1, the oracle's
own scan routine) as the ledger, D = Lg 2^-48 / a^2 with its k = 0 mode at
-P / V (Sec. V), B = 0.  Any D with div D = rho is a valid MEMD state; this
one is simply not relaxed.  The oracle's effective permittivity is the
closed form of a medium layered along one axis (harmonic mean across the
layers, arithmetic mean along them), exact for these profiles and pinned
as such in the oracle tests.

Tolerances as in test_gpu_parity: FP64 fields and forces 1e-12, FP32 1e-5
(relative RMS); with FP32 fields the FP64 positions differ by ~1e-12, so the
ledger is checked through the exact Gauss identity instead of bit for bit.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1309_7859_gb300 import inputs
from paper_1309_7859_gb300.inputs import EpsSpec, System
from tests import refs

pytestmark = pytest.mark.gpu

TH = (1.0, 1.0)


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.sqrt(np.sum(b * b))
    return float(np.sqrt(np.sum((a - b) ** 2)) / (den if den > 0 else 1.0))


def layered_eps_eff_inv(spec, mesh, a=1.0):
    """Inverse effective permittivity of a profile along spec.axis: links
    along the axis in series (mean of 1/eps at their midpoints), the others
    in parallel (1 / mean of eps at the vertex planes)."""
    ax = spec.axis
    N = mesh[ax]
    L = N * a
    s = np.arange(N, dtype=np.float64) * a
    e_par = refs.eps_at(spec.kind, spec.params, s, L)
    e_nrm = refs.eps_at(spec.kind, spec.params, s + 0.5 * a, L)
    M = np.zeros((3, 3))
    for d in range(3):
        M[d, d] = np.mean(1.0 / e_nrm) if d == ax else 1.0 / np.mean(e_par)
    return M


def oracle_for(sysc):
    okind = {"tanh": O.EPS_TANH, "sin": O.EPS_SIN}[sysc.eps.kind]
    return O.OracleSystem(sysc.mesh, sysc.box,
                          eps=dict(kind=okind, axis=sysc.eps.axis, params=sysc.eps.params),
                          c_light=sysc.c_light, dt=sysc.dt, seed=sysc.seed,
                          eps_eff_inv=layered_eps_eff_inv(sysc.eps, sysc.mesh))


def cpu_state(o, sysc):
    """The unrelaxed Gauss state of sysc on the CPU, loaded into the oracle
    (which then gathers its forces); returns (D, Lg) in the field layout."""
    o.set_particles(sysc.x, sysc.q, sysc.m, sysc.v)
    Q = o.cic_charges()
    st, Lg = O.gauss_scan(sysc.mesh, Q)
    assert st == 0
    a = o.a
    V = o.V
    Lg = Lg.reshape(3, V)
    P = refs.dipole_fixed(o.particles("x"), o.particles("img"), sysc.q, sysc.mesh, a)
    scale = 2.0 ** -48 / (a * a)
    D = np.empty((3, V))
    for d in range(3):
        shift = -P[d] / o.Vbox - (float(np.sum(Lg[d])) * scale) / V
        D[d] = Lg[d] * scale + shift
    Nx, Ny, Nz = sysc.mesh
    o.field("Lg")[...] = Lg.reshape(3, Nz, Ny, Nx)
    o.field("D")[...] = D.reshape(3, Nz, Ny, Nx)
    o.field("B")[...] = 0.0
    o.gather()
    return D.reshape(3, Nz, Ny, Nx), Lg.reshape(3, Nz, Ny, Nx)


def gpu_from(sysc, D, Lg, o, **kw):
    """A GPU context holding the same state (its own init is overwritten)."""
    from paper_1309_7859_gb300.memd import Memd
    g = Memd(sysc.mesh, sysc.box, sysc.eps, c_light=sysc.c_light, dt=sysc.dt,
             precision=sysc.precision, seed=sysc.seed, **kw)
    g.init_field(sysc.x, sysc.q, sysc.m, sysc.v)
    g.set_fields(D=D, B=np.zeros_like(D), Lg=Lg)
    g.set_particles(x=o.particles("x"), v=o.particles("v"), img=o.particles("img"))
    g.compute_forces()
    return g


def compare(g, o, tol, ledger_exact):
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
    assert g.energy()["gauss_exact"] == 1.0
    assert o.energy()["gauss_exact"] == 1.0


def slab_system(mesh, n, precision, seed):
    rng = np.random.default_rng(seed)
    box = tuple(float(N) for N in mesh)
    eps = inputs.random_slab_eps(rng, min(mesh))
    return System(name=f"slab-{mesh}", mesh=tuple(mesh), box=box, eps=eps, c_light=1.0,
                  dt=0.005, precision=precision, x=inputs.uniform_positions(rng, n, box),
                  q=inputs.neutral_charges(rng, n), m=np.ones(n),
                  v=inputs.thermal_velocities(rng, n), steps=3, thermostat=TH, seed=seed)


def test_rows_512_at_256_cubed_matches_oracle():
    # the instance the bench's large_mesh object times: k_rows<nt=512> on the
    # 256^3 slab of 1e5 charges, FP32 fields, 3 steps from one state
    sysc = inputs.big_slab(N=256)
    o = oracle_for(sysc)
    D, Lg = cpu_state(o, sysc)
    g = gpu_from(sysc, D, Lg, o, field_kernel="rows", field_shape=(0, 0, 0, 512),
                 step_engine="graph")
    assert rel(g.forces(), o.particles("F")) < 1e-5
    o.step(3, thermostat=TH)
    g.step(3, thermostat=TH)
    assert g.kernel_stats().field_kernel == "k_rows<nt=512>"
    compare(g, o, 1e-5, ledger_exact=False)
    g.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_site_8_16_1_on_a_ragged_mesh_matches_oracle(precision):
    # the instance the bench picks at 384^3: k_fused_site<ty=8, zchunk=16,
    # planes_ahead=1>, here on 136 x 130 x 129 (ragged tiles in x, y and z)
    sysc = slab_system((136, 130, 129), 40000, precision, seed=91)
    o = oracle_for(sysc)
    D, Lg = cpu_state(o, sysc)
    g = gpu_from(sysc, D, Lg, o, field_kernel="site", field_shape=(8, 16, 1, 0),
                 step_engine="graph")
    o.step(3, thermostat=TH)
    g.step(3, thermostat=TH)
    assert g.kernel_stats().field_kernel == "k_fused_site<ty=8, zchunk=16, planes_ahead=1>"
    tol = 1e-5 if precision == "fp32" else 1e-12
    compare(g, o, tol, ledger_exact=precision == "fp64")
    g.close()


def test_rows_512_on_a_ragged_mesh_matches_oracle():
    # k_rows<nt=512> with tiles of 13 rows (132 / 4 = 33 vectors a row)
    # cutting 130 rows and 129 planes unevenly
    sysc = slab_system((132, 130, 129), 40000, "fp32", seed=92)
    o = oracle_for(sysc)
    D, Lg = cpu_state(o, sysc)
    g = gpu_from(sysc, D, Lg, o, field_kernel="rows", field_shape=(0, 0, 0, 512),
                 step_engine="graph")
    o.step(3, thermostat=TH)
    g.step(3, thermostat=TH)
    assert g.kernel_stats().field_kernel == "k_rows<nt=512>"
    compare(g, o, 1e-5, ledger_exact=False)
    g.close()


def test_salt_64_ten_steps_from_one_state():
    # the 64^3 salt system (32768 charges, eps(x) from the salt modulation),
    # FP32 fields, stepped 10 steps on both sides with the engine and field
    # kernel the library picks for it
    sysc = inputs.salt_64()
    o = oracle_for(sysc)
    D, Lg = cpu_state(o, sysc)
    g = gpu_from(sysc, D, Lg, o)
    o.step(10, thermostat=sysc.thermostat)
    g.step(10, thermostat=sysc.thermostat)
    compare(g, o, 1e-5, ledger_exact=False)
    P = refs.dipole_fixed(*g.particles()[::2], sysc.q, sysc.mesh, 1.0)
    e = g.energy()
    assert np.allclose([e["P0"], e["P1"], e["P2"]], P, rtol=0, atol=1e-9)
    g.close()


def paired_request(N, n_pairs, seed, steps):
    """A served-size request whose charges start as coincident +1/-1 pairs:
    the charge density, the Gauss ledger and the dipole are then exactly 0,
    so the initial field is D = B = 0 on any solver; the pairs separate with
    their own thermal velocities and build the fields up from there."""
    rng = np.random.default_rng(seed)
    box = (float(N),) * 3
    xp = inputs.uniform_positions(rng, n_pairs, box)
    x = np.repeat(xp, 2, axis=0)
    q = np.tile(np.array([1, -1], dtype=np.int32), n_pairs)
    v = inputs.thermal_velocities(rng, 2 * n_pairs)
    eps = EpsSpec("tanh", 2, (41.0, 39.0, N / 2.0, N / 4.0, 1.5))
    return System(name=f"pairs-{N}^3", mesh=(N, N, N), box=box, eps=eps, c_light=1.0,
                  dt=0.005, precision="fp32", x=x, q=q, m=np.ones(2 * n_pairs), v=v,
                  steps=steps, thermostat=TH, seed=seed)


def test_served_size_request_through_the_server_matches_oracle():
    # a 95^3 request (x extent not a multiple of 4: no row kernel) run by the
    # server in a batch with other requests that join and leave around it,
    # over several scheduling rounds, against the oracle from the same state
    from paper_1309_7859_gb300.memd import Server
    big = paired_request(95, 6000, seed=77, steps=24)
    others = []
    rng = np.random.default_rng(5)
    for r in range(5):
        N = int(rng.choice([16, 20, 24]))
        box = (float(N),) * 3
        n = 40 + 20 * r
        others.append(System(name=f"o{r}", mesh=(N, N, N), box=box,
                             eps=EpsSpec("const", 0, (2.0 + r,)), c_light=1.0, dt=0.005,
                             precision="fp32", x=inputs.uniform_positions(rng, n, box),
                             q=inputs.neutral_charges(rng, n), m=np.ones(n),
                             v=inputs.thermal_velocities(rng, n), steps=6 + 5 * r,
                             thermostat=TH, seed=300 + r))
    srv = Server(precision="fp32", budget_bytes=4 << 30, max_slots=8, quantum=4, thermostat=TH)
    ids = [srv.submit(s) for s in others[:2]]
    bid = srv.submit(big)
    srv.pump()
    ids += [srv.submit(s) for s in others[2:]]
    for _ in range(2000):
        a, q, d = srv.pump()
        if d == len(others) + 1:
            break
    assert srv.status(bid) == 2
    x, v, img, f, e = srv.result(bid)
    srv.close()
    o = oracle_for(big)
    o.set_particles(big.x, big.q, big.m, big.v)
    assert not np.any(o.cic_charges())       # the pairs cancel vertex by vertex
    o.field("D")[...] = 0.0
    o.field("B")[...] = 0.0
    o.field("Lg")[...] = 0
    o.gather()
    o.step(big.steps, thermostat=TH)
    assert e["step"] == big.steps
    assert np.array_equal(img, o.particles("img"))
    assert np.max(np.abs(x - o.particles("x"))) < 1e-9
    assert rel(v, o.particles("v")) < 1e-5
    assert rel(f, o.particles("F")) < 1e-5
    eo = o.energy()
    assert e["gauss_exact"] == 1.0 and eo["gauss_exact"] == 1.0
    for k in ("electric", "magnetic"):
        assert abs(e[k] - eo[k]) <= 1e-5 * abs(eo[k]), k
