"""GPU parity of the permittivity from the local salt density (Sec. I
motivation; the rule is this library's reading: |q| cloud-in-cell density,
periodic Gaussian smoothing, clamped linear map, vertex values applied as
the vertex profile).  The vertex values come from FP64 sums in a different
order on the two sides (the mean is a tree reduction on the GPU), so they
agree to 1e-13; fields and forces then follow the usual tolerances."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1309_7859_gb300 import inputs
from paper_1309_7859_gb300.inputs import EpsSpec, System
from tests.test_gpu_parity import compare_state, load_oracle_state, make_pair, rel

pytestmark = pytest.mark.gpu

RULE = (60.0, -40.0, 40.0, 80.0, 1.5)


def salt_system(mesh, n, precision, seed=12):
    rng = np.random.default_rng(seed)
    box = tuple(float(N) for N in mesh)
    x = inputs.sine_modulated_positions(rng, n, box, 0, 0.5)
    return System(name="salt", mesh=tuple(mesh), box=box, eps=EpsSpec("const", 0, (60.0,)),
                  c_light=1.0, dt=0.005, precision=precision, x=x,
                  q=inputs.neutral_charges(rng, n), m=np.ones(n),
                  v=inputs.thermal_velocities(rng, n), steps=10, thermostat=(1.0, 1.0), seed=seed)


@pytest.mark.parametrize("precision,relax", [("fp64", False), ("fp64", True), ("fp32", False)])
def test_salt_eps_and_steps_match_oracle(precision, relax):
    sysc = salt_system((24, 20, 16), 3000, precision)
    g, o = make_pair(sysc)
    load_oracle_state(g, o)
    eg = g.eps_from_density(*RULE, relax=relax)
    eo = o.eps_from_density(*RULE, relax=relax)
    assert rel(eg, eo) < 1e-13
    assert eo.min() < 55.0 and eo.max() > 65.0          # the profile follows the salt
    ie, _, M = g.setup()
    assert rel(ie, o.field("ie")) < 1e-13
    assert np.max(np.abs(M - o.Minv)) < 1e-10 * np.max(np.abs(o.Minv))
    D, _, _ = g.fields()
    if precision == "fp64":
        assert rel(D, o.field("D")) < (1e-9 if relax else 1e-15)
        assert rel(g.forces(), o.particles("F")) < (1e-8 if relax else 1e-10)
    else:                                              # D held in FP32
        assert rel(D, o.field("D")) < 1e-7
        assert rel(g.forces(), o.particles("F")) < 1e-5
    # then 10 steps from one state
    load_oracle_state(g, o)
    o.step(10, thermostat=sysc.thermostat)
    g.step(10, thermostat=sysc.thermostat)
    compare_state(g, o, 1e-12 if precision == "fp64" else 1e-5, ledger_exact=precision == "fp64")
    assert g.energy()["gauss_exact"] == 1.0


def test_salt_eps_at_the_salt_workload_size():
    # the 64^3 salt workload (32768 charges): vertex values of the rule, GPU
    # against the oracle's values at full size (nothing applied on the
    # oracle's side, so its effective tensor need not be solved)
    from paper_1309_7859_gb300.memd import Memd
    sysc = inputs.salt_64(precision="fp32")
    g = Memd(sysc.mesh, sysc.box, sysc.eps, c_light=sysc.c_light, dt=sysc.dt, precision="fp32",
             seed=sysc.seed)
    g.init_field(sysc.x, sysc.q, sysc.m, sysc.v)
    g.step(5, thermostat=sysc.thermostat)
    x, v, img = g.particles()
    eg = g.eps_from_density(60.0, -40.0, 40.0, 80.0, 3.0)
    o = O.OracleSystem(sysc.mesh, sysc.box, c_light=sysc.c_light, dt=sysc.dt, seed=sysc.seed,
                       eps_eff_inv=np.eye(3) / 60.0)
    o.set_particles(x, sysc.q, sysc.m, v, img)
    eo = o.salt_vertex_eps(60.0, -40.0, 40.0, 80.0, 3.0)
    assert rel(eg, eo) < 1e-13
    # the rule recovers the workload's static profile, 60 - 20 sin(2 pi x / L),
    # up to sampling noise and the smoothing's attenuation at that wave number
    prof = eg.mean(axis=(0, 1))
    amp = 2 * np.mean(prof * np.sin(2 * np.pi * np.arange(64) / 64))
    H = np.exp(-(3.0 * 2 * np.pi / 64) ** 2 / 2)
    assert abs(amp + 20.0 * H) < 1.5
    g.step(5, thermostat=sysc.thermostat)             # stepping on in the new medium
    assert g.energy()["gauss_exact"] == 1.0


def test_salt_rule_is_refused_when_out_of_range():
    from paper_1309_7859_gb300.memd import MemdError
    sysc = salt_system((8, 8, 8), 20, "fp64")
    g, _ = make_pair(sysc, init=False)
    g.init_field(sysc.x, sysc.q, sysc.m, sysc.v)
    for bad in ((60.0, -40.0, 0.0, 80.0, 1.0), (60.0, -40.0, 50.0, 40.0, 1.0),
                (60.0, -40.0, 40.0, 80.0, -1.0), (np.nan, -40.0, 40.0, 80.0, 1.0)):
        with pytest.raises(MemdError):
            g.eps_from_density(*bad)
    g.step(2)
