"""The synthetic stand-ins for the paper's validation systems (dielectric
colloid in salt water, cloud-wall): their recipes, and a few oracle steps on
the small versions (no GPU)."""
import numpy as np

from oracle import oracle as O
from paper_1309_7859_gb300 import inputs
from tests import refs


def test_colloid_recipe():
    s = inputs.colloid()
    N, R, Qc = 64, 8.0, 60
    assert s.mesh == (N, N, N) and s.eps.kind == "sphere"
    assert s.eps.params[:2] == (80.0, 2.0) and s.eps.params[5] == R
    # 50 mmol/l of 1:1 salt in (64 nm)^3 is 0.0301 pairs per nm^3
    assert s.extra["salt_pairs"] == round(0.05 * 0.602214076 * N ** 3)
    assert s.q.sum() == 0 and s.q[:Qc].sum() == Qc and s.q[Qc:2 * Qc].sum() == -Qc
    c = np.array(s.box) / 2
    r_fixed = np.linalg.norm(s.x[:Qc] - c, axis=1)
    assert np.allclose(r_fixed, R - 0.5)
    d = s.x[Qc:] - c
    assert np.all(np.linalg.norm(d, axis=1) > R + 1.0)
    assert np.all(s.m[:Qc] >= 1e12) and np.all(s.m[Qc:] == 1.0)
    assert np.all(s.v[:Qc] == 0.0)


def test_cloud_wall_recipe():
    s = inputs.cloud_wall()
    nw = s.extra["wall_charges"]
    assert nw == 256 and s.q.sum() == 0
    assert np.all(s.x[:nw, 2] == 8.5) and np.all(s.x[nw:2 * nw, 2] == 24.5)
    P = refs.dipole_fixed(s.x[:2 * nw], np.zeros((2 * nw, 3)), s.q[:2 * nw], s.mesh, 1.0)
    assert abs(P[2] + nw * 16.0) < 1e-9       # the walls alone: -256 charges x 16 cells


def test_colloid_small_steps_on_the_oracle():
    s = inputs.colloid(N=16)
    o = O.OracleSystem(s.mesh, s.box, eps=dict(kind=O.EPS_SPHERE, params=s.eps.params),
                       c_light=s.c_light, dt=s.dt, seed=s.seed, relax_tol=1e-10)
    o.set_particles(s.x, s.q, s.m, s.v)
    o.init_field()
    x0 = o.particles("x").copy()
    o.step(5, thermostat=s.thermostat)
    e = o.energy()
    assert e["gauss_exact"] == 1.0
    assert np.max(np.abs(o.particles("x")[:60] - x0[:60])) < 1e-6
    assert np.max(np.abs(o.particles("x")[60:] - x0[60:])) > 1e-3
