"""Interface-link permittivity (Sec. II, Eq. dielectric-interpolation) and a
permittivity replaced on a live system: the CUDA path against the oracle.

Tolerances: 1/eps per link 1e-14 relative (the two sides write the series
average in different but equivalent forms, a few roundings each, with a
contrast of up to 40 between the media); eps_eff^-1 1e-10 (iterative solves);
states after stepping as in the step-parity tests (1e-12 FP64)."""
import numpy as np
import pytest

from paper_1309_7859_gb300.inputs import EpsSpec
from tests.test_gpu_parity import (ENGINES, compare_state, load_oracle_state, make_pair, rel,
                                   small_system)

pytestmark = pytest.mark.gpu


def cut_values(rng, mesh, frac_cut=0.4):
    """vertex eps in two media with noise, and random cut positions on a
    share of the links (the rest marked uncut)"""
    V = mesh[0] * mesh[1] * mesh[2]
    vals = np.where(rng.uniform(size=V) < 0.5, 2.0, 80.0) * rng.uniform(0.9, 1.1, size=V)
    t = rng.uniform(0.0, 1.0, size=3 * V)
    t[rng.uniform(size=3 * V) > frac_cut] = -1.0
    t[:5] = (0.0, 1.0, 0.5, -0.25, 1.5)
    return np.concatenate([vals, t])


def two_media_vertices(rng, mesh):
    V = mesh[0] * mesh[1] * mesh[2]
    return np.where(rng.uniform(size=V) < 0.3, 80.0, 2.0) * rng.uniform(0.95, 1.05, size=V)


CASES = [((8, 6, 8), EpsSpec("planes", 2, (2.0, 80.0, 2.3, 5.85))),
         ((16, 9, 7), EpsSpec("planes", 0, (3.0, 50.0, 4.0, 11.0))),     # faces on vertices
         ((33, 9, 7), EpsSpec("planes", 1, (80.0, 2.0, 0.0, 5.5))),
         ((16, 16, 16), EpsSpec("sphere", 0, (2.0, 80.0, 7.3, 8.1, 7.6, 4.2))),
         ((16, 16, 16), EpsSpec("sphere", 0, (2.0, 80.0, 8.0, 8.0, 8.0, 5.0))),  # 3-4-5 vertices
         ((40, 20, 12), EpsSpec("sphere", 0, (80.0, 2.0, 39.3, 9.7, 0.2, 4.5))),  # across the seam
         ((33, 9, 7), "cut"),
         ((40, 20, 12), "vertices-theta")]


def resolve(mesh, eps, seed=3):
    rng = np.random.default_rng(seed)
    if eps == "cut":
        return EpsSpec("cut", 0, (), cut_values(rng, mesh))
    if eps == "vertices-theta":
        return EpsSpec("vertices", 0, (1.0,), two_media_vertices(rng, mesh))
    return eps


@pytest.mark.parametrize("mesh,eps", CASES)
def test_interface_links_match_oracle(mesh, eps):
    sysc = small_system(mesh, 0, resolve(mesh, eps))
    g, o = make_pair(sysc, init=False)
    ie, G, M = g.setup()
    want = o.field("ie")
    assert np.max(np.abs(ie - want) / want) < 1e-14
    assert np.max(np.abs(M - o.Minv)) < 1e-10 * np.max(np.abs(o.Minv))


@pytest.mark.parametrize("mesh,eps", [CASES[0], CASES[3], CASES[6]])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_initial_solution_with_interfaces_matches_oracle(mesh, eps, precision):
    sysc = small_system(mesh, 40, resolve(mesh, eps), precision=precision)
    g, o = make_pair(sysc)
    D, B, Lg = g.fields()
    assert np.array_equal(Lg, o.field("Lg"))
    assert rel(D, o.field("D")) < (1e-9 if precision == "fp64" else 1e-6)
    assert rel(g.forces(), o.particles("F")) < (1e-8 if precision == "fp64" else 1e-5)


@pytest.mark.parametrize("engine,field_kernel", ENGINES)
def test_ten_steps_across_a_ball_fp64(engine, field_kernel):
    mesh, eps = CASES[5]
    sysc = small_system(mesh, 200, eps, dt=0.01)
    g, o = make_pair(sysc, field_kernel=field_kernel, step_engine=engine)
    load_oracle_state(g, o)
    o.step(10, thermostat=(1.0, 1.0))
    g.step(10, thermostat=(1.0, 1.0))
    compare_state(g, o, 1e-12)


def oracle_eps(spec):
    from tests.test_gpu_parity import oracle_eps as oe
    return oe(spec)


@pytest.mark.parametrize("engine,field_kernel", ENGINES)
def test_set_eps_keeps_D_and_steps_like_the_oracle(engine, field_kernel):
    # graphs captured under the old medium hold its effective tensor: the new
    # one must reach the dipole correction of the next steps
    mesh = (40, 20, 12)
    sysc = small_system(mesh, 200, EpsSpec("tanh", 2, (41.0, 39.0, 6.0, 3.0, 1.5)), dt=0.01)
    g, o = make_pair(sysc, field_kernel=field_kernel, step_engine=engine)
    load_oracle_state(g, o)
    o.step(5, thermostat=(1.0, 1.0))
    g.step(5, thermostat=(1.0, 1.0))
    then = CASES[5][1]
    D0, B0, _ = g.fields()
    o.set_eps(oracle_eps(then))
    g.set_eps(then)
    ie, _, M = g.setup()
    assert np.max(np.abs(ie - o.field("ie")) / o.field("ie")) < 1e-14
    assert np.max(np.abs(M - o.Minv)) < 1e-10 * np.max(np.abs(o.Minv))
    D1, B1, _ = g.fields()
    assert np.array_equal(D0, D1) and np.array_equal(B0, B1)
    # the forces now carry the new tensor, which each side solved
    # iteratively (to 1e-10): compare at that level
    compare_state(g, o, 1e-10)
    o.step(5, thermostat=(1.0, 1.0))
    g.step(5, thermostat=(1.0, 1.0))
    compare_state(g, o, 1e-9)


@pytest.mark.parametrize("engine", ["graph", "single"])
def test_set_eps_relaxed_matches_oracle(engine):
    mesh = (33, 9, 7)
    sysc = small_system(mesh, 60, EpsSpec("const", 0, (2.0,)), dt=0.01)
    g, o = make_pair(sysc, step_engine=engine)
    load_oracle_state(g, o)
    o.step(8, thermostat=(1.0, 1.0))
    g.step(8, thermostat=(1.0, 1.0))
    then = EpsSpec("planes", 2, (3.0, 30.0, 1.4, 4.9))
    o.set_eps(oracle_eps(then), relax=True)
    g.set_eps(then, relax=True)
    D, B, Lg = g.fields()
    assert np.array_equal(Lg, o.field("Lg"))
    assert rel(D, o.field("D")) < 1e-9
    assert np.all(B == 0)
    assert rel(g.forces(), o.particles("F")) < 1e-8
    assert g.energy()["gauss_exact"] == 1.0
    o.step(5, thermostat=(1.0, 1.0))
    g.step(5, thermostat=(1.0, 1.0))
    compare_state(g, o, 1e-7)


def test_set_eps_rejects_bad_profiles_and_keeps_the_old():
    from paper_1309_7859_gb300.memd import MemdError
    mesh = (16, 16, 16)
    sysc = small_system(mesh, 20, CASES[3][1])
    g, o = make_pair(sysc)
    ie0, _, M0 = g.setup()
    D0 = g.fields()[0]
    for bad in (EpsSpec("planes", 2, (2.0, 80.0, 9.0, 3.0)),
                EpsSpec("sphere", 0, (2.0, 80.0, 8.0, 8.0, 8.0, 7.5)),
                EpsSpec("links", 0, (), -np.ones(3 * 16 ** 3))):
        with pytest.raises(MemdError):
            g.set_eps(bad)
        ie, _, M = g.setup()
        assert np.array_equal(ie, ie0) and np.array_equal(M, M0)
        assert np.array_equal(g.fields()[0], D0)
    g.step(2)   # still usable


def test_batch_rebuilds_after_set_eps():
    import torch
    from paper_1309_7859_gb300.memd import Batch, Memd
    rng = np.random.default_rng(9)
    mesh = (16, 16, 16)
    box = tuple(float(n) for n in mesh)
    eps0, eps1 = EpsSpec("const", 0, (2.0,)), CASES[3][1]
    x = rng.uniform(0, 16, size=(40, 3))
    q = np.array([1, -1] * 20, dtype=np.int32)
    stream = torch.cuda.Stream()

    def make(s=None):
        g = Memd(mesh, box, eps0, c_light=1.0, dt=0.005, precision="fp64", seed=4,
                 field_kernel="ldg", stream=s)
        g.init_field(x, q)
        return g
    member, alone = make(stream), make()
    batch = Batch([member])
    batch.step(3)
    batch.synchronize()
    member.set_eps(eps1)
    alone.step(3)
    alone.set_eps(eps1)
    batch.step(4, thermostat=(1.0, 1.0))
    batch.synchronize()
    alone.step(4, thermostat=(1.0, 1.0))
    for u, w in zip(member.fields(), alone.fields()):
        assert np.array_equal(u, w)
    assert np.array_equal(member.forces(), alone.forces())
