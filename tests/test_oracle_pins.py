"""Pins of the CPU oracle against facts fixed outside it: published generator
vectors, exact integer identities of Gauss's law, closed-form lattice
electrostatics, the leapfrog mode amplitude, energy conservation and a
tinfoil Ewald sum.  Each test targets a mistake the oracle could plausibly
contain (a dropped term, a sign, a swapped weight, a transposed stencil)."""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from tests import refs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load_kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if not line:
                continue
            w = [int(t, 16) for t in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answers():
    rows = load_kat()
    assert len(rows) == 3
    for ctr, key, want in rows:
        assert list(O.philox4x32_10(ctr, key)) == want


def test_philox_noise_moments():
    # unit variance, zero mean noise from the 32-bit words (u + 1/2) 2^-32
    words = np.concatenate([O.philox4x32_10([i, 0, 7, 0], [123, 456]) for i in range(20000)])
    u = (words.astype(np.float64) + 0.5) * 2.0 ** -32
    xi = math.sqrt(3) * (2 * u - 1)
    assert abs(xi.mean()) < 0.02
    assert abs(xi.var() - 1.0) < 0.02


# ---------------------------------------------------------------- Green's table
@pytest.mark.parametrize("N", [(8, 8, 8), (6, 10, 4), (16, 16, 16)])
def test_green_table_matches_fft_and_laplacian(N):
    G8 = O.green_table(N)
    Gfull = refs.lattice_green_fft(N)
    for t in range(8):
        dx, dy, dz = t & 1, (t >> 1) & 1, (t >> 2) & 1
        assert abs(G8[t] - Gfull[dz, dy, dx]) < 1e-13
    # -Laplace G = delta - 1/V at the origin
    V = N[0] * N[1] * N[2]
    lap0 = sum(2 * (G8[0] - G8[1 << d]) for d in range(3))
    assert abs(lap0 - (1.0 - 1.0 / V)) < 1e-12


def test_green_origin_tends_to_watson_constant():
    # G at the origin of the infinite simple-cubic lattice is Watson's integral
    # W = 0.2527310098...; removing k = 0 on an N^3 torus lowers it by the
    # cubic-lattice constant xi / (4 pi N), xi = 2.837297479..., up to O(N^-3)
    W, xi = 0.2527310098586, 2.837297479481
    for n in (8, 16, 32):
        g0 = O.green_table((n, n, n))[0]
        assert abs(g0 - (W - xi / (4 * math.pi * n))) < 0.1 / n ** 3


# ------------------------------------------------------------ fixed point / CIC
def make(N=(8, 8, 8), a=1.0, **kw):
    L = tuple(n * a for n in N)
    return O.OracleSystem(N, L, **kw)


def test_quantization_round_trip_and_cic_moments():
    rng = np.random.default_rng(5)
    s = make((8, 8, 8), self_mode=O.SELF_NONE, dipole_corr=0)
    cells = rng.integers(1, 6, size=(40, 3))
    f = rng.integers(0, refs.S, size=(40, 3))
    x = (cells + (f + 0.5) / refs.S) * s.a
    c2, f2 = refs.quantize(x, s.a, s.N)
    assert np.array_equal(c2, cells) and np.array_equal(f2, f)
    for p in range(40):
        q = int(rng.choice([-2, -1, 1, 3]))
        s.set_particles(x[p:p + 1], [q])
        Q = s.cic_charges()
        bg = q * (1 << 48) // 512
        Q = Q + bg
        assert Q.sum() == q * (1 << 48)
        nz = np.argwhere(Q != 0)
        assert len(nz) <= 8
        # first moment about the cell corner: sum_corners Q a_d = q S^2 f_d
        for d, ax in enumerate((2, 1, 0)):
            mom = sum(int(Q[tuple(i)]) * int(i[ax] - cells[p][d]) for i in nz)
            assert mom == q * refs.S ** 2 * int(f[p][d])
        assert np.array_equal(Q - bg, refs.cic(x[p:p + 1], [q], s.N, s.a))


def test_background_must_be_exact():
    s = make((6, 6, 6))
    with pytest.raises(O.OracleError):
        s.set_particles([[1.0, 1.0, 1.0]], [1])   # 2^48 / 216 is not an integer
    s2 = make((8, 8, 8))
    s2.set_particles([[1.0, 1.0, 1.0]], [1])


# --------------------------------------------------------------- Gauss scan
@pytest.mark.parametrize("N", [(8, 8, 8), (5, 7, 3), (2, 2, 2), (16, 4, 9)])
def test_gauss_scan_is_exact(N):
    rng = np.random.default_rng(sum(N))
    V = N[0] * N[1] * N[2]
    Q = rng.integers(-(1 << 50), 1 << 50, size=V, dtype=np.int64)
    Q[-1] -= Q.sum()
    st, flux = O.gauss_scan(N, Q)
    assert st == O.OK
    F = flux.reshape(3, N[2], N[1], N[0])
    assert np.array_equal(refs.divergence(F), Q.reshape(N[2], N[1], N[0]))
    # the oracle's own divergence agrees with the definition
    assert np.array_equal(O.divergence(N, flux), refs.divergence(F).ravel())
    # Fig. 1: z-links of a plane carry the plane's cumulative charge evenly
    zf = F[2].reshape(N[2], -1)
    assert np.all(zf.max(axis=1) - zf.min(axis=1) <= 1)


def test_gauss_scan_rejects_non_neutral():
    Q = np.zeros(27, dtype=np.int64)
    Q[3] = 5
    st, _ = O.gauss_scan((3, 3, 3), Q)
    assert st == O.ERR_INVALID


# ------------------------------------------------------------ initial solution
def neutral_system(rng, n, N, a):
    L = np.array(N) * a
    x = rng.uniform(0, 1, size=(n, 3)) * L
    q = np.array([1, -1] * (n // 2), dtype=np.int32)
    return x, q


@pytest.mark.parametrize("N,eps", [((8, 8, 8), 1.0), ((6, 8, 10), 2.5), ((8, 8, 8), 40.0)])
def test_initial_solution_constant_eps_matches_fft(N, eps):
    rng = np.random.default_rng(11)
    a = 0.75
    s = make(N, a, eps=dict(kind=O.EPS_CONST, params=(eps,)))
    x, q = neutral_system(rng, 12, N, a)
    s.set_particles(x, q)
    s.init_field()
    Qe = refs.cic(x, q, N, a).astype(np.float64) * 2.0 ** -48
    P = refs.dipole_fixed(x, np.zeros((12, 3)), q, N, a)
    Dbar = -P / s.Vbox
    want = refs.fft_solution_const(N, a, Qe, eps, Dbar)
    got = s.field("D")
    assert np.max(np.abs(got - want)) < 1e-9 * np.max(np.abs(want))
    # the ledger is the exact Gauss flux of the vertex charges
    assert np.array_equal(refs.divergence(s.field("Lg")), refs.cic(x, q, N, a))
    e = s.energy()
    assert e["gauss_exact"] == 1.0
    assert e["gauss_residual"] < 1e-12
    assert np.allclose([e["P0"], e["P1"], e["P2"]], P, rtol=0, atol=1e-12)


@pytest.mark.parametrize("kind,params", [
    ("tanh", (41.0, 39.0, 4.0, 2.0, 1.5)),
    ("sin", (60.0, -20.0, 0.3)),
])
def test_initial_solution_layered_eps_matches_exact(kind, params):
    rng = np.random.default_rng(12)
    N, a = (8, 6, 8), 1.0
    okind = {"tanh": O.EPS_TANH, "sin": O.EPS_SIN}[kind]
    s = make(N, a, eps=dict(kind=okind, axis=2, params=params))
    x, q = neutral_system(rng, 10, N, a)
    s.set_particles(x, q)
    s.init_field()
    ex, ey, ez = refs.layer_eps(kind, params, N[2], a)
    ie = s.field("ie")
    assert np.allclose(1 / ie[0], ex[:, None, None], rtol=1e-14)
    assert np.allclose(1 / ie[2], ez[:, None, None], rtol=1e-14)
    Qe = refs.cic(x, q, N, a).astype(np.float64) * 2.0 ** -48
    P = refs.dipole_fixed(x, np.zeros((10, 3)), q, N, a)
    want = refs.layered_solution(N, a, Qe, ex, ey, ez, -P / s.Vbox)
    got = s.field("D")
    assert np.max(np.abs(got - want)) < 1e-9 * np.max(np.abs(want))
    # relaxed field is curl free
    E = got * ie
    assert np.max(np.abs(refs.curl_circulation(E))) < 1e-11 * np.max(np.abs(E))


def test_profile_axis_symmetry():
    # the same sine profile along x and along z gives transposed link eps
    sx = make((4, 6, 8), 1.0, eps=dict(kind=O.EPS_SIN, axis=0, params=(60.0, -20.0, 0.0)))
    sz = make((8, 6, 4), 1.0, eps=dict(kind=O.EPS_SIN, axis=2, params=(60.0, -20.0, 0.0)))
    ix, iz = sx.field("ie"), sz.field("ie")
    assert np.array_equal(ix[0], np.transpose(iz[2], (2, 1, 0)))
    assert np.array_equal(ix[1], np.transpose(iz[1], (2, 1, 0)))


def test_eps_effective_layered_closed_form():
    params = (41.0, 39.0, 4.0, 2.0, 1.5)
    s = make((8, 8, 8), 1.0, eps=dict(kind=O.EPS_TANH, axis=2, params=params))
    ex, ey, ez = refs.layer_eps("tanh", params, 8, 1.0)
    M = s.Minv
    assert abs(M[2, 2] - np.mean(1 / ez)) < 1e-12 * M[2, 2]       # series across layers
    assert abs(M[0, 0] - 1 / np.mean(ex)) < 1e-12 * M[0, 0]       # parallel along layers
    assert abs(M[1, 1] - 1 / np.mean(ey)) < 1e-12 * M[1, 1]
    assert np.max(np.abs(M - np.diag(np.diag(M)))) < 1e-13
    c = make((4, 4, 4), 1.0, eps=dict(kind=O.EPS_CONST, params=(7.0,)))
    assert np.allclose(c.Minv, np.eye(3) / 7.0, atol=1e-16)


# ------------------------------------------------------------- self energy
def test_single_charge_lattice_energy_is_self_energy_plus_dipole():
    # one charge on a uniform background, constant eps: the relaxed lattice
    # energy varies with the sub-cell position exactly as U_self + P^2/(2 V eps)
    eps, N, a = 2.0, (8, 8, 8), 1.0
    s = make(N, a, eps=dict(kind=O.EPS_CONST, params=(eps,)), relax_tol=1e-13)
    vals = []
    for fx in (0, 9000, 20000, 32768, 50000, 65535):
        f = np.array([fx, 13000, 41000])
        x = (np.array([3, 4, 2]) + (f + 0.5) / refs.S) * a
        s.set_particles([x], [1])
        s.init_field()
        el = s.energy()["electric"]
        U, _ = s.self_force([3, 4, 2], f, 1)
        P = refs.dipole_fixed([x], np.zeros((1, 3)), [1], N, a)
        vals.append((el, U + P @ P / (2 * s.Vbox * eps)))
    el0, pr0 = vals[0]
    for el, pr in vals[1:]:
        assert abs((el - el0) - (pr - pr0)) < 1e-11


def test_static_force_is_energy_gradient_and_corrections_cancel():
    eps, N, a = 3.0, (8, 8, 8), 1.0
    h = 64  # sub-cell steps for the central difference (exact for a quadratic)
    base = np.array([3, 4, 2])
    f0 = np.array([20000, 13000, 41000])

    def pos(f):
        return (base + (f + 0.5) / refs.S) * a

    raw = make(N, a, eps=dict(kind=O.EPS_CONST, params=(eps,)), self_mode=O.SELF_NONE,
               dipole_corr=0, relax_tol=1e-13)
    raw.set_particles([pos(f0)], [1])
    raw.init_field()
    F = raw.particles("F")[0].copy()
    for d in range(3):
        e = []
        for sg in (-1, 1):
            f = f0.copy()
            f[d] += sg * h
            raw.set_particles([pos(f)], [1])
            raw.init_field()
            e.append(raw.energy()["electric"])
        dE = (e[1] - e[0]) / (2 * h * a / refs.S)
        assert abs(F[d] + dE) < 1e-7 * max(1.0, abs(dE))
    cor = make(N, a, eps=dict(kind=O.EPS_CONST, params=(eps,)), self_mode=O.SELF_GF,
               dipole_corr=1, relax_tol=1e-13)
    for f in (f0, np.array([0, 0, 0]), np.array([32768, 100, 65000])):
        cor.set_particles([pos(f)], [1])
        cor.init_field()
        assert np.max(np.abs(cor.particles("F")[0])) < 1e-10


def test_self_force_symmetry_and_direct_reduces_to_gf():
    s = make((8, 8, 8), eps=dict(kind=O.EPS_CONST, params=(2.0,)))
    U, F = s.self_force([1, 1, 1], [32768, 32768, 32768])
    assert np.max(np.abs(F)) < 1e-15
    U1, F1 = s.self_force([1, 1, 1], [10000, 32768, 32768])
    U2, F2 = s.self_force([1, 1, 1], [65536 - 10000, 32768, 32768])
    assert abs(U1 - U2) < 1e-15 and abs(F1[0] + F2[0]) < 1e-15
    assert F1[0] < 0  # the correction pushes away from the cell centre
    d = make((8, 8, 8), eps=dict(kind=O.EPS_CONST, params=(2.0,)), self_mode=O.SELF_DIRECT)
    for f in ([1000, 30000, 60000], [40000, 5, 12345]):
        Ug, Fg = s.self_force([2, 3, 4], f)
        Ud, Fd = d.self_force([2, 3, 4], f)
        assert abs(Ug - Ud) < 1e-15 and np.max(np.abs(Fg - Fd)) < 1e-15


# ------------------------------------------ DIRECT self term in varying eps
# Eq. 29 is garbled; the reading (per direction d, 1/eps averaged over the
# cell's four d-links with the charge's weights) has no printed values to
# check against.  These pins use only what any correct reading of a local
# self term must satisfy: special media where it reduces to the uniform
# case (whose Green's table is pinned above), and lattice symmetries.
def _link_eps(N, fn):
    """eps on every link in the oracle's layout (component major, x
    fastest); fn(d, k, j, i) gives the (Nz, Ny, Nx) array of direction d."""
    return np.concatenate([np.asarray(fn(d, *np.meshgrid(np.arange(N[2]), np.arange(N[1]),
                                                           np.arange(N[0]), indexing="ij")),
                                      dtype=np.float64).ravel() for d in range(3)])


def test_direct_self_force_in_a_layered_medium_reduces_to_uniform_media():
    # eps varies only along z: the four z-links of a cell lie in one layer,
    # so the z-force is the uniform-medium self force of that layer; a charge
    # on lattice plane k puts no weight on plane k + 1, so its x- and y-forces
    # are those of a uniform medium with plane k's in-plane eps
    N = (8, 8, 8)
    rng = np.random.default_rng(31)
    ez = rng.uniform(2.0, 80.0, N[2])    # z-links from plane k to k + 1
    exy = rng.uniform(2.0, 80.0, N[2])   # x- and y-links in plane k
    vals = _link_eps(N, lambda d, k, j, i: (ez if d == 2 else exy)[k] + 0.0 * i)
    lay = make(N, eps=dict(kind=O.EPS_LINKS, values=vals), self_mode=O.SELF_DIRECT)
    gf = make(N, eps=dict(kind=O.EPS_LINKS, values=vals), self_mode=O.SELF_GF)
    for cell, f in (([2, 3, 4], [1000, 30000, 60000]), ([5, 0, 7], [40000, 5, 12345]),
                    ([0, 6, 1], [65535, 200, 33000])):
        k = cell[2]
        _, Fd = lay.self_force(cell, f)
        _, Fu = make(N, eps=dict(kind=O.EPS_CONST, params=(ez[k],))).self_force(cell, f)
        assert abs(Fd[2] - Fu[2]) <= 1e-14 * abs(Fu[2])
        _, Fg = gf.self_force(cell, f)          # the 12-link mean misses it
        assert abs(Fg[2] - Fu[2]) > 1e-3 * abs(Fu[2])
        f0 = [f[0], f[1], 0]
        _, Fd0 = lay.self_force(cell, f0)
        _, Fu0 = make(N, eps=dict(kind=O.EPS_CONST, params=(exy[k],))).self_force(cell, f0)
        assert np.max(np.abs(Fd0[:2] - Fu0[:2])) <= 1e-14 * np.max(np.abs(Fu0[:2]))


def test_direct_self_force_mirror_and_rotation_symmetry():
    # a random medium made mirror symmetric in z: the mirrored charge has the
    # same self energy and in-plane force and the opposite z-force; the same
    # medium with its axes permuted cyclically (a rotation) on a non-cubic
    # mesh: the force components permute with it
    S = refs.S
    N = (6, 8, 10)
    Nx, Ny, Nz = N
    rng = np.random.default_rng(37)
    A = rng.uniform(2.0, 80.0, (3, Nz, Ny, Nx))
    k = np.arange(Nz)
    mir = np.stack([A[0][(Nz - k) % Nz], A[1][(Nz - k) % Nz], A[2][Nz - 1 - k]])
    sym = 2.0 / (1.0 / A + 1.0 / mir)
    s = make(N, eps=dict(kind=O.EPS_LINKS, values=sym.ravel()), self_mode=O.SELF_DIRECT)
    # rotation: new (x, y, z) = old (z, x, y); direction d becomes (d + 1) % 3
    rot = np.empty((3, Ny, Nx, Nz))
    for d in range(3):
        rot[(d + 1) % 3] = A[d].transpose(1, 2, 0)
    r0 = make(N, eps=dict(kind=O.EPS_LINKS, values=A.ravel()), self_mode=O.SELF_DIRECT)
    r1 = make((Nz, Nx, Ny), eps=dict(kind=O.EPS_LINKS, values=rot.ravel()),
              self_mode=O.SELF_DIRECT)
    for cell, f in (([2, 3, 4], [1000, 30000, 60000]), ([5, 0, 9], [40000, 5, 12345]),
                    ([0, 7, 1], [65535, 200, 33000])):
        U1, F1 = s.self_force(cell, f)
        U2, F2 = s.self_force([cell[0], cell[1], Nz - 1 - cell[2]], [f[0], f[1], S - f[2]])
        tol = 1e-13 * np.max(np.abs(F1))
        assert abs(U1 - U2) <= 1e-13 * abs(U1)
        assert np.max(np.abs(F1[:2] - F2[:2])) <= tol and abs(F1[2] + F2[2]) <= tol
        U3, F3 = r0.self_force(cell, f)
        U4, F4 = r1.self_force([cell[2], cell[0], cell[1]], [f[2], f[0], f[1]])
        assert abs(U3 - U4) <= 1e-12 * abs(U3)
        assert np.max(np.abs(F4 - F3[[2, 0, 1]])) <= 1e-12 * np.max(np.abs(F3))


# ------------------------------------------------------ planar dielectric jump
def image_force_z(ein, eout, d, W, L):
    # charge +1 in a slab of eps_in, a distance d below its upper face, its
    # partner -1 at the same height L/2 away along x; continuum image charges
    # q' = (eps_in - eps_out) / (eps_in + eps_out) q for each face (first
    # reflection only), Coulomb constant 1 / (4 pi eps_in): own images above
    # (distance 2d) and below (2(W - d)), and the partner's two images
    beta = (ein - eout) / (ein + eout)
    k = 1.0 / (4.0 * math.pi * ein)
    own = -beta * k / (2 * d) ** 2 + beta * k / (2 * (W - d)) ** 2
    r1, r2 = math.hypot(L / 2, 2 * d), math.hypot(L / 2, 2 * (W - d))
    partner = beta * k * 2 * d / r1 ** 3 - beta * k * 2 * (W - d) / r2 ** 3
    return own + partner


@pytest.mark.parametrize("ein,eout,d", [(10.0, 15.0, 4.0), (10.0, 15.0, 5.0), (15.0, 10.0, 4.0)])
def test_static_force_near_a_planar_dielectric_jump_matches_image_charges(ein, eout, d):
    # The force on a charge near a flat interface between two dielectrics is
    # that of its image charge (method of images for a planar boundary; the
    # paper compares MEMD with image-charge/ICC results for such geometries).
    # Weak contrast (|beta| = 0.2) keeps the multiple reflections below 5%;
    # the lattice (linear charge assignment, eps sampled at link midpoints
    # across a 0.5-wide tanh step) adds the rest: 25% at d = 4-5 cells.  A
    # wrong sign, a factor 2, or eps on the wrong side of the face fails.
    N, W, c = 32, 16.0, 16.0
    z = c + W / 2 - d
    x = np.array([[N / 4 + 0.5, N / 2 + 0.5, z], [3 * N / 4 + 0.5, N / 2 + 0.5, z]])
    q = np.array([1, -1], dtype=np.int32)
    o = O.OracleSystem((N,) * 3, (float(N),) * 3,
                       eps=dict(kind=O.EPS_TANH, axis=2,
                                params=(0.5 * (ein + eout), 0.5 * (eout - ein), c, W / 2, 0.5)),
                       c_light=1.0, dt=0.01, seed=1, relax_tol=1e-9)
    o.set_particles(x, q, np.ones(2), np.zeros((2, 3)))
    o.init_field()
    F = o.particles("F")
    want = image_force_z(ein, eout, d, W, N)
    assert np.sign(F[0, 2]) == np.sign(want) and np.sign(F[1, 2]) == np.sign(want)
    assert abs(F[0, 2] / want - 1.0) < 0.25 and abs(F[1, 2] / want - 1.0) < 0.25
    assert abs(F[0, 0]) < 1e-6 * abs(want) + 1e-12   # the pair's x forces cancel by symmetry


# ---------------------------------------------------------- Ewald comparison
def test_static_forces_converge_to_tinfoil_ewald():
    # The lattice force with the charge-conserving linear scheme is the exact
    # gradient of a piecewise-quadratic lattice energy (Sec. IV: one-cell
    # linear interpolation): at a fixed configuration its error against the
    # continuum is first order in a/r; averaged over sub-cell translations of
    # the whole configuration (what thermal motion does) it falls faster.
    rng = np.random.default_rng(21)
    L, eps = 8.0, 1.0
    x = refs.random_positions_min_sep(rng, 8, L, 2.5)
    q = np.array([1, -1] * 4, dtype=np.int32)
    want = refs.ewald_forces(x, q, L, eps)
    snap, avg = [], []
    for Nn in (8, 16):
        s = O.OracleSystem((Nn,) * 3, (L,) * 3, eps=dict(kind=O.EPS_CONST, params=(eps,)),
                           self_mode=O.SELF_GF, dipole_corr=1, relax_tol=1e-10)
        rs = np.random.default_rng(3)
        acc, e = np.zeros_like(want), []
        for _ in range(16):
            s.set_particles((x + rs.uniform(0, L / Nn, size=3)) % L, q)
            s.init_field()
            F = s.particles("F").copy()
            acc += F
            e.append(np.sqrt(np.sum((F - want) ** 2) / np.sum(want ** 2)))
        snap.append(np.mean(e))
        acc /= 16
        avg.append(np.sqrt(np.sum((acc - want) ** 2) / np.sum(want ** 2)))
    assert snap[0] > 1.6 * snap[1] and snap[1] < 0.15
    assert avg[0] > 2.2 * avg[1] and avg[1] < 0.05
    assert avg[1] < 0.5 * snap[1]


# ----------------------------------------------------------------- curls
def test_curl_D_is_divergence_free_exactly():
    rng = np.random.default_rng(3)
    N = (5, 6, 7)
    s = make(N, 1.0, c_light=1.0, dt=0.25)
    s.field("B")[...] = rng.integers(-1000, 1000, size=(3, 7, 6, 5))
    s.field("D")[...] = 0.0
    s.curl_D()
    D = s.field("D")
    assert np.array_equal(refs.divergence(D), np.zeros((7, 6, 5)))
    # and it is c^2 dt/a times the transpose of the circulation map
    rng2 = np.random.default_rng(4)
    E = rng2.normal(size=(3, 7, 6, 5))
    lhs = np.sum(D * E)
    rhs = 0.25 * np.sum(s.field("B") * refs.curl_circulation(E))
    assert abs(lhs - rhs) < 1e-9 * abs(rhs)


def test_curl_B_matches_circulation_definition():
    rng = np.random.default_rng(8)
    N = (4, 5, 6)
    params = (60.0, -20.0, 0.4)
    s = make(N, 0.5, eps=dict(kind=O.EPS_SIN, axis=1, params=params), c_light=1.0, dt=0.1)
    D = rng.normal(size=(3, 6, 5, 4))
    s.field("D")[...] = D
    s.field("B")[...] = 0.0
    s.curl_B()
    want = -(0.1 / 0.5) * refs.curl_circulation(D * s.field("ie"))
    assert np.max(np.abs(s.field("B") - want)) < 1e-14 * np.max(np.abs(want))


@pytest.mark.parametrize("eps", [1.0, 2.5])
def test_yee_plane_wave_amplitude(eps):
    N, a, c, dt = (16, 4, 4), 1.0, 1.0, 0.3
    s = make(N, a, eps=dict(kind=O.EPS_CONST, params=(eps,)), c_light=c, dt=dt)
    s.set_particles(np.zeros((0, 3)), np.zeros(0, dtype=np.int32))
    s.init_field()
    k = 2 * math.pi * 3 / 16
    xs = np.arange(16) * a
    D = s.field("D")
    D[...] = 0.0
    D[1] = np.cos(k * xs)[None, None, :]          # transverse D_y(x)
    for n in range(1, 41):
        s.step(1)
        amp = refs.yee_mode_amplitude(n, c, dt, a, eps, (k, 0.0, 0.0))
        assert np.max(np.abs(s.field("D")[1] - amp * np.cos(k * xs)[None, None, :])) < 1e-12


def test_vacuum_energy_conserved_with_varying_eps():
    rng = np.random.default_rng(9)
    N = (6, 5, 7)
    V = 6 * 5 * 7
    epsl = rng.uniform(2.0, 80.0, size=3 * V)
    s = make(N, 1.0, eps=dict(kind=O.EPS_LINKS, values=epsl), c_light=1.0, dt=0.2)
    s.set_particles(np.zeros((0, 3)), np.zeros(0, dtype=np.int32))
    s.init_field()
    # a random divergence-free D: c^2 dt/a curl of a random B
    s.field("B")[...] = rng.normal(size=(3, 7, 5, 6))
    s.field("D")[...] = 0.0
    s.curl_D()
    s.field("B")[...] = 0.0
    e0 = s.energy()
    E0 = e0["electric"] + e0["magnetic"]
    for _ in range(20):
        s.step(10)
        e = s.energy()
        assert abs(e["electric"] + e["magnetic"] - E0) < 1e-12 * E0
    assert e["magnetic"] > 0.01 * E0   # energy really moved into B


# ------------------------------------------------------- deposition / ledger
def test_deposition_keeps_gauss_exact_and_tracks_dipole():
    rng = np.random.default_rng(13)
    N, a = (6, 5, 4), 0.5
    L = np.array(N) * a
    n = 20
    x = rng.uniform(0, 1, size=(n, 3)) * L
    q = rng.choice([-2, -1, 1, 2], size=n).astype(np.int32)
    q[-1] -= q.sum()
    s = make(N, a)
    s.set_particles(x, q)
    s.init_field()
    img = np.zeros((n, 3), dtype=np.int32)
    P0 = refs.dipole_fixed(x, img, q, N, a)
    Lg0 = s.field("Lg").copy()
    for it in range(60):
        step = rng.uniform(-0.95, 0.95, size=(n, 3)) * a
        if it % 7 == 0:
            step[:, 0] = rng.choice([-0.999, 0.999], size=n) * a
        un = x + img * L + step
        img = np.floor(un / L).astype(np.int32)
        x = un - img * L
        s.move(x, img)
        xs, ims = s.particles("x").copy(), s.particles("img").copy()
        assert np.array_equal(refs.divergence(s.field("Lg")), refs.cic(xs, q, N, a))
        P = refs.dipole_fixed(xs, ims, q, N, a)
        dLg = (s.field("Lg") - Lg0).reshape(3, -1).sum(axis=1)
        want = -np.rint((P - P0) * refs.S / a).astype(np.int64) * refs.S ** 2
        assert np.array_equal(dLg, want)
        assert np.all(s.field("Tb") == 0)


def test_cell_jump_is_reported():
    s = make((4, 4, 4))
    s.set_particles([[0.5, 0.5, 0.5], [2.5, 2.5, 2.5]], [1, -1])
    s.init_field()
    with pytest.raises(O.OracleError):
        s.move([[2.2, 0.5, 0.5], [2.5, 2.5, 2.5]], np.zeros((2, 3), dtype=np.int32))


# ----------------------------------------------------------------- dynamics
def run_nve(dt, steps, **kw):
    from paper_1309_7859_gb300 import inputs
    sysc = inputs.plain_8()
    s = O.OracleSystem(sysc.mesh, sysc.box, c_light=sysc.c_light, dt=dt, **kw)
    s.set_particles(sysc.x, sysc.q, sysc.m, sysc.v * 0.3)
    s.init_field()
    H = [s.energy()["total"]]
    for _ in range(steps):
        s.step(1)
        H.append(s.energy()["total"])
    return np.array(H)


def test_nve_energy_bounded():
    # Sec. II: energy is conserved without the magnetic Lorentz force.  The
    # lattice force jumps where a charge crosses a cell face and the
    # corrections use the static self field, so the discrete total energy
    # fluctuates at the 1e-4 level instead of to round-off; a wrong sign or
    # factor in the current or the force makes it drift by orders more.
    T = 2.0
    dev = {}
    for dt in (0.04, 0.01):
        H = run_nve(dt, int(T / dt))
        dev[dt] = np.max(np.abs(H - H[0])) / abs(H[0])
        assert dev[dt] < 5e-4
    assert dev[0.01] < 0.5 * dev[0.04]
    H = run_nve(0.02, 100, self_mode=O.SELF_NONE, dipole_corr=0)
    assert np.max(np.abs(H - H[0])) / abs(H[0]) < 1e-3


def test_langevin_drives_charged_system_to_kT():
    # a charged system of mixed masses equilibrates its kinetic energy to
    # 3/2 N kT (the thermostat acts on the particles, the fields follow
    # through the coupled dynamics); 4000 steps at gamma = 5 average over
    # about 5000 independent samples (2% statistical error)
    from paper_1309_7859_gb300 import inputs
    sysc = inputs.plain_8()
    s = O.OracleSystem(sysc.mesh, sysc.box, dt=0.01, seed=77)
    m = np.tile([0.5, 2.0], 8)
    s.set_particles(sysc.x, sysc.q, m, np.zeros((16, 3)))
    s.init_field()
    s.step(200, thermostat=(5.0, 1.0))
    ke = []
    for _ in range(4000):
        s.step(1, thermostat=(5.0, 1.0))
        v = s.particles("v")
        ke.append(np.sum(0.5 * m[:, None] * v * v))
    assert abs(np.mean(ke) / (1.5 * 16) - 1.0) < 0.08


def free_langevin_velocities(gamma, kT, dt=0.01, n=600, burn=200, steps=4000):
    """Velocities (steps x n x 3) of uncharged particles with masses 0.25, 1
    and 4 in turn under the thermostat alone (no field force acts)."""
    rng = np.random.default_rng(5)
    x = rng.uniform(0.0, 4.0, (n, 3))
    m = np.tile([0.25, 1.0, 4.0], n // 3)
    s = O.OracleSystem((4, 4, 4), (4.0, 4.0, 4.0), dt=dt, seed=91)
    s.set_particles(x, np.zeros(n, dtype=np.int32), m, np.zeros((n, 3)))
    s.init_field()
    s.step(burn, thermostat=(gamma, kT))
    V = np.empty((steps, n, 3))
    for i in range(steps):
        s.step(1, thermostat=(gamma, kT))
        V[i] = s.particles("v")
    return V, m


def test_langevin_equipartition_for_every_mass():
    # Free particles under the velocity-Verlet Langevin scheme (friction on
    # the half-step velocity u, kick factor dt/2m on each side): per step
    # u' = (1 - gamma dt) u + (dt/m) sigma xi with sigma^2 = 2 gamma m kT/dt,
    # whose stationary variance makes the full-step velocity v = (1 -
    # gamma dt/2) u + (dt/2m) sigma xi have m <v^2> = kT exactly, for any dt
    # and any mass (textbook fluctuation-dissipation balance).  A noise
    # amplitude scaled as sqrt(2 gamma kT/(m dt)) gives kT/m^2; friction
    # without the mass gives m kT; a kT slip gives the wrong level.  Each
    # mass group averages ~10^4 independent samples (1.4% error).
    kT = 1.5
    V, m = free_langevin_velocities(gamma=2.0, kT=kT)
    for mm in (0.25, 1.0, 4.0):
        sel = m == mm
        assert abs(np.mean(mm * V[:, sel, :] ** 2) / kT - 1.0) < 0.05, mm


def test_langevin_velocity_autocorrelation_is_ornstein_uhlenbeck():
    # The same scheme's full-step velocity autocorrelation after k >= 1
    # steps is (1 - gamma dt)^(k-1) (1 - gamma dt/2), the discrete form of
    # exp(-gamma t), the same for every mass.  Friction without the mass
    # would decay at gamma/m instead (e^-0.25 or e^-4 at t = 0.5 for m = 4,
    # 0.25); a wrong gamma moves the decay for all.
    gamma, dt, k = 2.0, 0.01, 50
    V, m = free_langevin_velocities(gamma=gamma, kT=1.5, dt=dt)
    want = (1 - gamma * dt) ** (k - 1) * (1 - gamma * dt / 2)
    for mm in (0.25, 1.0, 4.0):
        sel = m == mm
        c = np.mean(V[k:, sel] * V[:-k, sel]) / np.mean(V[:, sel] ** 2)
        assert abs(c - want) < 0.03, (mm, c, want)


def test_langevin_noise_is_keyed_by_counter():
    # the noise of a step is a function of (seed, particle, step) only: two
    # systems with the same seed and state draw the same words, another seed
    # draws others
    from paper_1309_7859_gb300 import inputs
    sysc = inputs.plain_8()
    out = []
    for seed in (77, 77, 78):
        s = O.OracleSystem(sysc.mesh, sysc.box, dt=0.01, seed=seed)
        s.set_particles(sysc.x, sysc.q, sysc.m, np.zeros((16, 3)))
        s.init_field()
        s.step(5, thermostat=(1.0, 1.0))
        out.append(s.particles("v").copy())
    assert np.array_equal(out[0], out[1])
    assert not np.array_equal(out[0], out[2])


def test_fold_keeps_unfolded_position():
    # folding shifts by whole box lengths: x + img L is unchanged (exactly,
    # when the shift is exact), the result lies in [0, L), and a value that
    # rounds up to L becomes 0 in the next image
    s = make((4, 4, 4), 1.0)
    L = 4.0
    xs = np.array([[4.0, -1e-17, 7.9999], [-4.0, 3.0, 12.0 - 1e-15], [15.9, -15.9, 0.0]])
    s.set_particles(xs, [1, -1, 0])
    x, img = s.particles("x"), s.particles("img")
    assert np.all((x >= 0) & (x < L))
    assert np.allclose(x + img * L, xs, rtol=0, atol=1e-14)
    assert x[0, 1] == 0.0 and img[0, 1] == 0      # -1e-17 + 4 rounds to 4 -> 0, same image
    assert x[0, 0] == 0.0 and img[0, 0] == 1


# ------------------------------------------------------------ interface links
# Eq. (dielectric-interpolation) read as the harmonic average its text names:
# an interface link is the two media in series, 1/eps_link = (d1/eps1 +
# d2/eps2)/a.  The pins below use geometry and continuum closed forms only.
@pytest.mark.parametrize("lo,hi,a", [(2.3, 5.85, 1.0), (0.0, 2.6, 1.0), (2.0, 6.0, 1.0),
                                     (1.15, 2.925, 0.5), (0.0, 0.0, 1.0)])
def test_planar_slab_links_match_the_series_integral(lo, hi, a):
    # z-links: the mean of 1/eps over their length (exact for any plane
    # position); tangential links: the medium of their plane, both media
    # averaged on a face.  A swapped d1/d2 or an arithmetic mean fails.
    e_out, e_in, N = 2.0, 80.0, (8, 6, 8)
    s = make(N, a, eps=dict(kind=O.EPS_PLANES, axis=2, params=(e_out, e_in, lo, hi)))
    ex, ey, ez = refs.planes_layer_eps(e_out, e_in, lo, hi, N[2], a)
    ie = s.field("ie")
    assert np.allclose(1 / ie[0], ex[:, None, None], rtol=1e-14)
    assert np.allclose(1 / ie[1], ey[:, None, None], rtol=1e-14)
    assert np.allclose(1 / ie[2], ez[:, None, None], rtol=1e-14)
    # homogenised tensor: the continuum series value across the layers
    L = N[2] * a
    w = hi - lo
    assert abs(s.Minv[2, 2] - (w / e_in + (L - w) / e_out) / L) < 1e-12 * s.Minv[2, 2]
    assert abs(s.Minv[0, 0] - 1 / np.mean(ex)) < 1e-12 * s.Minv[0, 0]


def test_planar_slab_along_x_is_the_transpose_of_z():
    sx = make((8, 6, 4), 1.0, eps=dict(kind=O.EPS_PLANES, axis=0, params=(3.0, 50.0, 1.7, 4.2)))
    sz = make((4, 6, 8), 1.0, eps=dict(kind=O.EPS_PLANES, axis=2, params=(3.0, 50.0, 1.7, 4.2)))
    ix, iz = sx.field("ie"), sz.field("ie")
    assert np.array_equal(ix[0], np.transpose(iz[2], (2, 1, 0)))
    assert np.array_equal(ix[2], np.transpose(iz[0], (2, 1, 0)))


def test_planar_slab_initial_solution_matches_layered_exact():
    rng = np.random.default_rng(14)
    N, a, params = (8, 6, 8), 1.0, (2.0, 80.0, 2.3, 5.85)
    s = make(N, a, eps=dict(kind=O.EPS_PLANES, axis=2, params=params))
    x, q = neutral_system(rng, 10, N, a)
    s.set_particles(x, q)
    s.init_field()
    ex, ey, ez = refs.planes_layer_eps(*params, N[2], a)
    Qe = refs.cic(x, q, N, a).astype(np.float64) * 2.0 ** -48
    P = refs.dipole_fixed(x, np.zeros((10, 3)), q, N, a)
    want = refs.layered_solution(N, a, Qe, ex, ey, ez, -P / s.Vbox)
    assert np.max(np.abs(s.field("D") - want)) < 1e-9 * np.max(np.abs(want))


def test_slab_thinner_than_a_link_is_not_seen():
    # the interface rule compares end values: a slab between two vertices
    # changes no vertex, so no link is an interface link
    s = make((8, 8, 8), 1.0, eps=dict(kind=O.EPS_PLANES, axis=2, params=(2.0, 80.0, 0.7, 0.9)))
    assert np.all(s.field("ie") == 0.5)


@pytest.mark.parametrize("centre,r", [((7.3, 8.1, 7.6), 4.2), ((8.0, 8.0, 8.0), 5.0),
                                      ((1.5, 14.2, 0.4), 3.3)])
def test_ball_link_fractions_sum_to_chord_lengths(centre, r):
    # along every lattice line the fractions of its links inside the ball add
    # up to the chord the ball cuts from the line (Pythagoras); the integer
    # centre and radius 5 put vertices exactly on the surface (3-4-5 triples)
    N, e_out, e_in = (16, 16, 16), 2.0, 80.0
    s = make(N, 1.0, eps=dict(kind=O.EPS_SPHERE, params=(e_out, e_in) + tuple(centre) + (r,)),
             eps_eff_inv=np.eye(3))
    got, want = refs.chord_fraction_sums(s.field("ie"), e_out, e_in, centre, r, N)
    assert np.max(np.abs(got - want)) < 1e-12
    assert np.count_nonzero(want) > 100


def test_ball_with_spacing_scales_with_the_cell():
    # the same ball in a box of half the spacing gives the same link values
    p1 = (2.0, 80.0, 7.3, 8.1, 7.6, 4.2)
    p2 = (2.0, 80.0, 3.65, 4.05, 3.8, 2.1)
    s1 = make((16, 16, 16), 1.0, eps=dict(kind=O.EPS_SPHERE, params=p1), eps_eff_inv=np.eye(3))
    s2 = make((16, 16, 16), 0.5, eps=dict(kind=O.EPS_SPHERE, params=p2), eps_eff_inv=np.eye(3))
    assert np.max(np.abs(s1.field("ie") - s2.field("ie"))) < 1e-14


@pytest.mark.parametrize("r", [3.3, 4.2])
def test_ball_lattice_eps_eff_matches_maxwell_garnett(r):
    # a cubic array of dielectric balls at volume fraction f: Maxwell Garnett
    # eps_eff = eps_o (1 + 2 f b) / (1 - f b), b = (eps_i - eps_o)/(eps_i +
    # 2 eps_o) (exact to O(f^(10/3)) for the array).  With interface links the
    # excess over eps_o is within 5% at r = 3-4 cells; the plain mean of the
    # same vertex values is 30% or more off, so the pin tells them apart.
    Nn, e_out, e_in, c = 16, 2.0, 80.0, (7.3, 8.1, 7.6)
    s = make((Nn,) * 3, 1.0, eps=dict(kind=O.EPS_SPHERE, params=(e_out, e_in) + c + (r,)),
             relax_tol=1e-10)
    f = 4.0 / 3.0 * math.pi * r ** 3 / Nn ** 3
    b = (e_in - e_out) / (e_in + 2 * e_out)
    mg = e_out * (1 + 2 * f * b) / (1 - f * b) - e_out
    got = 1.0 / np.mean(np.diag(s.Minv)) - e_out
    assert abs(got / mg - 1.0) < 0.05
    assert np.max(np.abs(s.Minv - np.diag(np.diag(s.Minv)))) < 1e-3 * s.Minv[0, 0]
    k, j, i = np.meshgrid(*(np.arange(Nn),) * 3, indexing="ij")
    off = [np.mod(v - cc + Nn / 2, Nn) - Nn / 2 for v, cc in ((i, c[0]), (j, c[1]), (k, c[2]))]
    vals = np.where(off[0] ** 2 + off[1] ** 2 + off[2] ** 2 < r * r, e_in, e_out)
    m = make((Nn,) * 3, 1.0, eps=dict(kind=O.EPS_VERTICES, values=vals, params=(0.0,)),
             relax_tol=1e-10)
    assert abs((1.0 / np.mean(np.diag(m.Minv)) - e_out) / mg - 1.0) > 0.3


def cut_planes(e_out, e_in, lo, hi, N, a):
    """CUT profile of a planar slab written by hand: vertex values by plane,
    and on z-links crossing a face the distance of the face from the lower
    end as a fraction of a."""
    Nx, Ny, Nz = N
    z = np.arange(Nz) * a
    side = np.where((z > lo) & (z < hi), e_in, e_out)
    side = np.where((z == lo) | (z == hi), 0.5 * (e_in + e_out), side)
    vals = np.broadcast_to(side[:, None, None], (Nz, Ny, Nx)).astype(np.float64)
    t = -np.ones((3, Nz, Ny, Nx))
    for k in range(Nz):
        for face in (lo, hi):
            if z[k] < face < z[k] + a:
                t[2, k] = (face - z[k]) / a
    return np.concatenate([vals.ravel(), t.ravel()])


def test_cut_links_reproduce_the_series_integral():
    N, a, e_out, e_in, lo, hi = (6, 5, 8), 1.0, 2.0, 80.0, 2.3, 5.85
    s = make(N, a, eps=dict(kind=O.EPS_CUT, values=cut_planes(e_out, e_in, lo, hi, N, a)))
    ex, ey, ez = refs.planes_layer_eps(e_out, e_in, lo, hi, N[2], a)
    ie = s.field("ie")
    assert np.allclose(1 / ie[0], ex[:, None, None], rtol=1e-14)
    assert np.allclose(1 / ie[2], ez[:, None, None], rtol=1e-14)
    # no cut anywhere: the plain endpoint mean of the vertex values
    rng = np.random.default_rng(5)
    vals = rng.uniform(1.0, 40.0, size=N[::-1])
    c = make(N, a, eps=dict(kind=O.EPS_CUT, values=np.concatenate([vals.ravel(),
                                                                    -np.ones(3 * vals.size)])))
    v = make(N, a, eps=dict(kind=O.EPS_VERTICES, values=vals, params=(0.0,)))
    assert np.array_equal(c.field("ie"), v.field("ie"))


def test_vertex_threshold_marks_interface_links_at_midpoints():
    # layers whose jumps sit halfway between vertex planes: with theta = 1
    # every jump link is an interface link cut at its midpoint, which is the
    # continuum series value exactly; theta = 0 (the plain mean) is not
    N, a = (4, 4, 8), 1.0
    eps_k = np.array([2.0, 2.0, 80.0, 80.0, 80.0, 2.0, 2.0, 2.0])
    vals = np.broadcast_to(eps_k[:, None, None], N[::-1]).astype(np.float64)
    lo, hi = 1.5, 4.5
    _, _, ez = refs.planes_layer_eps(2.0, 80.0, lo, hi, N[2], a)
    on = make(N, a, eps=dict(kind=O.EPS_VERTICES, values=vals, params=(1.0,)))
    assert np.allclose(1 / on.field("ie")[2], ez[:, None, None], rtol=1e-14)
    off = make(N, a, eps=dict(kind=O.EPS_VERTICES, values=vals, params=(0.0,)))
    big = make(N, a, eps=dict(kind=O.EPS_VERTICES, values=vals, params=(100.0,)))
    assert np.array_equal(off.field("ie"), big.field("ie"))
    assert abs(1 / off.field("ie")[2, 1, 0, 0] - 41.0) < 1e-12


def test_invalid_interface_profiles_are_rejected():
    for eps in (dict(kind=O.EPS_PLANES, axis=2, params=(2.0, 80.0, 5.0, 3.0)),
                dict(kind=O.EPS_PLANES, axis=2, params=(2.0, 80.0, 1.0, 8.0)),
                dict(kind=O.EPS_PLANES, axis=3, params=(2.0, 80.0, 1.0, 3.0)),
                dict(kind=O.EPS_PLANES, axis=2, params=(0.0, 80.0, 1.0, 3.0)),
                dict(kind=O.EPS_SPHERE, params=(2.0, 80.0, 4.0, 4.0, 4.0, 3.5)),
                dict(kind=O.EPS_SPHERE, params=(2.0, 80.0, 4.0, 4.0, 4.0, 0.0)),
                dict(kind=O.EPS_VERTICES, values=np.ones(512), params=(-1.0,)),
                dict(kind=O.EPS_CUT, params=())):
        with pytest.raises(O.OracleError):
            make((8, 8, 8), 1.0, eps=eps)


@pytest.mark.parametrize("ein,eout,c", [(10.0, 15.0, 16.3), (15.0, 10.0, 16.3),
                                        (10.0, 15.0, 15.7)])
def test_sharp_planar_faces_give_the_image_charge_force(ein, eout, c):
    # faces off the lattice planes, the charge 4 cells below the upper face:
    # first-reflection image force within 10% (the weak contrast keeps the
    # higher reflections near 4%)
    N, W, d = 32, 16.0, 4.0
    z = c + W / 2 - d
    x = np.array([[N / 4 + 0.5, N / 2 + 0.5, z], [3 * N / 4 + 0.5, N / 2 + 0.5, z]])
    o = O.OracleSystem((N,) * 3, (float(N),) * 3,
                       eps=dict(kind=O.EPS_PLANES, axis=2, params=(eout, ein, c - W / 2, c + W / 2)),
                       c_light=1.0, dt=0.01, seed=1, relax_tol=1e-9)
    o.set_particles(x, np.array([1, -1], dtype=np.int32), np.ones(2), np.zeros((2, 3)))
    o.init_field()
    F = o.particles("F")
    want = image_force_z(ein, eout, d, W, N)
    assert abs(F[0, 2] / want - 1.0) < 0.10 and abs(F[1, 2] / want - 1.0) < 0.10


# ---------------------------------------------------- moving the permittivity
def test_set_eps_keeps_D_and_maps_like_a_fresh_system():
    rng = np.random.default_rng(31)
    N, a = (8, 6, 8), 1.0
    first = dict(kind=O.EPS_TANH, axis=2, params=(41.0, 39.0, 4.0, 2.0, 1.5))
    then = dict(kind=O.EPS_SPHERE, params=(2.0, 80.0, 4.1, 2.9, 3.6, 1.8))
    s = make(N, a, eps=first, relax_tol=1e-11)
    x, q = neutral_system(rng, 10, N, a)
    s.set_particles(x, q)
    s.init_field()
    s.step(5)
    D0, B0 = s.field("D").copy(), s.field("B").copy()
    s.set_eps(then)
    fresh = make(N, a, eps=then, relax_tol=1e-11)
    assert np.array_equal(s.field("ie"), fresh.field("ie"))
    assert np.array_equal(s.Minv, fresh.Minv)
    assert np.array_equal(s.field("D"), D0) and np.array_equal(s.field("B"), B0)
    e = s.energy()
    assert e["gauss_exact"] == 1.0
    # the electric energy now weighs the same D with the new 1/eps
    assert abs(e["electric"] - 0.5 * a ** 3 * np.sum(D0 ** 2 * fresh.field("ie"))) < \
        1e-12 * e["electric"]


def test_set_eps_with_relaxation_is_the_fresh_electrostatic_minimum():
    # after a few steps, re-relaxing under a new profile reaches the unique
    # minimum for the present charges and dipole: the same field as a fresh
    # system initialised at the present positions
    rng = np.random.default_rng(32)
    N, a = (8, 6, 8), 1.0
    then = dict(kind=O.EPS_PLANES, axis=1, params=(3.0, 30.0, 1.4, 3.9))
    s = make(N, a, eps=dict(kind=O.EPS_CONST, params=(2.0,)), relax_tol=1e-11)
    x, q = neutral_system(rng, 10, N, a)
    s.set_particles(x, q, v=rng.normal(size=(10, 3)))
    s.init_field()
    s.step(20)
    s.set_eps(then, relax=True)
    fresh = make(N, a, eps=then, relax_tol=1e-11)
    fresh.set_particles(s.particles("x"), q, img=s.particles("img"))
    fresh.init_field()
    D, Df = s.field("D"), fresh.field("D")
    assert np.max(np.abs(D - Df)) < 1e-9 * np.max(np.abs(Df))
    assert np.all(s.field("B") == 0.0)
    assert np.max(np.abs(s.particles("F") - fresh.particles("F"))) < \
        1e-8 * np.max(np.abs(fresh.particles("F")))
    assert s.step_count == 20


def test_set_eps_failure_leaves_the_system_unchanged():
    s = make((8, 8, 8), 1.0, eps=dict(kind=O.EPS_CONST, params=(3.0,)))
    ie0, M0 = s.field("ie").copy(), s.Minv
    with pytest.raises(O.OracleError):
        s.set_eps(dict(kind=O.EPS_LINKS, values=-np.ones(3 * 512)))
    assert np.array_equal(s.field("ie"), ie0) and np.array_equal(s.Minv, M0)


# ------------------------------------------- permittivity from salt density
# Reading of Sec. I (eps falls with the local salt content; the paper gives
# no rule): |q| cloud-in-cell density at the vertices, periodic Gaussian
# smoothing, eps = eps0 + slope (rho / mean - 1) clamped, applied as vertex
# values.  Pinned by a uniform density, the convolution theorem, an exact
# profile through the map and clamps, and the salt-modulated workload.
def _gauss_kernel(sigma, N):
    R = int(np.ceil(3 * sigma))
    j = np.arange(-R, R + 1)
    w = np.exp(-(j * j) / (2 * sigma * sigma))
    w /= w.sum()
    k = np.zeros(N)
    np.add.at(k, j % N, w)           # the truncated kernel folded onto a periodic axis
    return k


def test_uniform_salt_density_gives_eps0_everywhere():
    # one unit charge at every cell centre (a checkerboard of signs): each
    # vertex receives 8 x 1/8 of |q|, exactly 1, so eps = eps0 at every vertex
    N = (6, 4, 8)
    cells = np.stack(np.meshgrid(*[np.arange(n) for n in N], indexing="ij"), -1).reshape(-1, 3)
    x = cells + 0.5
    q = np.where(cells.sum(axis=1) % 2 == 0, 1, -1).astype(np.int32)
    for sigma in (0.0, 1.5):
        s = make(N, 1.0)
        s.set_particles(x, q)
        e = s.eps_from_density(55.0, -30.0, 40.0, 80.0, sigma)
        assert np.all(e == 55.0)
        assert np.allclose(s.field("ie"), 1 / 55.0, rtol=1e-15)


def test_salt_smoothing_is_a_periodic_convolution():
    # direct periodic sums along x, y, z against the convolution theorem
    # (product of discrete Fourier transforms) with the same folded kernel;
    # the smoothing keeps the mean
    rng = np.random.default_rng(21)
    N = (10, 7, 9)
    rho = rng.uniform(0.0, 2.0, size=(N[2], N[1], N[0]))
    for sigma in (0.7, 1.3, 2.6):       # 2.6: the kernel is wider than the 7-cell axis
        got = O.smooth_periodic(N, sigma, rho).reshape(rho.shape)
        F = np.fft.fftn(rho)
        for ax, n in zip((2, 1, 0), N):
            shape = [1, 1, 1]
            shape[ax] = n
            F = F * np.fft.fft(_gauss_kernel(sigma, n)).reshape(shape)
        want = np.real(np.fft.ifftn(F))
        assert np.max(np.abs(got - want)) < 1e-13
        assert abs(got.mean() - rho.mean()) < 1e-14


def test_salt_map_and_clamps_on_an_exact_profile():
    # valences on the vertices (sub-cell step 0: all weight on one vertex) give
    # an exact integer density along x; eps follows the linear map and clamps
    N = (12, 3, 2)
    L = float(N[0])
    xs, qs = [], []
    prof = np.round(100 * (2 + np.cos(2 * np.pi * np.arange(N[0]) / L))).astype(int)
    for i in range(N[0]):
        for j in range(N[1]):
            for k in range(N[2]):
                xs += [[i, j, k], [i, j, k]]
                qs += [prof[i], -prof[i]]      # a neutral pair at each vertex
    s = make(N, 1.0)
    s.set_particles(np.array(xs, dtype=float), np.array(qs, dtype=np.int32))
    e = s.eps_from_density(60.0, -45.0, 42.0, 78.0, 0.0)
    rho = 2.0 * prof
    want = np.clip(60.0 - 45.0 * (rho / rho.mean() - 1.0), 42.0, 78.0)
    assert np.array_equal(e, np.broadcast_to(want, e.shape))
    assert want.min() == 42.0 and want.max() == 78.0         # both clamps reached
    assert np.any((want > 42.0) & (want < 78.0))            # and the map between them


def test_salt_rule_reproduces_the_modulated_profile():
    # the salt-modulated workload's charges (density 1 + 0.5 sin(2 pi x / L))
    # through eps0 = 60, slope -40, sigma 2: the vertex eps follows
    # 60 - 20 H sin(2 pi x / L), H = exp(-(sigma k)^2 / 2) the attenuation of
    # the smoothing at that wave number, up to sampling noise
    from paper_1309_7859_gb300 import inputs
    N, n, sigma = 32, 8000, 2.0
    rng = np.random.default_rng(5)
    x = inputs.sine_modulated_positions(rng, n, (float(N),) * 3, 0, 0.5)
    q = inputs.neutral_charges(rng, n)
    s = make((N, N, N), 1.0, eps_eff_inv=np.eye(3) / 60.0)
    s.set_particles(x, q)
    e = s.eps_from_density(60.0, -40.0, 40.0, 80.0, sigma)
    prof = e.mean(axis=(0, 1))                       # along x
    sx = np.sin(2 * np.pi * np.arange(N) / N)
    amp = 2 * np.mean(prof * sx)
    H = np.exp(-(sigma * 2 * np.pi / N) ** 2 / 2)
    assert abs(prof.mean() - 60.0) < 0.5
    assert abs(amp - (-20.0 * H)) < 2.0
