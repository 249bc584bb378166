"""Seeded synthetic inputs for MEMD runs.

This module only draws random numbers and states profile parameters: it holds
none of the method's arithmetic (no link mapping, no charge assignment, no
field update), so both the CUDA library's tests and the oracle may use it.

The workloads mirror the shapes of the paper's test systems (random
electrolytes in a periodic box, a low-permittivity slab in water-like
surroundings, a salt-modulated permittivity, many independent systems, a
stream of requests); the paper's own datasets are not available, so every
system is synthetic.  Seeds are 1000 + workload index; replica or request r
of a batched workload uses seed * 2**16 + r.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class EpsSpec:
    """Permittivity profile: kind is one of 'const', 'links', 'vertices',
    'tanh', 'sin', 'planes', 'sphere', 'cut'.  tanh: eps = p0 + p1 tanh((|s -
    p2| - p3) / p4) with s the periodic distance along `axis`; sin: eps = p0 +
    p1 sin(2 pi s / L + p2); planes: p1 between s = p2 and s = p3 along `axis`,
    p0 elsewhere; sphere: p1 within p5 of (p2, p3, p4), p0 outside; cut:
    vertex values then per-link cut fractions; vertices: params[0] is the
    interface threshold (0: none)."""
    kind: str = "const"
    axis: int = 0
    params: tuple = (1.0,)
    values: np.ndarray | None = None


@dataclass
class System:
    name: str
    mesh: tuple
    box: tuple
    eps: EpsSpec
    c_light: float
    dt: float
    precision: str          # "fp64" or "fp32" link/plaquette fields
    x: np.ndarray           # (n, 3) positions in [0, L)
    q: np.ndarray           # (n,) integer valences
    m: np.ndarray           # (n,) masses
    v: np.ndarray           # (n, 3) velocities
    steps: int
    thermostat: tuple | None = (1.0, 1.0)   # (gamma, kT) or None for NVE
    seed: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def n(self):
        return int(self.q.shape[0])

    @property
    def sites(self):
        return int(np.prod(self.mesh))


def neutral_charges(rng, n):
    """n valences +-1 with total zero (n even): half +1, half -1, shuffled."""
    if n % 2:
        raise ValueError("neutral +-1 systems need an even particle count")
    q = np.concatenate([np.ones(n // 2, np.int32), -np.ones(n // 2, np.int32)])
    rng.shuffle(q)
    return q


def thermal_velocities(rng, n, kT=1.0, m=1.0):
    return rng.normal(0.0, math.sqrt(kT / m), size=(n, 3))


def uniform_positions(rng, n, box):
    return rng.uniform(0.0, 1.0, size=(n, 3)) * np.asarray(box, dtype=np.float64)


def sine_modulated_positions(rng, n, box, axis=0, amp=0.5):
    """Rejection sampling of density proportional to 1 + amp sin(2 pi s / L)."""
    box = np.asarray(box, dtype=np.float64)
    out = np.empty((0, 3))
    while out.shape[0] < n:
        cand = rng.uniform(0.0, 1.0, size=(2 * n, 3)) * box
        acc = rng.uniform(0.0, 1.0 + amp, size=2 * n)
        dens = 1.0 + amp * np.sin(2.0 * np.pi * cand[:, axis] / box[axis])
        out = np.concatenate([out, cand[acc < dens]])
    return out[:n]


def smooth_random_vertices(rng, mesh, sigma_cells=2.0, lo=2.0, hi=80.0):
    """Gaussian-filtered (periodic, sigma in cells) white noise at the vertices,
    rescaled to [lo, hi].  Array shape (Nz, Ny, Nx)."""
    Nx, Ny, Nz = mesh
    white = rng.normal(size=(Nz, Ny, Nx))
    kz = np.fft.fftfreq(Nz)[:, None, None]
    ky = np.fft.fftfreq(Ny)[None, :, None]
    kx = np.fft.fftfreq(Nx)[None, None, :]
    filt = np.exp(-2.0 * (np.pi * sigma_cells) ** 2 * (kx ** 2 + ky ** 2 + kz ** 2))
    sm = np.real(np.fft.ifftn(np.fft.fftn(white) * filt))
    sm = (sm - sm.min()) / max(sm.max() - sm.min(), 1e-300)
    return lo + (hi - lo) * sm


def _system(name, mesh, n, eps, dt, precision, steps, seed, c_light=1.0,
            positions=None, thermostat=(1.0, 1.0)):
    rng = np.random.default_rng(seed)
    box = tuple(float(N) for N in mesh)  # lattice spacing a = 1
    q = neutral_charges(rng, n)
    x = uniform_positions(rng, n, box) if positions is None else positions(rng, n, box)
    v = thermal_velocities(rng, n)
    return System(name=name, mesh=tuple(mesh), box=box, eps=eps, c_light=c_light, dt=dt,
                  precision=precision, x=x, q=q, m=np.ones(n), v=v, steps=steps,
                  thermostat=thermostat, seed=seed)


def plain_8(seed=1000):
    """Plain MEMD: 8^3, L = 8, eps = 1, 16 charges (8 +, 8 -), Langevin kT = 1,
    c = 1, dt = 0.01, 100 steps, FP64 fields."""
    return _system("plain-8^3-eps1-16q-fp64", (8, 8, 8), 16, EpsSpec("const", 0, (1.0,)),
                   0.01, "fp64", 100, seed)


def slab_32(seed=1001, precision="fp32"):
    """Inhomogeneous slab: 32^3, L = 32, 1000 charges,
    eps(z) = 41 + 39 tanh((|z - 16| - 8) / 1.5), dt = 0.005, 1000 steps."""
    eps = EpsSpec("tanh", 2, (41.0, 39.0, 16.0, 8.0, 1.5))
    return _system("slab-32^3-1000q", (32, 32, 32), 1000, eps, 0.005, precision, 1000, seed)


def salt_64(seed=1002, precision="fp32"):
    """Salt-dependent dielectric: 64^3, L = 64, 32768 charges with density
    1 + 0.5 sin(2 pi x / L), eps(x) = 60 - 20 sin(2 pi x / L) in [40, 80],
    2000 steps."""
    eps = EpsSpec("sin", 0, (60.0, -20.0, 0.0))
    return _system("salt-64^3-32768q", (64, 64, 64), 32768, eps, 0.005, precision, 2000,
                   seed, positions=lambda r, n, b: sine_modulated_positions(r, n, b, 0, 0.5))


def random_slab_eps(rng, N):
    axis = int(rng.integers(0, 3))
    centre = float(rng.uniform(0.0, N))
    half = float(rng.uniform(N / 8.0, N / 4.0))
    e_in, e_out = (float(t) for t in rng.uniform(2.0, 80.0, size=2))
    return EpsSpec("tanh", axis, (0.5 * (e_in + e_out), 0.5 * (e_out - e_in), centre, half, 1.5))


def log_uniform_even(rng, lo, hi):
    n = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
    return max(2, n - (n % 2))


def batch_replicas(seed=1003, count=64, meshes=(16, 24, 32, 48), nmin=200, nmax=8000,
                   steps=500, precision="fp32"):
    """Batched replicas: meshes from {16,24,32,48}^3 (L = N), 200-8000 charges
    (log-uniform), a random tanh slab per replica (eps 2-80), 500 steps."""
    rng = np.random.default_rng(seed)
    out = []
    for r in range(count):
        N = int(rng.choice(meshes))
        n = log_uniform_even(rng, nmin, nmax)
        eps = random_slab_eps(rng, N)
        out.append(_system(f"replica{r}-{N}^3-{n}q", (N, N, N), n, eps, 0.005, precision,
                           steps, seed * 65536 + r))
    return out


def served_stream(seed=1004, count=512, nmin_mesh=16, nmax_mesh=96, qmin=100, qmax=50000,
                  smin=200, smax=5000, precision="fp32"):
    """Served stream: mesh N uniform in {16..96} (L = N), 100-50000 charges
    (log-uniform, capped at 0.5 per site), smooth random eps at the vertices in
    [2, 80], 200-5000 steps (log-uniform).  Arrival times are drawn by the
    caller from a Poisson process."""
    rng = np.random.default_rng(seed)
    out = []
    for r in range(count):
        N = int(rng.integers(nmin_mesh, nmax_mesh + 1))
        n = min(log_uniform_even(rng, qmin, qmax), (N ** 3) // 2 // 2 * 2)
        steps = int(round(math.exp(rng.uniform(math.log(smin), math.log(max(smax, smin))))))
        vals = smooth_random_vertices(np.random.default_rng(seed * 65536 + r), (N, N, N))
        eps = EpsSpec("vertices", 0, (), vals)
        out.append(_system(f"request{r}-{N}^3-{n}q", (N, N, N), n, eps, 0.005, precision,
                           steps, seed * 65536 + r))
    return out


def big_slab(N=256, n=100000, seed=1005, steps=200, precision="fp32"):
    """Large single system to show the field stencils against HBM bandwidth:
    N^3 with a random slab, 1e5 charges."""
    rng = np.random.default_rng(seed)
    eps = random_slab_eps(rng, N)
    return _system(f"bigslab-{N}^3-{n}q", (N, N, N), n, eps, 0.005, precision, steps, seed)


def fibonacci_sphere(n, radius, centre):
    """n nearly uniform points on a sphere (golden-angle spiral)."""
    k = np.arange(n, dtype=np.float64) + 0.5
    z = 1.0 - 2.0 * k / n
    r = np.sqrt(1.0 - z * z)
    phi = k * math.pi * (3.0 - math.sqrt(5.0))
    pts = np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)
    return np.asarray(centre, dtype=np.float64) + radius * pts


def outside_ball(rng, n, box, centre, radius):
    """n uniform positions in the box farther than `radius` from `centre`
    (periodic distance)."""
    box = np.asarray(box, dtype=np.float64)
    out = np.empty((0, 3))
    while out.shape[0] < n:
        cand = rng.uniform(0.0, 1.0, size=(2 * n + 16, 3)) * box
        d = cand - centre
        d -= box * np.round(d / box)
        out = np.concatenate([out, cand[np.sum(d * d, axis=1) > radius * radius]])
    return out[:n]


def salt_pairs(mM, box_cells, cell_nm):
    """ion pairs of a 1:1 salt at `mM` millimol per litre in a box of
    box_cells cells of edge cell_nm nanometres (1 mol/l = 0.6022 per nm^3)."""
    volume_nm3 = float(np.prod(box_cells)) * cell_nm ** 3
    return int(round(mM * 1e-3 * 0.602214076 * volume_nm3))


def colloid(N=64, seed=1006, precision="fp32", Qc=60, salt_mM=50.0, cell_nm=1.0,
            eps_in=2.0, eps_out=80.0, heavy=1e12, steps=2000):
    """Dielectric colloid in salt water (the dynamic-sphere validation system
    of the paper, with our own parameters, which the text does not give): a
    ball of eps_in = 2 and radius N/8 at the box centre in water of eps_out =
    80, with sharp interface links; its charge Qc as Qc unit charges fixed
    half a cell inside its surface (mass `heavy`: their thermal speed
    sqrt(kT/m) is 1e-6, so a step moves them by ~5e-9 cells); Qc monovalent
    counterions and 1:1 salt at 50 mmol/l (a cell
    edge of 1 nm) placed uniformly at least one cell outside the ball."""
    rng = np.random.default_rng(seed)
    box = (float(N),) * 3
    c = np.array(box) / 2.0
    R = N / 8.0
    eps = EpsSpec("sphere", 0, (eps_out, eps_in, c[0], c[1], c[2], R))
    pairs = salt_pairs(salt_mM, (N, N, N), cell_nm)
    surf = fibonacci_sphere(Qc, R - 0.5, c)
    ions = outside_ball(rng, Qc + 2 * pairs, box, c, R + 1.0)
    x = np.concatenate([surf, ions])
    q = np.concatenate([np.ones(Qc, np.int32), -np.ones(Qc, np.int32),
                        neutral_charges(rng, 2 * pairs)])
    m = np.concatenate([np.full(Qc, heavy), np.ones(Qc + 2 * pairs)])
    v = np.concatenate([np.zeros((Qc, 3)), thermal_velocities(rng, Qc + 2 * pairs)])
    return System(name=f"colloid-{N}^3-{x.shape[0]}q", mesh=(N, N, N), box=box, eps=eps,
                  c_light=1.0, dt=0.005, precision=precision, x=x, q=q, m=m, v=v,
                  steps=steps, thermostat=(1.0, 1.0), seed=seed,
                  extra=dict(Qc=Qc, radius=R, salt_pairs=pairs, heavy=Qc))


def cloud_wall(N=32, seed=1007, precision="fp32", spacing=2, n_cloud=2000, heavy=1e12,
               steps=2000):
    """Cloud-wall (the paper's third error system, our own parameters): two
    oppositely charged walls normal to z at L/4 and 3L/4, each a square grid
    of fixed unit charges `spacing` cells apart (mass `heavy`), in a neutral
    cloud of n_cloud random +-1 charges; eps = 1.  The walls give the box a
    large dipole moment and a field throughout."""
    rng = np.random.default_rng(seed)
    box = (float(N),) * 3
    g = (np.arange(N // spacing) * spacing + 0.5).astype(np.float64)
    gx, gy = np.meshgrid(g, g, indexing="ij")
    w = np.stack([gx.ravel(), gy.ravel()], axis=1)
    nw = w.shape[0]
    lo = np.concatenate([w, np.full((nw, 1), N / 4.0 + 0.5)], axis=1)
    hi = np.concatenate([w, np.full((nw, 1), 3.0 * N / 4.0 + 0.5)], axis=1)
    x = np.concatenate([lo, hi, uniform_positions(rng, n_cloud, box)])
    q = np.concatenate([np.ones(nw, np.int32), -np.ones(nw, np.int32),
                        neutral_charges(rng, n_cloud)])
    m = np.concatenate([np.full(2 * nw, heavy), np.ones(n_cloud)])
    v = np.concatenate([np.zeros((2 * nw, 3)), thermal_velocities(rng, n_cloud)])
    return System(name=f"cloud-wall-{N}^3-{x.shape[0]}q", mesh=(N, N, N), box=box,
                  eps=EpsSpec("const", 0, (1.0,)), c_light=1.0, dt=0.005, precision=precision,
                  x=x, q=q, m=m, v=v, steps=steps, thermostat=(1.0, 1.0), seed=seed,
                  extra=dict(wall_charges=nw, heavy=2 * nw))
