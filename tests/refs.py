"""Independent numpy references that pin the oracle (and through it the GPU).

Each routine is a plain definition or a textbook solution, written without
looking at the oracle's code paths: cloud-in-cell charges and the lattice
divergence by their definitions, exact lattice electrostatics by FFT
(constant eps) or by FFT in the plane plus a periodic tridiagonal solve across
the layers (eps varying along one axis), the Yee leapfrog mode amplitude in
closed form, and a tinfoil Ewald sum for point charges.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erfc

S = 1 << 16


def quantize(x, a, N):
    """cell c = floor(x/a) and sub-cell step f = floor((x/a - c) S) per axis."""
    u = np.asarray(x, dtype=np.float64) / a
    c = np.floor(u)
    f = np.floor((u - c) * S)
    c = c.astype(np.int64)
    f = f.astype(np.int64)
    N = np.asarray(N, dtype=np.int64)
    hi = c >= N
    c = np.where(hi, N - 1, c)
    f = np.where(hi, S - 1, f)
    return c, f


def cic(x, q, N, a, background=True):
    """Vertex charges in units of e 2^-48: q (S - f or f) products over the 8
    corners, minus the uniform background of a non-neutral system."""
    Nx, Ny, Nz = N
    Q = np.zeros((Nz, Ny, Nx), dtype=np.int64)
    c, f = quantize(x, a, N)
    for p in range(len(q)):
        for az in (0, 1):
            for ay in (0, 1):
                for ax in (0, 1):
                    w = 1
                    for d, ad in enumerate((ax, ay, az)):
                        w *= int(f[p, d]) if ad else int(S - f[p, d])
                    Q[(c[p, 2] + az) % Nz, (c[p, 1] + ay) % Ny, (c[p, 0] + ax) % Nx] += int(q[p]) * w
    tot = int(np.sum(np.asarray(q, dtype=np.int64))) * (1 << 48)
    if background and tot:
        assert tot % (Nx * Ny * Nz) == 0
        Q -= tot // (Nx * Ny * Nz)
    return Q


def divergence(F):
    """sum_d F_d(v) - F_d(v - e_d) for link arrays shaped (3, Nz, Ny, Nx)."""
    return (F[0] - np.roll(F[0], 1, axis=2)) + (F[1] - np.roll(F[1], 1, axis=1)) + \
           (F[2] - np.roll(F[2], 1, axis=0))


def curl_circulation(E):
    """circulation of a link field around each plaquette (d, v), shape (3, Nz, Ny, Nx):
    normal x: E_y(v) + E_z(v+y) - E_y(v+z) - E_z(v), and cyclic."""
    Ex, Ey, Ez = E
    sh = lambda A, d: np.roll(A, -1, axis=2 - d)  # value at v + e_d
    cx = Ey + sh(Ez, 1) - sh(Ey, 2) - Ez
    cy = Ez + sh(Ex, 2) - sh(Ez, 0) - Ex
    cz = Ex + sh(Ey, 0) - sh(Ex, 1) - Ey
    return np.stack([cx, cy, cz])


def dipole_fixed(x, img, q, N, a):
    """P_d = sum q (img L + c a + f a / S) from the fixed-point positions."""
    c, f = quantize(x, a, N)
    U = (np.asarray(img, dtype=np.int64) * np.asarray(N, dtype=np.int64) + c) * S + f
    return (np.asarray(q, dtype=np.int64)[:, None] * U).sum(axis=0).astype(np.float64) * (a / S)


def eps_at(kind, params, s, L):
    if kind == "tanh":
        dz = s - params[2]
        dz = dz - L * np.round(dz / L)
        return params[0] + params[1] * np.tanh((np.abs(dz) - params[3]) / params[4])
    if kind == "sin":
        return params[0] + params[1] * np.sin(2.0 * np.pi * s / L + params[2])
    raise ValueError(kind)


def layer_eps(kind, params, Nz, a):
    """eps of x-, y- and z-links per plane k for a profile along z."""
    L = Nz * a
    k = np.arange(Nz, dtype=np.float64)
    e_par = eps_at(kind, params, k * a, L)
    e_z = eps_at(kind, params, (k + 0.5) * a, L)
    return e_par, e_par.copy(), e_z


def planes_layer_eps(e_out, e_in, lo, hi, Nz, a):
    """Link eps per plane k for a slab of e_in between the planes z = lo and
    z = hi (0 <= lo <= hi < Nz a) in e_out.  Tangential links lie in plane k:
    the medium there, or the mean of both media on a face.  A z-link from
    plane k to k + 1 takes the mean of 1/eps along its length (the two media
    in series), from the overlap of the link with the slab."""
    k = np.arange(Nz, dtype=np.float64)
    z = k * a
    if lo == hi:
        e_par = np.full(Nz, e_out)
    else:
        e_par = np.where((z > lo) & (z < hi), e_in, e_out)
        e_par = np.where((z == lo) | (z == hi), 0.5 * (e_in + e_out), e_par)
    inside = np.clip(np.minimum(z + a, hi) - np.maximum(z, lo), 0.0, a)
    inv = (inside / e_in + (a - inside) / e_out) / a
    return e_par, e_par.copy(), 1.0 / inv


def chord_fraction_sums(ie, e_out, e_in, centre, r, N):
    """Per lattice line along each axis: the summed fraction of its links
    inside a ball, read back from 1/eps (a link's 1/eps is the mix of the
    two media by the fraction of its length in each), and the chord length
    the ball cuts from that line (zero when no vertex lies strictly inside
    the chord).  Lengths in cells; centre and r in cells."""
    f = (ie - 1.0 / e_out) / (1.0 / e_in - 1.0 / e_out)
    got, want = [], []
    Nx, Ny, Nz = N
    for d in range(3):
        others = [e for e in range(3) if e != d]
        n = N[d]
        for i in range(N[others[0]]):
            for j in range(N[others[1]]):
                idx = [slice(None)] * 3
                # arrays are [z, y, x]; axis e sits at position 2 - e
                idx[2 - others[0]] = i
                idx[2 - others[1]] = j
                line = f[d][tuple(idx)]
                o0 = i - centre[others[0]]
                o0 -= N[others[0]] * round(o0 / N[others[0]])
                o1 = j - centre[others[1]]
                o1 -= N[others[1]] * round(o1 / N[others[1]])
                rho2 = o0 * o0 + o1 * o1
                chord = 0.0
                if rho2 < r * r:
                    h = math.sqrt(r * r - rho2)
                    ks = [k for k in range(-n, 2 * n) if abs(k - centre[d]) < h]
                    chord = 2 * h if ks else 0.0
                got.append(float(line.sum()))
                want.append(chord)
    return np.array(got), np.array(want)


def layered_solution(N, a, Qe, ex, ey, ez, Dbar):
    """Exact curl-free lattice field with div D = Qe / a^2 (flux form) and mean
    D = Dbar, for eps varying only with the plane index k.  Returns D shaped
    (3, Nz, Ny, Nx).  In-plane Fourier modes give periodic tridiagonal systems
    across the planes; the in-plane mean mode is solved directly."""
    Nx, Ny, Nz = N
    Qh = np.fft.fft2(Qe, axes=(1, 2))
    phih = np.zeros_like(Qh)
    kx = 2 * np.pi * np.arange(Nx) / Nx
    ky = 2 * np.pi * np.arange(Ny) / Ny
    for my in range(Ny):
        for mx in range(Nx):
            if mx == 0 and my == 0:
                continue
            sx = 4 * math.sin(kx[mx] / 2) ** 2
            sy = 4 * math.sin(ky[my] / 2) ** 2
            A = np.zeros((Nz, Nz))
            for k in range(Nz):
                A[k, k] += ex[k] * sx + ey[k] * sy + ez[k] + ez[k - 1]
                A[k, (k + 1) % Nz] -= ez[k]
                A[k, (k - 1) % Nz] -= ez[k - 1]
            phih[:, my, mx] = np.linalg.solve(A, Qh[:, my, mx] / a)
    phi = np.real(np.fft.ifft2(phih, axes=(1, 2)))
    grad = lambda ax: (np.roll(phi, -1, axis=ax) - phi) / a
    hx = Dbar[0] / np.mean(ex)
    hy = Dbar[1] / np.mean(ey)
    Dx = ex[:, None, None] * (-grad(2) + hx)
    Dy = ey[:, None, None] * (-grad(1) + hy)
    qbar = Qe.mean(axis=(1, 2))            # per-vertex mean charge of each plane
    dz = np.cumsum(qbar) / a ** 2
    dz = dz - dz.mean() + Dbar[2]
    Dz = ez[:, None, None] * (-grad(0)) + dz[:, None, None]
    return np.stack([Dx, Dy, Dz])


def fft_solution_const(N, a, Qe, eps, Dbar):
    """Exact lattice field for constant eps by a full 3-d FFT of the 7-point
    Laplacian: -eps a sum_d (phi(v+e_d) - 2 phi(v) + phi(v-e_d)) = Qe."""
    Nx, Ny, Nz = N
    kz = 2 * np.pi * np.fft.fftfreq(Nz)[:, None, None]
    ky = 2 * np.pi * np.fft.fftfreq(Ny)[None, :, None]
    kx = 2 * np.pi * np.fft.fftfreq(Nx)[None, None, :]
    lam = 4 * (np.sin(kx / 2) ** 2 + np.sin(ky / 2) ** 2 + np.sin(kz / 2) ** 2)
    lam[0, 0, 0] = 1.0
    ph = np.fft.fftn(Qe) / (eps * a * lam)
    ph[0, 0, 0] = 0.0
    phi = np.real(np.fft.ifftn(ph))
    D = []
    for d, ax in enumerate((2, 1, 0)):
        D.append(eps * (-(np.roll(phi, -1, axis=ax) - phi) / a) + Dbar[d])
    return np.stack(D)


def lattice_green_fft(N):
    """G on the whole periodic lattice by inverse FFT of 1 / sum 4 sin^2(k/2),
    k = 0 removed; G[z, y, x]."""
    Nx, Ny, Nz = N
    kz = 2 * np.pi * np.fft.fftfreq(Nz)[:, None, None]
    ky = 2 * np.pi * np.fft.fftfreq(Ny)[None, :, None]
    kx = 2 * np.pi * np.fft.fftfreq(Nx)[None, None, :]
    lam = 4 * (np.sin(kx / 2) ** 2 + np.sin(ky / 2) ** 2 + np.sin(kz / 2) ** 2)
    lam[0, 0, 0] = np.inf
    return np.real(np.fft.ifftn(1.0 / lam))


def yee_mode_amplitude(nsteps, c, dt, a, eps, k_vec):
    """Amplitude of a transverse lattice mode after n leapfrog steps started
    with B = 0:  cos((n + 1/2) theta) / cos(theta / 2), where
    sin(theta / 2) = (c dt / (a sqrt(eps))) sqrt(sum_d sin^2(k_d a / 2))."""
    s = c * dt / (a * math.sqrt(eps)) * math.sqrt(sum(math.sin(k * a / 2) ** 2 for k in k_vec))
    th = 2 * math.asin(s)
    return math.cos((nsteps + 0.5) * th) / math.cos(th / 2)


def ewald_forces(x, q, L, eps=1.0, tol=1e-12):
    """Tinfoil Ewald forces for point charges in a cubic periodic box, potential
    q / (4 pi eps r)."""
    x = np.asarray(x, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    n = len(q)
    rc = L / 2
    alpha = math.sqrt(-math.log(tol)) / rc
    F = np.zeros((n, 3))
    shifts = np.array([[i, j, k] for i in (-1, 0, 1) for j in (-1, 0, 1) for k in (-1, 0, 1)],
                      dtype=np.float64) * L
    for i in range(n):
        for j in range(n):
            r = x[i] - x[j]
            r = r - L * np.round(r / L)
            for sft in shifts:
                rr = r + sft
                d = math.sqrt(rr @ rr)
                if d == 0.0 or d > rc:
                    continue
                g = erfc(alpha * d) / d ** 2 + 2 * alpha / math.sqrt(math.pi) * math.exp(-(alpha * d) ** 2) / d
                F[i] += q[i] * q[j] * g * rr / d / (4 * math.pi * eps)
    kmax = int(math.ceil(2 * alpha * math.sqrt(-math.log(tol)) * L / (2 * math.pi)))
    m = np.arange(-kmax, kmax + 1)
    K = np.stack(np.meshgrid(m, m, m, indexing="ij"), axis=-1).reshape(-1, 3) * (2 * math.pi / L)
    K = K[np.any(K != 0, axis=1)]
    k2 = np.sum(K * K, axis=1)
    w = np.exp(-k2 / (4 * alpha ** 2)) / k2
    phase = x @ K.T                        # (n, nk)
    Sk = (q[:, None] * np.exp(1j * phase)).sum(axis=0)
    im = np.imag(np.exp(1j * phase) * np.conj(Sk)[None, :])   # (n, nk)
    F += (q[:, None] / (eps * L ** 3)) * ((im * w[None, :]) @ K)
    return F


def random_positions_min_sep(rng, n, L, min_sep):
    pts = []
    while len(pts) < n:
        p = rng.uniform(0, L, size=3)
        ok = True
        for o in pts:
            r = p - o
            r -= L * np.round(r / L)
            if math.sqrt(r @ r) < min_sep:
                ok = False
                break
        if ok:
            pts.append(p)
    return np.array(pts)
