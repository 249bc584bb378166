"""Python handle on the FP64 CPU oracle of MEMD (oracle/memd_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg load this module; the product path never does.  It compiles the
C oracle with gcc (no CUDA, no code shared with the library) and exposes its
arrays as numpy views.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "memd_oracle.c")
_HDR = os.path.join(_HERE, "memd_oracle.h")
_OUT = os.path.join(_HERE, "_build", "libmemd_oracle.so")
_lock = threading.Lock()
_lib = None

S = 1 << 16

EPS_CONST, EPS_LINKS, EPS_VERTICES, EPS_TANH, EPS_SIN = 0, 1, 2, 3, 4
EPS_PLANES, EPS_SPHERE, EPS_CUT = 5, 6, 7
SELF_NONE, SELF_GF, SELF_DIRECT = 0, 1, 2
OK, ERR_INVALID, ERR_COURANT, ERR_OOM, ERR_CELL_JUMP = 0, 1, 2, 3, 5
ERR_RELAX_NOCONV, ERR_OVERFLOW = 7, 11

(A_IE, A_D, A_B, A_LG, A_TB, A_X, A_V, A_IMG, A_Q, A_M, A_F, A_FT, A_G,
 A_MINV) = range(14)
ENERGY_KEYS = ("kinetic", "electric", "magnetic", "self", "dipole", "total",
               "P0", "P1", "P2", "gauss_residual", "gauss_exact")


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build (plain gcc, FP64, no FMA contraction)."""
    with _lock:
        newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
        if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= newest:
            return _OUT
        os.makedirs(os.path.dirname(_OUT), exist_ok=True)
        tmp = _OUT + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _OUT)
        return _OUT


class _Eps(C.Structure):
    _fields_ = [("kind", C.c_int32), ("axis", C.c_int32),
                ("values", C.POINTER(C.c_double)), ("params", C.c_double * 8)]


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        i32p, f64p, i64p = (C.POINTER(C.c_int32), C.POINTER(C.c_double),
                            C.POINTER(C.c_int64))
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [i32p, f64p, C.POINTER(_Eps), C.c_double, C.c_double,
                                 C.c_int32, C.c_int32, C.c_double, C.c_int32,
                                 C.c_double, C.c_uint64, f64p, i32p]
        L.orc_destroy.argtypes = [C.c_void_p]
        for f in ("orc_nsites", "orc_nparticles", "orc_stepcount"):
            getattr(L, f).restype = C.c_int64
            getattr(L, f).argtypes = [C.c_void_p]
        L.orc_ptr.restype = C.c_void_p
        L.orc_ptr.argtypes = [C.c_void_p, C.c_int32]
        L.orc_scalar.restype = C.c_double
        L.orc_scalar.argtypes = [C.c_void_p, C.c_int32]
        L.orc_set_particles.restype = C.c_int32
        L.orc_set_particles.argtypes = [C.c_void_p, C.c_int64, f64p, i32p, f64p, i32p, f64p]
        L.orc_init_field.restype = C.c_int32
        L.orc_init_field.argtypes = [C.c_void_p]
        L.orc_step.restype = C.c_int32
        L.orc_step.argtypes = [C.c_void_p, C.c_int64, C.c_int32, C.c_double, C.c_double]
        L.orc_move.restype = C.c_int32
        L.orc_move.argtypes = [C.c_void_p, f64p, i32p]
        L.orc_gather.argtypes = [C.c_void_p]
        L.orc_energy.argtypes = [C.c_void_p, f64p]
        L.orc_relax.restype = C.c_int32
        L.orc_relax.argtypes = [C.c_void_p, C.c_double, C.c_int32, i32p]
        L.orc_set_eps.restype = C.c_int32
        L.orc_set_eps.argtypes = [C.c_void_p, C.POINTER(_Eps), C.c_int32]
        L.orc_cic_charges.argtypes = [C.c_void_p, i64p]
        L.orc_eps_from_density.restype = C.c_int32
        L.orc_eps_from_density.argtypes = [C.c_void_p, f64p, C.c_int32, f64p]
        L.orc_smooth_periodic.argtypes = [i32p, C.c_double, f64p]
        L.orc_salt_vertex_eps.restype = C.c_int32
        L.orc_salt_vertex_eps.argtypes = [C.c_void_p, f64p, f64p]
        L.orc_gauss_scan.restype = C.c_int32
        L.orc_gauss_scan.argtypes = [i32p, i64p, i64p]
        L.orc_divergence.argtypes = [i32p, i64p, i64p]
        L.orc_green_table.argtypes = [i32p, f64p]
        L.orc_self_force.argtypes = [C.c_void_p, i32p, i32p, C.c_int32, f64p, f64p]
        L.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32),
                                        C.POINTER(C.c_uint32)]
        L.orc_curl_B.argtypes = [C.c_void_p]
        L.orc_curl_D.argtypes = [C.c_void_p]
        _lib = L
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def philox4x32_10(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c, C.c_uint32), _p(k, C.c_uint32), _p(out, C.c_uint32))
    return out


def green_table(N):
    n = np.asarray(N, dtype=np.int32)
    out = np.zeros(8)
    lib().orc_green_table(_p(n, C.c_int32), _p(out, C.c_double))
    return out


def gauss_scan(N, Q):
    n = np.asarray(N, dtype=np.int32)
    Q = np.ascontiguousarray(Q, dtype=np.int64).ravel()
    flux = np.zeros(3 * Q.size, dtype=np.int64)
    st = lib().orc_gauss_scan(_p(n, C.c_int32), _p(Q, C.c_int64), _p(flux, C.c_int64))
    return st, flux


def smooth_periodic(N, sigma, rho):
    """The oracle's periodic Gaussian smoothing of a vertex array (x fastest)."""
    n = np.asarray(N, dtype=np.int32)
    r = np.ascontiguousarray(rho, dtype=np.float64).ravel().copy()
    lib().orc_smooth_periodic(_p(n, C.c_int32), float(sigma), _p(r, C.c_double))
    return r


def divergence(N, flux):
    n = np.asarray(N, dtype=np.int32)
    flux = np.ascontiguousarray(flux, dtype=np.int64).ravel()
    out = np.zeros(flux.size // 3, dtype=np.int64)
    lib().orc_divergence(_p(n, C.c_int32), _p(flux, C.c_int64), _p(out, C.c_int64))
    return out


def eps_struct(kind=EPS_CONST, axis=0, values=None, params=()):
    e = _Eps()
    e.kind = kind
    e.axis = axis
    keep = None
    if values is not None:
        keep = np.ascontiguousarray(values, dtype=np.float64).ravel()
        e.values = _p(keep, C.c_double)
    pp = list(params) + [0.0] * (8 - len(params))
    for i in range(8):
        e.params[i] = float(pp[i])
    return e, keep


class OracleSystem:
    """One MEMD system held by the C oracle.  Arrays are numpy views of the
    oracle's own memory, shaped [3, Nz, Ny, Nx] for link/plaquette fields."""

    def __init__(self, N, L, eps=None, c_light=1.0, dt=0.01, self_mode=SELF_GF,
                 dipole_corr=1, relax_tol=1e-12, relax_maxit=200000, omega=0.0,
                 seed=0, eps_eff_inv=None):
        self._lib = lib()
        self.N = tuple(int(n) for n in N)
        self.L = tuple(float(x) for x in L)
        n = np.asarray(self.N, dtype=np.int32)
        Lb = np.asarray(self.L, dtype=np.float64)
        if eps is None:
            eps = dict(kind=EPS_CONST, params=(1.0,))
        e, keep = eps_struct(**eps)
        st = C.c_int32(0)
        Mi = None
        if eps_eff_inv is not None:
            Mi = np.ascontiguousarray(eps_eff_inv, dtype=np.float64).reshape(9)
        self._h = self._lib.orc_create(_p(n, C.c_int32), _p(Lb, C.c_double), C.byref(e),
                                       c_light, dt, self_mode, dipole_corr, relax_tol,
                                       relax_maxit, omega, C.c_uint64(seed),
                                       None if Mi is None else _p(Mi, C.c_double), C.byref(st))
        del keep
        if not self._h:
            raise OracleError(f"orc_create failed with status {st.value}")
        self.V = self._lib.orc_nsites(self._h)
        self.a = self._lib.orc_scalar(self._h, 0)
        self.c = self._lib.orc_scalar(self._h, 1)
        self.dt = self._lib.orc_scalar(self._h, 2)
        self.Vbox = self._lib.orc_scalar(self._h, 3)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_destroy(h)
            self._h = None

    # ------------------------------------------------------------ arrays
    def _view(self, which, ctype, count, shape):
        ptr = self._lib.orc_ptr(self._h, which)
        if not ptr or count == 0:
            return np.zeros(shape, dtype=np.ctypeslib.as_array(ctype()).dtype)
        arr = np.ctypeslib.as_array(C.cast(ptr, C.POINTER(ctype)), shape=(count,))
        return arr.reshape(shape)

    def field(self, name):
        sel = {"ie": (A_IE, C.c_double), "D": (A_D, C.c_double), "B": (A_B, C.c_double),
               "Lg": (A_LG, C.c_int64), "Tb": (A_TB, C.c_int64)}[name]
        Nx, Ny, Nz = self.N
        return self._view(sel[0], sel[1], 3 * self.V, (3, Nz, Ny, Nx))

    @property
    def n(self):
        return self._lib.orc_nparticles(self._h)

    def particles(self, name):
        n = self.n
        sel = {"x": (A_X, C.c_double, 3), "v": (A_V, C.c_double, 3),
               "img": (A_IMG, C.c_int32, 3), "q": (A_Q, C.c_int32, 1),
               "m": (A_M, C.c_double, 1), "F": (A_F, C.c_double, 3),
               "Ft": (A_FT, C.c_double, 3)}[name]
        shape = (n, 3) if sel[2] == 3 else (n,)
        return self._view(sel[0], sel[1], n * sel[2], shape)

    @property
    def G(self):
        return self._view(A_G, C.c_double, 8, (8,)).copy()

    @property
    def Minv(self):
        return self._view(A_MINV, C.c_double, 9, (3, 3)).copy()

    @property
    def step_count(self):
        return self._lib.orc_stepcount(self._h)

    # ------------------------------------------------------------ actions
    def set_particles(self, x, q, m=None, v=None, img=None):
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
        n = x.shape[0]
        q = np.ascontiguousarray(q, dtype=np.int32).reshape(n)
        m = np.ones(n) if m is None else np.ascontiguousarray(m, dtype=np.float64).reshape(n)
        v = np.zeros((n, 3)) if v is None else np.ascontiguousarray(v, dtype=np.float64).reshape(n, 3)
        img = (np.zeros((n, 3), dtype=np.int32) if img is None
               else np.ascontiguousarray(img, dtype=np.int32).reshape(n, 3))
        st = self._lib.orc_set_particles(self._h, n, _p(x, C.c_double), _p(img, C.c_int32),
                                         _p(v, C.c_double), _p(q, C.c_int32), _p(m, C.c_double))
        if st != OK:
            raise OracleError(f"orc_set_particles failed with status {st}")

    def init_field(self):
        st = self._lib.orc_init_field(self._h)
        if st != OK:
            raise OracleError(f"orc_init_field failed with status {st}")

    def step(self, nsteps=1, thermostat=None):
        if thermostat is None:
            st = self._lib.orc_step(self._h, nsteps, 0, 0.0, 0.0)
        else:
            st = self._lib.orc_step(self._h, nsteps, 1, float(thermostat[0]),
                                    float(thermostat[1]))
        if st != OK:
            raise OracleError(f"orc_step failed with status {st}")

    def move(self, x_new, img_new):
        x_new = np.ascontiguousarray(x_new, dtype=np.float64).reshape(-1, 3)
        img_new = np.ascontiguousarray(img_new, dtype=np.int32).reshape(-1, 3)
        st = self._lib.orc_move(self._h, _p(x_new, C.c_double), _p(img_new, C.c_int32))
        if st != OK:
            raise OracleError(f"orc_move failed with status {st}")

    def gather(self):
        self._lib.orc_gather(self._h)

    def curl_B(self):
        self._lib.orc_curl_B(self._h)

    def curl_D(self):
        self._lib.orc_curl_D(self._h)

    def relax(self, tol=1e-12, maxit=200000):
        it = C.c_int32(0)
        st = self._lib.orc_relax(self._h, tol, maxit, C.byref(it))
        return st, it.value

    def set_eps(self, eps, relax=False):
        e, keep = eps_struct(**eps)
        st = self._lib.orc_set_eps(self._h, C.byref(e), 1 if relax else 0)
        del keep
        if st != OK:
            raise OracleError(f"orc_set_eps failed with status {st}")

    def eps_from_density(self, eps0, slope, eps_lo, eps_hi, sigma, relax=False):
        """orc_eps_from_density: the vertex permittivity from the local |q|
        density (returned as [Nz, Ny, Nx]), applied to the system."""
        rule = np.array([eps0, slope, eps_lo, eps_hi, sigma], dtype=np.float64)
        out = np.zeros(self.V, dtype=np.float64)
        st = self._lib.orc_eps_from_density(self._h, _p(rule, C.c_double), 1 if relax else 0,
                                            _p(out, C.c_double))
        if st != OK:
            raise OracleError(f"orc_eps_from_density failed with status {st}")
        Nx, Ny, Nz = self.N
        return out.reshape(Nz, Ny, Nx)

    def salt_vertex_eps(self, eps0, slope, eps_lo, eps_hi, sigma):
        """orc_salt_vertex_eps: the vertex permittivity of the salt rule alone
        ([Nz, Ny, Nx]), nothing applied."""
        rule = np.array([eps0, slope, eps_lo, eps_hi, sigma], dtype=np.float64)
        out = np.zeros(self.V, dtype=np.float64)
        st = self._lib.orc_salt_vertex_eps(self._h, _p(rule, C.c_double), _p(out, C.c_double))
        if st != OK:
            raise OracleError(f"orc_salt_vertex_eps failed with status {st}")
        Nx, Ny, Nz = self.N
        return out.reshape(Nz, Ny, Nx)

    def energy(self):
        out = np.zeros(len(ENERGY_KEYS))
        self._lib.orc_energy(self._h, _p(out, C.c_double))
        return dict(zip(ENERGY_KEYS, out.tolist()))

    def cic_charges(self):
        Q = np.zeros(self.V, dtype=np.int64)
        self._lib.orc_cic_charges(self._h, _p(Q, C.c_int64))
        Nx, Ny, Nz = self.N
        return Q.reshape(Nz, Ny, Nx)

    def self_force(self, cell, f, q=1):
        cell = np.asarray(cell, dtype=np.int32)
        f = np.asarray(f, dtype=np.int32)
        U = np.zeros(1)
        F = np.zeros(3)
        self._lib.orc_self_force(self._h, _p(f, C.c_int32), _p(cell, C.c_int32), int(q),
                                 _p(U, C.c_double), _p(F, C.c_double))
        return float(U[0]), F
