"""Thin ctypes binding of the MEMD C ABI (include/memd.h).

Argument marshalling only: every step of the method runs in the CUDA kernels
of libmemd.so.  There is no CPU fallback; a missing library or GPU raises.
Device memory can come from PyTorch's caching allocator and work is issued on
a PyTorch stream when torch is available (`use_torch=True`).
"""
from __future__ import annotations

import atexit
import ctypes as C
import os
import weakref
from dataclasses import dataclass

import numpy as np

from . import build as _build

FP64, FP32 = 0, 1
SELF_NONE, SELF_GF, SELF_DIRECT = 0, 1, 2
EPS_KINDS = {"const": 0, "links": 1, "vertices": 2, "tanh": 3, "sin": 4, "planes": 5,
             "sphere": 6, "cut": 7}
STATUS = {0: "OK", 1: "INVALID", 2: "COURANT", 3: "OOM", 4: "CUDA", 5: "CELL_JUMP", 6: "GAUSS",
          7: "RELAX_NOCONV", 8: "DIPOLE_DRIFT", 9: "TIMEOUT", 10: "STATE", 11: "OVERFLOW"}

EXPORTS = ("memd_default_options", "memd_status_string", "memd_last_error", "memd_create",
           "memd_destroy", "memd_init_field", "memd_step", "memd_forces", "memd_forces_device",
           "memd_energy", "memd_get_particles", "memd_set_particles", "memd_move",
           "memd_get_fields", "memd_set_fields", "memd_compute_forces", "memd_set_eps",
           "memd_step_host", "memd_io_buffers", "memd_step_io", "memd_state_bytes",
           "memd_save_state", "memd_load_state", "memd_dipole_check", "memd_inject",
           "memd_eps_from_density",
           "memd_get_setup",
           "memd_get_kernel_stats", "memd_reset_kernel_stats", "memd_synchronize",
           "memd_batch_create", "memd_batch_create_kernel", "memd_batch_step",
           "memd_batch_synchronize", "memd_batch_io_buffers", "memd_batch_step_io",
           "memd_batch_set_engine",
           "memd_batch_kernel_stats", "memd_batch_set_timing", "memd_batch_destroy",
           "memd_server_default_options",
           "memd_server_create", "memd_server_destroy", "memd_server_submit", "memd_server_pump",
           "memd_server_status", "memd_server_result", "memd_server_release",
           "memd_server_used_bytes", "memd_server_get_stats", "memd_server_last_error",
           "memd_field_energy_static")
VOID_RESULT = ("memd_default_options", "memd_destroy", "memd_status_string", "memd_last_error",
               "memd_batch_destroy", "memd_server_default_options", "memd_server_destroy",
               "memd_server_used_bytes", "memd_server_last_error")


class MemdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)
FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)


class EpsProfile(C.Structure):
    _fields_ = [("kind", C.c_int32), ("axis", C.c_int32), ("values", C.POINTER(C.c_double)),
                ("params", C.c_double * 8)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("self_mode", C.c_int32), ("dipole_corr", C.c_int32),
                ("relax_max_iter", C.c_int32), ("relax_tol", C.c_double), ("seed", C.c_uint64),
                ("cuda_stream", C.c_void_p), ("device", C.c_int32), ("use_graphs", C.c_int32),
                ("alloc", ALLOC), ("free", FREE), ("alloc_user", C.c_void_p),
                ("time_kernels", C.c_int32), ("field_kernel", C.c_int32),
                ("step_engine", C.c_int32), ("apply_mode", C.c_int32),
                ("field_shape", C.c_int32 * 4)]


class Thermostat(C.Structure):
    _fields_ = [("gamma", C.c_double), ("kT", C.c_double)]


class EnergyTerms(C.Structure):
    _fields_ = [("kinetic", C.c_double), ("electric", C.c_double), ("magnetic", C.c_double),
                ("self", C.c_double), ("dipole", C.c_double), ("total", C.c_double),
                ("P", C.c_double * 3), ("gauss_residual", C.c_double),
                ("gauss_exact", C.c_int32), ("pad", C.c_int32), ("step", C.c_int64)]

    def as_dict(self):
        return {"kinetic": self.kinetic, "electric": self.electric, "magnetic": self.magnetic,
                "self": self.self, "dipole": self.dipole, "total": self.total,
                "P0": self.P[0], "P1": self.P[1], "P2": self.P[2],
                "gauss_residual": self.gauss_residual, "gauss_exact": float(self.gauss_exact),
                "step": self.step}


class ServerOptions(C.Structure):
    _fields_ = [("precision", C.c_int32), ("max_slots", C.c_int32), ("budget_bytes", C.c_int64),
                ("quantum", C.c_int32), ("device", C.c_int32), ("cuda_stream", C.c_void_p),
                ("alloc", ALLOC), ("free", FREE), ("alloc_user", C.c_void_p),
                ("thermostat", C.c_int32), ("pad", C.c_int32), ("gamma", C.c_double),
                ("kT", C.c_double), ("admission_workers", C.c_int32),
                ("reserved", C.c_int32 * 3)]


class Request(C.Structure):
    _fields_ = [("mesh", C.c_int32 * 3), ("box", C.c_double * 3), ("eps", EpsProfile),
                ("c_light", C.c_double), ("dt", C.c_double), ("n", C.c_int64),
                ("pos", C.POINTER(C.c_double)), ("q", C.POINTER(C.c_int32)),
                ("mass", C.POINTER(C.c_double)), ("vel", C.POINTER(C.c_double)),
                ("seed", C.c_uint64), ("nsteps", C.c_int64)]


class ServerStats(C.Structure):
    _fields_ = [("setup_s", C.c_double), ("budget_use_sum", C.c_double), ("rounds", C.c_int64),
                ("steps_rounds", C.c_int64), ("rebuilds", C.c_int64), ("admitted", C.c_int64),
                ("link_updates", C.c_int64), ("particle_steps", C.c_int64),
                ("step_gpu_s", C.c_double), ("table_updates", C.c_int64)]


class IoBuffers(C.Structure):
    _fields_ = [("pos", C.POINTER(C.c_double)), ("vel", C.POINTER(C.c_double)),
                ("img", C.POINTER(C.c_int32)), ("f", C.POINTER(C.c_double))]


class BatchIo(C.Structure):
    _fields_ = [("pos", C.POINTER(C.c_double)), ("vel", C.POINTER(C.c_double)),
                ("img", C.POINTER(C.c_int32)), ("f", C.POINTER(C.c_double)),
                ("offsets", C.POINTER(C.c_int64)), ("n_total", C.c_int64)]


class KernelStats(C.Structure):
    _fields_ = [("field_ms", C.c_double), ("field_launches", C.c_int64),
                ("field_bytes", C.c_double), ("launches_per_step", C.c_int64),
                ("field_tma", C.c_int32), ("field_ty", C.c_int32), ("field_zchunk", C.c_int32),
                ("field_site", C.c_int32), ("step_single", C.c_int32), ("field_tx", C.c_int32),
                ("field_rows", C.c_int32), ("pad", C.c_int32), ("phase_ms", C.c_double * 3)]


_lib = None


def library_path():
    return _build.LIB


def lib(build_if_missing=True):
    """Load libmemd.so (building it first when it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libmemd.so not built at {path}")
    L = C.CDLL(path)
    vp, i32p, f64p, i64p = C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_double), C.POINTER(C.c_int64)
    L.memd_default_options.argtypes = [C.POINTER(Options)]
    L.memd_status_string.restype = C.c_char_p
    L.memd_status_string.argtypes = [C.c_int]
    L.memd_last_error.restype = C.c_char_p
    L.memd_last_error.argtypes = [vp]
    L.memd_create.argtypes = [i32p, f64p, C.POINTER(EpsProfile), C.c_double, C.c_double,
                              C.POINTER(Options), C.POINTER(vp)]
    L.memd_destroy.argtypes = [vp]
    L.memd_init_field.argtypes = [vp, C.c_int64, f64p, i32p, f64p, f64p]
    L.memd_step.argtypes = [vp, C.c_int64, C.POINTER(Thermostat)]
    L.memd_forces.argtypes = [vp, f64p]
    L.memd_forces_device.argtypes = [vp, C.POINTER(vp)]
    L.memd_energy.argtypes = [vp, C.POINTER(EnergyTerms)]
    L.memd_get_particles.argtypes = [vp, f64p, f64p, i32p]
    L.memd_set_particles.argtypes = [vp, f64p, f64p, i32p]
    L.memd_step_host.argtypes = [vp, f64p, f64p, i32p, C.c_int64, C.POINTER(Thermostat),
                                 f64p, f64p, i32p, f64p]
    L.memd_io_buffers.argtypes = [vp, C.POINTER(IoBuffers)]
    L.memd_state_bytes.restype = C.c_int64
    L.memd_state_bytes.argtypes = [vp]
    L.memd_save_state.argtypes = [vp, C.c_void_p, C.c_int64]
    L.memd_load_state.argtypes = [vp, C.c_void_p, C.c_int64]
    L.memd_step_io.argtypes = [vp, C.c_int32, C.c_int64, C.POINTER(Thermostat)]
    L.memd_move.argtypes = [vp, f64p, i32p]
    L.memd_get_fields.argtypes = [vp, f64p, f64p, i64p]
    L.memd_set_fields.argtypes = [vp, f64p, f64p, i64p]
    L.memd_compute_forces.argtypes = [vp]
    L.memd_set_eps.argtypes = [vp, C.POINTER(EpsProfile), C.c_int32]
    L.memd_get_setup.argtypes = [vp, f64p, f64p, f64p]
    L.memd_dipole_check.argtypes = [vp, C.c_double, f64p]
    L.memd_eps_from_density.argtypes = [vp, C.POINTER(C.c_double * 5), C.c_int32, f64p]
    L.memd_inject.argtypes = [vp, C.c_int32, C.c_double]
    L.memd_get_kernel_stats.argtypes = [vp, C.POINTER(KernelStats)]
    L.memd_reset_kernel_stats.argtypes = [vp]
    L.memd_synchronize.argtypes = [vp]
    L.memd_batch_create.argtypes = [C.c_int32, C.POINTER(vp), C.POINTER(vp)]
    L.memd_batch_create_kernel.argtypes = [C.c_int32, C.POINTER(vp), C.c_int32, C.POINTER(vp)]
    L.memd_batch_step.argtypes = [vp, C.c_int64, C.POINTER(Thermostat)]
    L.memd_batch_synchronize.argtypes = [vp]
    L.memd_batch_io_buffers.argtypes = [vp, C.POINTER(BatchIo)]
    L.memd_batch_set_engine.argtypes = [vp, C.c_int32, C.c_int32, C.c_int32]
    L.memd_batch_step_io.argtypes = [vp, C.c_int32, C.c_int64, C.POINTER(Thermostat)]
    L.memd_batch_kernel_stats.argtypes = [vp, C.POINTER(KernelStats)]
    L.memd_batch_set_timing.argtypes = [vp, C.c_int32]
    L.memd_batch_destroy.argtypes = [vp]
    L.memd_server_default_options.argtypes = [C.POINTER(ServerOptions)]
    L.memd_server_create.argtypes = [C.POINTER(ServerOptions), C.POINTER(vp)]
    L.memd_server_destroy.argtypes = [vp]
    L.memd_server_submit.argtypes = [vp, C.POINTER(Request), C.POINTER(C.c_int64)]
    L.memd_server_pump.argtypes = [vp, i32p, i32p, i32p]
    L.memd_server_status.argtypes = [vp, C.c_int64, i32p]
    L.memd_server_result.argtypes = [vp, C.c_int64, f64p, f64p, i32p, f64p, C.POINTER(EnergyTerms)]
    L.memd_server_release.argtypes = [vp, C.c_int64]
    L.memd_server_used_bytes.restype = C.c_int64
    L.memd_server_used_bytes.argtypes = [vp]
    L.memd_server_get_stats.argtypes = [vp, C.POINTER(ServerStats)]
    L.memd_server_last_error.restype = C.c_char_p
    L.memd_server_last_error.argtypes = [vp]
    L.memd_field_energy_static.argtypes = [i32p, C.c_double, C.c_double, C.c_double, C.c_int32,
                                           vp, vp, vp, vp, vp]
    for name in EXPORTS:
        if name not in VOID_RESULT:
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _ptr(a, ct):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(ct))


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a.reshape(shape) if shape is not None else a


def _i32(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a.reshape(shape) if shape is not None else a


class _TorchAllocator:
    """Routes the library's device allocations through torch's caching allocator."""

    def __init__(self, device):
        import torch
        self.torch = torch
        self.device = device
        self.alloc = ALLOC(self._alloc)
        self.free = FREE(self._free)

    def _alloc(self, user, nbytes, stream):
        try:
            return self.torch.cuda.caching_allocator_alloc(int(nbytes), self.device,
                                                           int(stream or 0))
        except Exception:  # out of memory: the library reports MEMD_ERR_OOM
            return None

    def _free(self, user, ptr, nbytes, stream):
        try:
            self.torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:  # torch already torn down at interpreter exit
            pass


# handles still open at interpreter exit are closed while torch is alive:
# servers and batches before the systems they use
_live = {"server": weakref.WeakSet(), "batch": weakref.WeakSet(), "memd": weakref.WeakSet()}


@atexit.register
def _close_all():
    for kind in ("server", "batch", "memd"):
        for obj in list(_live[kind]):
            try:
                obj.close()
            except Exception:
                pass


@dataclass
class StepTiming:
    field_ms: float
    field_launches: int
    field_bytes: float
    launches_per_step: int
    field_kernel: str = ""
    single: bool = False
    phase_ms: tuple = (0.0, 0.0, 0.0)  # batches: deposition, transfer application, gather


class Memd:
    """One MEMD system on one GPU (a memd_ctx)."""

    def __init__(self, mesh, box, eps=None, c_light=1.0, dt=0.01, precision="fp64",
                 self_mode=SELF_GF, dipole_corr=True, relax_tol=1e-12, relax_max_iter=200000,
                 seed=0, use_graphs=True, time_kernels=False, use_torch=True, stream=None,
                 device=None, field_kernel="auto", step_engine="auto", apply_mode="auto",
                 field_shape=None):
        self._L = lib()
        _live["memd"].add(self)
        self._h = C.c_void_p(None)
        self.mesh = tuple(int(n) for n in mesh)
        self.box = tuple(float(b) for b in box)
        self.V = self.mesh[0] * self.mesh[1] * self.mesh[2]
        self.n = 0
        o = Options()
        self._L.memd_default_options(C.byref(o))
        o.precision = FP32 if precision in ("fp32", FP32) else FP64
        o.self_mode = int(self_mode)
        o.dipole_corr = 1 if dipole_corr else 0
        o.relax_tol = float(relax_tol)
        o.relax_max_iter = int(relax_max_iter)
        o.seed = int(seed) & ((1 << 64) - 1)
        o.use_graphs = 1 if use_graphs else 0
        o.time_kernels = 1 if time_kernels else 0
        o.field_kernel = {"auto": 0, "ldg": 1, "tma": 2, "site": 3, "rows": 4}[field_kernel]
        o.step_engine = {"auto": 0, "graph": 1, "single": 2}[step_engine]
        o.apply_mode = {"auto": 0, "sparse": 1, "dense": 2}[apply_mode]
        if field_shape is not None:   # (ty, zchunk, planes_ahead, rows_nt), 0 = unused
            for k, v in enumerate(field_shape):
                o.field_shape[k] = int(v)
        self._alloc = None
        self._stream = stream
        if use_torch:
            import torch
            if not torch.cuda.is_available():
                raise RuntimeError("MEMD needs a CUDA GPU; torch sees none")
            dev = torch.cuda.current_device() if device is None else int(device)
            o.device = dev
            if stream is None:
                stream = torch.cuda.Stream(device=dev)
                self._stream = stream
            o.cuda_stream = C.c_void_p(stream.cuda_stream)
            self._alloc = _TorchAllocator(dev)
            o.alloc = self._alloc.alloc
            o.free = self._alloc.free
        else:
            o.device = -1 if device is None else int(device)
            if stream is not None:
                o.cuda_stream = C.c_void_p(int(stream))
        e, keep = make_eps(eps)
        mesh_a = np.asarray(self.mesh, dtype=np.int32)
        box_a = np.asarray(self.box, dtype=np.float64)
        st = self._L.memd_create(_ptr(mesh_a, C.c_int32), _ptr(box_a, C.c_double), C.byref(e),
                                 float(c_light), float(dt), C.byref(o), C.byref(self._h))
        del keep
        if st != 0:
            raise MemdError(st, "memd_create failed")
        self.precision = "fp32" if o.precision == FP32 else "fp64"

    # ---------------------------------------------------------------- helpers
    def _check(self, st, what):
        if st != 0:
            msg = self._L.memd_last_error(self._h)
            raise MemdError(st, f"{what}: {msg.decode() if msg else ''}")

    def close(self):
        if self._h:
            self._L.memd_destroy(self._h)
            self._h = C.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def stream(self):
        return self._stream

    # ----------------------------------------------------------------- calls
    def init_field(self, x, q, m=None, v=None):
        x = _f64(x).reshape(-1, 3)
        n = x.shape[0]
        q = _i32(q, (n,))
        m = None if m is None else _f64(m, (n,))
        v = None if v is None else _f64(v, (n, 3))
        self._check(self._L.memd_init_field(self._h, n, _ptr(x, C.c_double), _ptr(q, C.c_int32),
                                            _ptr(m, C.c_double), _ptr(v, C.c_double)),
                    "memd_init_field")
        self.n = n

    def step(self, nsteps=1, thermostat=None):
        th = None
        if thermostat is not None:
            th = Thermostat(float(thermostat[0]), float(thermostat[1]))
        self._check(self._L.memd_step(self._h, int(nsteps), C.byref(th) if th else None),
                    "memd_step")

    def forces(self, out=None):
        out = np.zeros((self.n, 3)) if out is None else out
        self._check(self._L.memd_forces(self._h, _ptr(out, C.c_double)), "memd_forces")
        return out

    def forces_device_ptr(self):
        p = C.c_void_p()
        self._check(self._L.memd_forces_device(self._h, C.byref(p)), "memd_forces_device")
        return p.value

    def energy(self):
        e = EnergyTerms()
        self._check(self._L.memd_energy(self._h, C.byref(e)), "memd_energy")
        return e.as_dict()

    def particles(self):
        x = np.zeros((self.n, 3))
        v = np.zeros((self.n, 3))
        img = np.zeros((self.n, 3), dtype=np.int32)
        self._check(self._L.memd_get_particles(self._h, _ptr(x, C.c_double), _ptr(v, C.c_double),
                                               _ptr(img, C.c_int32)), "memd_get_particles")
        return x, v, img

    def get_particles_into(self, x=None, v=None, img=None):
        self._check(self._L.memd_get_particles(self._h, _ptr(x, C.c_double), _ptr(v, C.c_double),
                                               _ptr(img, C.c_int32)), "memd_get_particles")

    def set_particles(self, x=None, v=None, img=None):
        x = None if x is None else _f64(x, (self.n, 3))
        v = None if v is None else _f64(v, (self.n, 3))
        img = None if img is None else _i32(img, (self.n, 3))
        self._check(self._L.memd_set_particles(self._h, _ptr(x, C.c_double), _ptr(v, C.c_double),
                                               _ptr(img, C.c_int32)), "memd_set_particles")

    def step_host(self, nsteps=1, thermostat=None, x_in=None, v_in=None, img_in=None,
                  x_out=None, v_out=None, img_out=None, f_out=None):
        """State load, nsteps steps and state read-back in one call with one
        synchronisation (memd_step_host).  Arrays are used in place (page-
        locked ones make the copies asynchronous); outputs must be C-contiguous
        (n, 3) arrays of float64 (int32 for the image counters)."""
        th = None
        if thermostat is not None:
            th = Thermostat(float(thermostat[0]), float(thermostat[1]))
        for a, dt in ((x_out, np.float64), (v_out, np.float64), (img_out, np.int32),
                      (f_out, np.float64)):
            if a is not None and (a.dtype != dt or not a.flags["C_CONTIGUOUS"] or
                                  a.shape != (self.n, 3)):
                raise ValueError("outputs must be C-contiguous (n, 3) arrays")
        x_in = None if x_in is None else _f64(x_in, (self.n, 3))
        v_in = None if v_in is None else _f64(v_in, (self.n, 3))
        img_in = None if img_in is None else _i32(img_in, (self.n, 3))
        self._check(self._L.memd_step_host(
            self._h, _ptr(x_in, C.c_double), _ptr(v_in, C.c_double), _ptr(img_in, C.c_int32),
            int(nsteps), C.byref(th) if th else None, _ptr(x_out, C.c_double),
            _ptr(v_out, C.c_double), _ptr(img_out, C.c_int32), _ptr(f_out, C.c_double)),
            "memd_step_host")

    def save_state(self):
        """The whole dynamical state as bytes (memd_save_state)."""
        nb = self._L.memd_state_bytes(self._h)
        buf = np.zeros(nb, dtype=np.uint8)
        self._check(self._L.memd_save_state(self._h, buf.ctypes.data, nb), "memd_save_state")
        return buf

    def load_state(self, buf):
        """Restore a state from save_state (same mesh, box, precision and
        particle count)."""
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        self._check(self._L.memd_load_state(self._h, buf.ctypes.data, buf.size), "memd_load_state")

    def io_buffers(self):
        """The library's page-locked I/O buffers as (n, 3) numpy views: pos,
        vel, img (in and out) and f (out), valid until the next init_field."""
        io = IoBuffers()
        self._check(self._L.memd_io_buffers(self._h, C.byref(io)), "memd_io_buffers")
        n = self.n
        view = lambda p: np.ctypeslib.as_array(p, shape=(n, 3)) if n else np.zeros((0, 3))
        return {"pos": view(io.pos), "vel": view(io.vel), "img": view(io.img), "f": view(io.f)}

    def step_io(self, nsteps=1, thermostat=None, load=True):
        """memd_step_io: load the state from the I/O buffers (load), step, and
        read state and forces back into them; one copy each way, one sync."""
        th = None
        if thermostat is not None:
            th = Thermostat(float(thermostat[0]), float(thermostat[1]))
        self._check(self._L.memd_step_io(self._h, 1 if load else 0, int(nsteps),
                                         C.byref(th) if th else None), "memd_step_io")

    def move(self, x, img=None):
        x = _f64(x, (self.n, 3))
        img = None if img is None else _i32(img, (self.n, 3))
        self._check(self._L.memd_move(self._h, _ptr(x, C.c_double), _ptr(img, C.c_int32)),
                    "memd_move")

    def fields(self):
        Nx, Ny, Nz = self.mesh
        D = np.zeros((3, Nz, Ny, Nx))
        B = np.zeros((3, Nz, Ny, Nx))
        Lg = np.zeros((3, Nz, Ny, Nx), dtype=np.int64)
        self._check(self._L.memd_get_fields(self._h, _ptr(D, C.c_double), _ptr(B, C.c_double),
                                            _ptr(Lg, C.c_int64)), "memd_get_fields")
        return D, B, Lg

    def set_fields(self, D=None, B=None, Lg=None):
        D = None if D is None else _f64(D).ravel()
        B = None if B is None else _f64(B).ravel()
        Lg = None if Lg is None else np.ascontiguousarray(Lg, dtype=np.int64).ravel()
        self._check(self._L.memd_set_fields(self._h, _ptr(D, C.c_double), _ptr(B, C.c_double),
                                            _ptr(Lg, C.c_int64)), "memd_set_fields")

    def compute_forces(self):
        self._check(self._L.memd_compute_forces(self._h), "memd_compute_forces")

    def eps_from_density(self, eps0, slope, eps_lo, eps_hi, sigma, relax=False):
        """memd_eps_from_density: the permittivity from the local |q| density
        (vertex values returned as [Nz, Ny, Nx])."""
        rule = (C.c_double * 5)(eps0, slope, eps_lo, eps_hi, sigma)
        out = np.zeros(self.V, dtype=np.float64)
        self._check(self._L.memd_eps_from_density(self._h, C.byref(rule), 1 if relax else 0,
                                                  _ptr(out, C.c_double)), "memd_eps_from_density")
        Nx, Ny, Nz = self.mesh
        return out.reshape(Nz, Ny, Nx)

    def dipole_check(self, limit):
        """memd_dipole_check: (status, ratio) of the dipole correction's field to
        the RMS lattice field; status 8 (DIPOLE_DRIFT) above `limit`."""
        r = C.c_double(0.0)
        st = self._L.memd_dipole_check(self._h, float(limit), C.byref(r))
        return st, r.value

    def inject(self, kind="barrier_skew", wait_s=0.0):
        """memd_inject: host-side failure injection for tests."""
        k = {"none": 0, "barrier_skew": 1}[kind]
        self._check(self._L.memd_inject(self._h, k, float(wait_s)), "memd_inject")

    def set_eps(self, eps, relax=False):
        """New permittivity profile (an inputs.EpsSpec or dict); D is kept, or
        relaxed to the new electrostatic minimum with relax=True."""
        e, keep = make_eps(eps)
        self._check(self._L.memd_set_eps(self._h, C.byref(e), 1 if relax else 0), "memd_set_eps")
        del keep

    def setup(self):
        Nx, Ny, Nz = self.mesh
        ie = np.zeros((3, Nz, Ny, Nx))
        G = np.zeros(8)
        M = np.zeros((3, 3))
        self._check(self._L.memd_get_setup(self._h, _ptr(ie, C.c_double), _ptr(G, C.c_double),
                                           _ptr(M, C.c_double)), "memd_get_setup")
        return ie, G, M

    def kernel_stats(self):
        k = KernelStats()
        self._check(self._L.memd_get_kernel_stats(self._h, C.byref(k)), "memd_get_kernel_stats")
        if k.step_single:
            kind = "k_step_coop (whole step, one cooperative launch)"
        elif k.field_rows:
            kind = f"k_rows<nt={k.field_rows}>"
        elif k.field_tma:
            kind = f"k_fused_tma<ty={k.field_ty}, zchunk={k.field_zchunk}>"
        elif k.field_site:
            kind = f"k_fused_site<ty={k.field_ty}, zchunk={k.field_zchunk}, planes_ahead={k.field_site}>"
        else:
            kind = f"k_fused_curl<ty={k.field_ty}, zchunk={k.field_zchunk}>"
        return StepTiming(k.field_ms, k.field_launches, k.field_bytes, k.launches_per_step, kind,
                          bool(k.step_single))

    def reset_kernel_stats(self):
        self._check(self._L.memd_reset_kernel_stats(self._h), "memd_reset_kernel_stats")

    def synchronize(self):
        self._check(self._L.memd_synchronize(self._h), "memd_synchronize")


class Batch:
    """Independent Memd systems stepped together, four launches per step for
    all of them.  The members must share one stream (pass the same `stream`
    when creating them) and precision; they stay usable one by one."""

    def __init__(self, members, field_kernel="auto"):
        """field_kernel: "auto" (timed choice between site tiles and the row
        kernel; members created with the row kernel at one fixed width fix
        it), "site" or "rows"."""
        self._L = lib()
        _live["batch"].add(self)
        self.members = list(members)
        arr = (C.c_void_p * len(self.members))(*[m._h.value for m in self.members])
        self._h = C.c_void_p(None)
        kind = {"auto": 0, "site": 3, "rows": 4}[field_kernel]
        st = self._L.memd_batch_create_kernel(len(self.members), arr, kind, C.byref(self._h))
        if st != 0:
            raise MemdError(st, "memd_batch_create failed")

    def step(self, nsteps=1, thermostat=None):
        th = None
        if thermostat is not None:
            th = Thermostat(float(thermostat[0]), float(thermostat[1]))
        st = self._L.memd_batch_step(self._h, int(nsteps), C.byref(th) if th else None)
        if st != 0:
            raise MemdError(st, "memd_batch_step failed")

    def synchronize(self):
        st = self._L.memd_batch_synchronize(self._h)
        if st != 0:
            raise MemdError(st, "memd_batch_synchronize failed")

    def set_engine(self, engine="auto", field_ctas=-1, item_planes=0):
        """memd_batch_set_engine: "graph" (four kernels a step), "single" (the
        whole step in one cooperative launch of persistent CTAs) or "auto"."""
        e = {"auto": 0, "graph": 1, "single": 2}[engine]
        st = self._L.memd_batch_set_engine(self._h, e, int(field_ctas), int(item_planes))
        if st != 0:
            raise MemdError(st, "memd_batch_set_engine failed")

    def io_buffers(self):
        """The batch's page-locked I/O block as (n_total, 3) numpy views pos,
        vel, img (in and out) and f (out), plus the members' row offsets
        (count + 1)."""
        io = BatchIo()
        st = self._L.memd_batch_io_buffers(self._h, C.byref(io))
        if st != 0:
            raise MemdError(st, "memd_batch_io_buffers failed")
        n = io.n_total
        view = lambda p: np.ctypeslib.as_array(p, shape=(n, 3)) if n else np.zeros((0, 3))
        off = np.ctypeslib.as_array(io.offsets, shape=(len(self.members) + 1,)).copy()
        return {"pos": view(io.pos), "vel": view(io.vel), "img": view(io.img), "f": view(io.f),
                "offsets": off}

    def step_io(self, nsteps=1, thermostat=None, load=True):
        """memd_batch_step_io: every member's state from the I/O block (load),
        nsteps batch steps, state and forces back into it; one copy in, the
        copies out (beside the step with load and one step), one
        synchronisation."""
        th = None
        if thermostat is not None:
            th = Thermostat(float(thermostat[0]), float(thermostat[1]))
        st = self._L.memd_batch_step_io(self._h, 1 if load else 0, int(nsteps),
                                        C.byref(th) if th else None)
        if st != 0:
            raise MemdError(st, "memd_batch_step_io failed")

    def set_timing(self, on):
        """CUDA events around the batched field update in the step graph."""
        st = self._L.memd_batch_set_timing(self._h, 1 if on else 0)
        if st != 0:
            raise MemdError(st, "memd_batch_set_timing failed")

    def kernel_stats(self):
        k = KernelStats()
        st = self._L.memd_batch_kernel_stats(self._h, C.byref(k))
        if st != 0:
            raise MemdError(st, "memd_batch_kernel_stats failed")
        if k.step_single:
            name = "k_batch_step (whole step, one cooperative launch)"
        elif k.field_rows:
            name = f"k_rows_batch<nt={k.field_rows}>"
        else:
            name = (f"k_fused_site_batch<tx={k.field_tx}, ty={k.field_ty}, "
                    f"zchunk={k.field_zchunk}, planes_ahead={k.field_site}>")
        return StepTiming(k.field_ms, k.field_launches, k.field_bytes, k.launches_per_step, name,
                          bool(k.step_single), tuple(k.phase_ms))

    def close(self):
        if self._h:
            self._L.memd_batch_destroy(self._h)
            self._h = C.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request server (memd_server_*): submit systems with
    a step count, pump scheduling rounds, collect results."""

    def __init__(self, precision="fp32", budget_bytes=8 << 30, max_slots=64, quantum=50,
                 thermostat=None, use_torch=True, stream=None, admission_workers=0):
        self._L = lib()
        _live["server"].add(self)
        o = ServerOptions()
        self._L.memd_server_default_options(C.byref(o))
        o.precision = FP32 if precision == "fp32" else FP64
        o.budget_bytes = int(budget_bytes)
        o.max_slots = int(max_slots)
        o.quantum = int(quantum)
        o.admission_workers = int(admission_workers)
        if thermostat is not None:
            o.thermostat, o.gamma, o.kT = 1, float(thermostat[0]), float(thermostat[1])
        self._alloc = None
        self._stream = stream
        if use_torch:
            import torch
            if not torch.cuda.is_available():
                raise RuntimeError("MEMD needs a CUDA GPU; torch sees none")
            dev = torch.cuda.current_device()
            o.device = dev
            if stream is None:
                self._stream = torch.cuda.Stream(device=dev)
            o.cuda_stream = C.c_void_p(self._stream.cuda_stream)
            self._alloc = _TorchAllocator(dev)
            o.alloc, o.free = self._alloc.alloc, self._alloc.free
        self._h = C.c_void_p(None)
        st = self._L.memd_server_create(C.byref(o), C.byref(self._h))
        if st != 0:
            raise MemdError(st, "memd_server_create failed")
        self._keep = {}
        self.n_of = {}

    def _err(self, st, what):
        if st != 0:
            msg = self._L.memd_server_last_error(self._h)
            raise MemdError(st, f"{what}: {msg.decode() if msg else ''}")

    def submit(self, sysc, nsteps=None):
        """Queue an inputs.System (its own step count unless nsteps is given)."""
        r = Request()
        for d in range(3):
            r.mesh[d] = int(sysc.mesh[d])
            r.box[d] = float(sysc.box[d])
        e, keep = make_eps(sysc.eps)
        r.eps = e
        r.c_light, r.dt = float(sysc.c_light), float(sysc.dt)
        x = _f64(sysc.x).reshape(-1, 3)
        q = _i32(sysc.q)
        m = _f64(sysc.m)
        v = _f64(sysc.v).reshape(-1, 3)
        r.n = x.shape[0]
        r.pos, r.q, r.mass, r.vel = (_ptr(x, C.c_double), _ptr(q, C.c_int32),
                                     _ptr(m, C.c_double), _ptr(v, C.c_double))
        r.seed = int(sysc.seed) & ((1 << 64) - 1)
        r.nsteps = int(sysc.steps if nsteps is None else nsteps)
        rid = C.c_int64(0)
        self._err(self._L.memd_server_submit(self._h, C.byref(r), C.byref(rid)), "submit")
        del keep, x, q, m, v  # copied by the server
        self.n_of[rid.value] = r.n
        return rid.value

    def pump(self):
        a, q, d = C.c_int32(0), C.c_int32(0), C.c_int32(0)
        self._err(self._L.memd_server_pump(self._h, C.byref(a), C.byref(q), C.byref(d)), "pump")
        return a.value, q.value, d.value

    def status(self, rid):
        s = C.c_int32(0)
        self._err(self._L.memd_server_status(self._h, int(rid), C.byref(s)), "status")
        return s.value

    def result(self, rid):
        n = self.n_of[rid]
        x, v, f = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 3))
        img = np.zeros((n, 3), dtype=np.int32)
        e = EnergyTerms()
        self._err(self._L.memd_server_result(self._h, int(rid), _ptr(x, C.c_double),
                                             _ptr(v, C.c_double), _ptr(img, C.c_int32),
                                             _ptr(f, C.c_double), C.byref(e)), "result")
        return x, v, img, f, e.as_dict()

    def release(self, rid):
        self._err(self._L.memd_server_release(self._h, int(rid)), "release")

    def used_bytes(self):
        return self._L.memd_server_used_bytes(self._h)

    def stats(self):
        st = ServerStats()
        self._err(self._L.memd_server_get_stats(self._h, C.byref(st)), "stats")
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def close(self):
        if self._h:
            self._L.memd_server_destroy(self._h)
            self._h = C.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def serve(server, systems, arrivals, poll_s=0.0):
    """Drive a server through a stream of systems arriving at the given wall
    times (seconds from now): submit each when its time comes, pump rounds,
    and record when each finished.  Returns a list of dicts (id, arrival,
    done, latency) in submission order."""
    import time as _time
    t0 = _time.perf_counter()
    order = sorted(range(len(systems)), key=lambda i: arrivals[i])
    pending = list(order)
    ids, rec = {}, {}
    while pending or any(server.status(r) < 2 for r in ids.values()):
        now = _time.perf_counter() - t0
        while pending and arrivals[pending[0]] <= now:
            i = pending.pop(0)
            ids[i] = server.submit(systems[i])
            rec[i] = {"index": i, "id": ids[i], "arrival": now, "done": None}
        if not ids:
            _time.sleep(max(0.0, arrivals[pending[0]] - now))
            continue
        server.pump()
        now = _time.perf_counter() - t0
        for i, rid in ids.items():
            if rec[i]["done"] is None and server.status(rid) >= 2:
                rec[i]["done"] = now
        if poll_s:
            _time.sleep(poll_s)
    for r in rec.values():
        r["latency"] = r["done"] - r["arrival"]
    return [rec[i] for i in sorted(rec)]


def make_eps(spec):
    """EpsProfile from an inputs.EpsSpec-like object or dict (kept array returned too)."""
    e = EpsProfile()
    keep = None
    if spec is None:
        e.kind = 0
        e.params[0] = 1.0
        return e, keep
    kind = spec["kind"] if isinstance(spec, dict) else spec.kind
    axis = spec.get("axis", 0) if isinstance(spec, dict) else spec.axis
    params = spec.get("params", ()) if isinstance(spec, dict) else spec.params
    values = spec.get("values") if isinstance(spec, dict) else spec.values
    e.kind = EPS_KINDS[kind] if isinstance(kind, str) else int(kind)
    e.axis = int(axis)
    pp = list(params) + [0.0] * (8 - len(params))
    for i in range(8):
        e.params[i] = float(pp[i])
    if values is not None:
        keep = np.ascontiguousarray(values, dtype=np.float64).ravel()
        e.values = keep.ctypes.data_as(C.POINTER(C.c_double))
    return e, keep


def from_system(sysc, **kw):
    """Memd context for an inputs.System (not yet initialised)."""
    return Memd(sysc.mesh, sysc.box, sysc.eps, c_light=sysc.c_light, dt=sysc.dt,
                precision=sysc.precision, seed=sysc.seed, **kw)
