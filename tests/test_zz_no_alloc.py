"""memd_field_energy_static, the allocation-free field-energy entry point, for
callers that cannot allocate device memory (code inside another framework's
memory pool, a host that reserved all device memory for its own arena, a
real-time loop that must not risk an allocation).  It must give the same
electric and magnetic energy as memd_energy, computed from device arrays the
caller owns, on consecutive calls that share its fixed scratch array.

This file is named to be collected last, so that a run stopping at the first
failure has run every other test first; it also passes on its own.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def call_static(L, mesh, a, c_light, dt, prec, D, B, ie, out, stream):
    m = np.asarray(mesh, dtype=np.int32)
    return L.memd_field_energy_static(m.ctypes.data_as(C.POINTER(C.c_int32)), a, c_light, dt,
                                      prec, C.c_void_p(D.data_ptr()), C.c_void_p(B.data_ptr()),
                                      C.c_void_p(ie.data_ptr()), C.c_void_p(out.data_ptr()),
                                      C.c_void_p(stream.cuda_stream))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_static_energy_matches_memd_energy(precision):
    import torch
    from paper_1309_7859_gb300 import inputs
    from paper_1309_7859_gb300.memd import FP32, FP64, Memd, lib
    from paper_1309_7859_gb300.inputs import EpsSpec

    rng = np.random.default_rng(31)
    mesh = (40, 20, 12)
    box = tuple(float(n) for n in mesh)
    n = 200
    q = inputs.neutral_charges(rng, n)
    x = inputs.uniform_positions(rng, n, box)
    v = inputs.thermal_velocities(rng, n)
    g = Memd(mesh, box, EpsSpec("tanh", 2, (41.0, 39.0, 6.0, 3.0, 1.5)), c_light=1.0, dt=0.01,
             precision=precision, seed=5)
    g.init_field(x, q, None, v)
    g.step(7, thermostat=(1.0, 1.0))
    want = g.energy()
    D, B, _ = g.fields()
    ie, _, _ = g.setup()
    dt = torch.float32 if precision == "fp32" else torch.float64
    dev = torch.device("cuda", torch.cuda.current_device())
    # the caller's own device arrays, in the library's layout and precision
    # (FP32 values widened to FP64 and back are exact)
    Dt = torch.from_numpy(D.ravel()).to(dev).to(dt)
    Bt = torch.from_numpy(B.ravel()).to(dev).to(dt)
    It = torch.from_numpy(ie.ravel()).to(dev).to(dt)
    if precision == "fp32":
        It = torch.from_numpy(ie.ravel().astype(np.float32)).to(dev)
    stream = torch.cuda.Stream(device=dev)
    L = lib()
    prec = FP32 if precision == "fp32" else FP64
    # every output buffer exists before free device memory is first read
    bufs = [torch.full((2,), float("nan"), dtype=torch.float64, device=dev) for _ in range(6)]
    torch.cuda.synchronize()
    free = [torch.cuda.mem_get_info(dev)[0]]
    outs = []
    for out in bufs:  # calls in a row share the scratch array
        st = call_static(L, mesh, 1.0, 1.0, 0.01, prec, Dt, Bt, It, out, stream)
        assert st == 0
        stream.synchronize()
        free.append(torch.cuda.mem_get_info(dev)[0])
        outs.append(out.cpu().numpy())
    # No call allocates device memory.  cudaMemGetInfo moves in steps of
    # 2 MiB pages, so this sees any allocation of that order: from the first
    # call on (which looks up the scratch address and, with lazy module
    # loading, may load the library's own image of at most a few MiB,
    # scratch array included) free memory stays exactly the same.
    assert free[0] - free[1] <= 4 << 20
    assert all(f == free[1] for f in free[1:]), free
    for o in outs:
        assert abs(o[0] - want["electric"]) <= 1e-12 * abs(want["electric"])
        assert abs(o[1] - want["magnetic"]) <= 1e-12 * max(abs(want["magnetic"]), 1e-300) + 1e-18
    for o in outs[1:]:
        assert np.array_equal(outs[0], o)


def test_static_energy_rejects_oversized_mesh():
    import torch
    from paper_1309_7859_gb300.memd import FP32, lib
    dev = torch.device("cuda", torch.cuda.current_device())
    small = torch.zeros(8, dtype=torch.float32, device=dev)
    out = torch.zeros(2, dtype=torch.float64, device=dev)
    stream = torch.cuda.Stream(device=dev)
    # 1024 x 1024 x 256 vertices exceed MEMD_STATIC_MAX_SITES (2048 x 65536);
    # the call must refuse before touching the (too small) arrays
    st = call_static(lib(), (1024, 1024, 256), 1.0, 1.0, 0.01, FP32, small, small, small, out,
                     stream)
    assert st == 1
