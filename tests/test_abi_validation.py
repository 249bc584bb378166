"""CPU checks of memd_create's and memd_server_create's argument validation
through the C ABI.

Every check below runs before the library touches CUDA, so these calls need
no GPU: each bad argument must come back as its status code (INVALID, or
COURANT for a time step beyond the 3-d leapfrog limit of Eq. 30) with the
output handle left NULL."""
import ctypes as C

import pytest

from paper_1309_7859_gb300 import memd as M

INVALID, COURANT = 1, 2


def create(mesh=(8, 8, 8), box=(8.0, 8.0, 8.0), kind=0, axis=0, params=(1.0,), values=None,
           c_light=1.0, dt=0.01, **opts):
    L = M.lib()
    o = M.Options()
    L.memd_default_options(C.byref(o))
    for k, v in opts.items():
        if k == "field_shape":
            for i, x in enumerate(v):
                o.field_shape[i] = x
        else:
            setattr(o, k, v)
    e = M.EpsProfile()
    e.kind, e.axis = kind, axis
    for i, p in enumerate(params):
        e.params[i] = p
    if values is not None:
        e.values = values.ctypes.data_as(C.POINTER(C.c_double))
    m = (C.c_int32 * 3)(*mesh)
    b = (C.c_double * 3)(*box)
    h = C.c_void_p(12345)                    # must come back NULL on failure
    st = L.memd_create(m, b, C.byref(e), c_light, dt, C.byref(o), C.byref(h))
    return st, h.value


@pytest.mark.parametrize("args,status", [
    (dict(mesh=(1, 8, 8), box=(1.0, 8.0, 8.0)), INVALID),          # fewer than 2 vertices
    (dict(box=(8.0, 8.0, 9.0)), INVALID),                           # cells not cubic
    (dict(box=(8.0, -8.0, 8.0)), INVALID),                          # negative box edge
    (dict(mesh=(1300, 1300, 1300), box=(1300.0,) * 3), INVALID),    # 3 V beyond int32 indexing
    (dict(dt=0.0), INVALID),
    (dict(c_light=-1.0), INVALID),
    (dict(c_light=1.0, dt=0.6), COURANT),                           # c dt sqrt(3) >= a
    (dict(precision=7), INVALID),
    (dict(self_mode=3), INVALID),
    (dict(field_kernel=9), INVALID),
    (dict(step_engine=5), INVALID),
    (dict(apply_mode=3), INVALID),
    (dict(kind=3, axis=5, params=(41.0, 39.0, 4.0, 2.0, 1.5)), INVALID),   # tanh, no such axis
    (dict(kind=1), INVALID),                                        # per-link eps without values
    (dict(kind=6, params=(80.0, 2.0, 4.0, 4.0, 4.0, 4.5)), INVALID),       # ball wider than the box
    (dict(kind=99), INVALID),                                       # unknown profile
    (dict(field_shape=(8, 4, 0, 0)), INVALID),                      # a fixed shape needs a kernel
    (dict(field_kernel=4, field_shape=(0, 0, 0, 384)), INVALID),    # rows: 256 or 512 threads
    (dict(field_kernel=4, field_shape=(8, 0, 0, 256)), INVALID),    # rows use no tile height
    (dict(field_kernel=3, field_shape=(6, 4, 1, 0)), INVALID),      # no such tile height
    (dict(field_kernel=3, field_shape=(8, 0, 1, 0)), INVALID),      # no planes per CTA
    (dict(field_kernel=3, field_shape=(8, 4, 3, 0)), INVALID),      # 1 or 2 planes ahead
    (dict(field_kernel=1, field_shape=(8, 4, 1, 0)), INVALID),      # halo loops load no planes ahead
    (dict(field_kernel=3, field_shape=(16, 4, 1, 0)), INVALID),     # 16 rows need FP32
])
def test_create_refuses_bad_arguments_before_touching_the_gpu(args, status):
    st, h = create(**args)
    assert st == status
    assert h is None


def test_status_strings_and_null_context_messages():
    L = M.lib()
    texts = {L.memd_status_string(s) for s in range(11)}
    assert len(texts) == 11 and all(texts)
    assert L.memd_last_error(None)           # a static message for a NULL context


@pytest.mark.parametrize("field,value", [("max_slots", 0), ("quantum", 0), ("budget_bytes", 0),
                                         ("precision", 5)])
def test_server_create_refuses_bad_options_before_touching_the_gpu(field, value):
    L = M.lib()
    o = M.ServerOptions()
    L.memd_server_default_options(C.byref(o))
    setattr(o, field, value)
    h = C.c_void_p(12345)
    assert L.memd_server_create(C.byref(o), C.byref(h)) == INVALID
    assert h.value is None


@pytest.mark.parametrize("mesh", [(1 << 30, 1 << 30, 16),     # V wraps to 0 in int64
                                  ((1 << 31) - 1, 2, 2),       # one edge beyond the limit
                                  (65536, 65536, 65536),       # no wrap, far beyond the limit
                                  (2, 1, 2)])                  # an edge below 2
def test_static_energy_refuses_bad_meshes_before_touching_the_gpu(mesh):
    """memd_field_energy_static bounds each edge and the vertex count before
    any CUDA call; the dummy pointers below are never dereferenced."""
    L = M.lib()
    m = (C.c_int32 * 3)(*mesh)
    dummy = C.c_void_p(0x1000)
    st = L.memd_field_energy_static(m, 1.0, 1.0, 0.01, 1, dummy, dummy, dummy, dummy, None)
    assert st == INVALID
