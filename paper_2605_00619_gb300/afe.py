"""Thin ctypes binding of the C ABI in ``include/afe.h`` (argument marshalling only).

Every function has the name of the C entry point it calls.  Host arrays are numpy
arrays; device arrays are passed as integer addresses (e.g. ``tensor.data_ptr()``).
A non-OK status raises :class:`AfeError` carrying the status and ``afe_last_error()``,
except where ``check=False`` is given (then the status code is returned).  There is no
fallback: if the in-tree library is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "lib", "libafe.so")

AFE_OK, AFE_EINVAL, AFE_EMESH, AFE_ENOMEM, AFE_ECUDA, AFE_ENOCONV, AFE_ENONFINITE, AFE_ETIMEOUT = range(8)
STATUS_NAMES = ["AFE_OK", "AFE_EINVAL", "AFE_EMESH", "AFE_ENOMEM", "AFE_ECUDA", "AFE_ENOCONV",
                "AFE_ENONFINITE", "AFE_ETIMEOUT"]
AFE_EULER, AFE_NAVIER_STOKES = 0, 1
AFE_FP64, AFE_FP32 = 0, 1
AFE_BC_PERIODIC, AFE_BC_TRANSMISSIVE = 0, 1


class afe_params(ctypes.Structure):
    _fields_ = [
        ("order", ctypes.c_int),
        ("equations", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("gamma", ctypes.c_double),
        ("R", ctypes.c_double),
        ("mu", ctypes.c_double),
        ("Pr", ctypes.c_double),
        ("kappa", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("limiter", ctypes.c_int),
        ("m1", ctypes.c_double),
        ("picard_tol", ctypes.c_double),
        ("picard_max", ctypes.c_int),
        ("period", ctypes.c_double * 3),
        ("visc_dt_subtet", ctypes.c_int),
        ("h_diameter", ctypes.c_int),
    ]


class afe_stats(ctypes.Structure):
    _fields_ = [
        ("dt", ctypes.c_double),
        ("t", ctypes.c_double),
        ("steps", ctypes.c_int64),
        ("picard_mean", ctypes.c_double),
        ("picard_max", ctypes.c_int32),
        ("nonconverged", ctypes.c_int64),
        ("troubled", ctypes.c_int64),
        ("totals", ctypes.c_double * 5),
        ("kernel_launches", ctypes.c_int64),
    ]


class afe_plan(ctypes.Structure):
    _fields_ = [
        ("fp32_shared", ctypes.c_int32),
        ("corrector_block", ctypes.c_int32),
        ("smem_bytes", ctypes.c_int64),
        ("max_nodes", ctypes.c_int32),
        ("max_subtets", ctypes.c_int32),
        ("ring_min", ctypes.c_int32),
        ("ring_max", ctypes.c_int32),
        ("narrow_cells", ctypes.c_int64),
        ("masked_cells", ctypes.c_int64),
        ("tcgen05", ctypes.c_int32),
        ("stage_rows_min", ctypes.c_int32),
    ]


class afe_schedule(ctypes.Structure):
    _fields_ = [
        ("cost_order", ctypes.c_int32),
        ("variant", ctypes.c_int32),
        ("ring_cap", ctypes.c_int32),
        ("narrow", ctypes.c_int32),
    ]


class AfeError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {message}")
        self.status = status


_lib = None
_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)
_I32 = ctypes.POINTER(ctypes.c_int32)
_I8 = ctypes.POINTER(ctypes.c_int8)

_SIGS = {
    "afe_default_params": (ctypes.c_int, [ctypes.POINTER(afe_params), ctypes.c_int]),
    "afe_mesh_create": (ctypes.c_int, [ctypes.POINTER(afe_params), ctypes.c_int64, _D, ctypes.c_int64, _I64, _I64,
                                       _I8, ctypes.c_int, _P, ctypes.POINTER(_P)]),
    "afe_mesh_validate": (ctypes.c_int, [ctypes.POINTER(afe_params), ctypes.c_int64, _D, ctypes.c_int64, _I64,
                                         _I64, _I8, ctypes.c_int, _I64, _I64]),
    "afe_num_nodes": (ctypes.c_int, [_P, _I64, _I64]),
    "afe_get_node_coords": (ctypes.c_int, [_P, _D]),
    "afe_set_stream": (ctypes.c_int, [_P, _P]),
    "afe_set_state": (ctypes.c_int, [_P, _D]),
    "afe_set_state_device": (ctypes.c_int, [_P, _P, _P]),
    "afe_get_state": (ctypes.c_int, [_P, _D]),
    "afe_get_state_device": (ctypes.c_int, [_P, _P]),
    "afe_compute_dt": (ctypes.c_int, [_P, _D]),
    "afe_step": (ctypes.c_int, [_P, ctypes.c_double]),
    "afe_step_async": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_int]),
    "afe_sync": (ctypes.c_int, [_P]),
    "afe_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(afe_stats)]),
    "afe_set_diagnostics": (ctypes.c_int, [_P, ctypes.c_int]),
    "afe_get_diagnostics": (ctypes.c_int, [_P, _D, _I32, _D, _D]),
    "afe_device_bytes": (ctypes.c_int, [_P, _I64]),
    "afe_set_profiling": (ctypes.c_int, [_P, ctypes.c_int]),
    "afe_conserved_totals_noalloc": (ctypes.c_int, [_P, _P, _P, _P]),
    "afe_plan_info": (ctypes.c_int, [_P, ctypes.POINTER(afe_plan)]),
    "afe_set_wait_limit": (ctypes.c_int, [_P, ctypes.c_int32]),
    "afe_cfl_pieces": (ctypes.c_int, [_P, ctypes.c_int64, _D, _D]),
    "afe_set_predictor_variant": (ctypes.c_int, [_P, ctypes.c_int32]),
    "afe_set_schedule": (ctypes.c_int, [_P, ctypes.POINTER(afe_schedule)]),
    "afe_get_schedule": (ctypes.c_int, [_P, ctypes.POINTER(afe_schedule)]),
    "afe_autotune": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(afe_schedule), _D, _D]),
    "afe_batch_set_schedule": (ctypes.c_int, [_P, ctypes.POINTER(afe_schedule)]),
    "afe_batch_autotune": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(afe_schedule), _D, _D]),
    "afe_stage_times": (ctypes.c_int, [_P, _D, _I64, ctypes.c_int]),
    "afe_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, _P, ctypes.POINTER(_P)]),
    "afe_batch_step_async": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_int, ctypes.c_int]),
    "afe_batch_sync": (ctypes.c_int, [_P, _I32]),
    "afe_batch_info": (ctypes.c_int, [_P, _I64, _I64, _I64, _I64]),
    "afe_batch_destroy": (None, [_P]),
    "afe_last_error": (ctypes.c_char_p, []),
    "afe_mesh_destroy": (None, [_P]),
}


def lib():
    """Load the in-tree library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIBPATH):
            raise RuntimeError(f"{LIBPATH} is missing: build it with paper_2605_00619_gb300.build.build()")
        L = ctypes.CDLL(LIBPATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def _check(status, check=True):
    if status != AFE_OK and check:
        raise AfeError(status, lib().afe_last_error().decode())
    return status


def _dptr(a):
    return a.ctypes.data_as(_D)


def afe_last_error() -> str:
    return lib().afe_last_error().decode()


def afe_default_params(order: int, **overrides) -> afe_params:
    p = afe_params()
    _check(lib().afe_default_params(ctypes.byref(p), order))
    for k, v in overrides.items():
        if k == "period":
            for d in range(3):
                p.period[d] = float(v[d])
        else:
            setattr(p, k, v)
    return p


def afe_mesh_create(params: afe_params, xyz, cell_subtet_ptr, subtet_vtx, subtet_shift, boundary: int,
                    stream: int = 0, check: bool = True):
    """Returns an opaque handle (ctypes void pointer), or (None, status) with check=False."""
    xyz = np.ascontiguousarray(xyz, np.float64)
    ptr = np.ascontiguousarray(cell_subtet_ptr, np.int64)
    vtx = np.ascontiguousarray(subtet_vtx, np.int64)
    sh = None if subtet_shift is None else np.ascontiguousarray(subtet_shift, np.int8)
    out = _P()
    st = lib().afe_mesh_create(ctypes.byref(params), len(xyz), _dptr(xyz), len(ptr) - 1, ptr.ctypes.data_as(_I64),
                               vtx.ctypes.data_as(_I64), None if sh is None else sh.ctypes.data_as(_I8), boundary,
                               _P(stream), ctypes.byref(out))
    if not check:
        return (out if st == AFE_OK else None), st
    _check(st)
    return out


def afe_mesh_validate(params: afe_params, xyz, cell_subtet_ptr, subtet_vtx, subtet_shift, boundary: int,
                      check: bool = True):
    """Host-only validation; returns (status, n_nodes, n_face_tris)."""
    xyz = np.ascontiguousarray(xyz, np.float64)
    ptr = np.ascontiguousarray(cell_subtet_ptr, np.int64)
    vtx = np.ascontiguousarray(subtet_vtx, np.int64)
    sh = None if subtet_shift is None else np.ascontiguousarray(subtet_shift, np.int8)
    nn, nf = ctypes.c_int64(), ctypes.c_int64()
    st = lib().afe_mesh_validate(ctypes.byref(params), len(xyz), _dptr(xyz), len(ptr) - 1, ptr.ctypes.data_as(_I64),
                                 vtx.ctypes.data_as(_I64), None if sh is None else sh.ctypes.data_as(_I8), boundary,
                                 ctypes.byref(nn), ctypes.byref(nf))
    _check(st, check)
    return st, int(nn.value), int(nf.value)


def afe_num_nodes(m):
    n = ctypes.c_int64()
    _check(lib().afe_num_nodes(m, ctypes.byref(n), None))
    return int(n.value)


def afe_node_ptr(m, n_cells):
    n = ctypes.c_int64()
    ptr = np.empty(n_cells + 1, np.int64)
    _check(lib().afe_num_nodes(m, ctypes.byref(n), ptr.ctypes.data_as(_I64)))
    return ptr


def afe_get_node_coords(m):
    x = np.empty((afe_num_nodes(m), 3), np.float64)
    _check(lib().afe_get_node_coords(m, _dptr(x)))
    return x


def afe_set_stream(m, stream: int):
    _check(lib().afe_set_stream(m, _P(stream)))


def afe_set_state(m, q):
    q = np.ascontiguousarray(q, np.float64)
    if q.shape != (afe_num_nodes(m), 5):
        raise ValueError("state must be [n_nodes, 5]")
    _check(lib().afe_set_state(m, _dptr(q)))


def afe_set_state_device(m, dptr: int, stream: int = 0):
    _check(lib().afe_set_state_device(m, _P(dptr), _P(stream)))


def afe_get_state(m, out=None):
    """State [n_nodes, 5] into ``out`` (C-contiguous float64, e.g. pinned host memory) or a new array."""
    q = np.empty((afe_num_nodes(m), 5), np.float64) if out is None else out
    if q.dtype != np.float64 or not q.flags.c_contiguous or q.shape != (afe_num_nodes(m), 5):
        raise ValueError("out must be a C-contiguous float64 array of shape [n_nodes, 5]")
    _check(lib().afe_get_state(m, _dptr(q)))
    return q


def afe_get_state_device(m, dptr: int):
    _check(lib().afe_get_state_device(m, _P(dptr)))


def afe_compute_dt(m) -> float:
    dt = ctypes.c_double()
    _check(lib().afe_compute_dt(m, ctypes.byref(dt)))
    return dt.value


def afe_step(m, dt: float = 0.0, check: bool = True) -> int:
    return _check(lib().afe_step(m, float(dt)), check)


def afe_step_async(m, dt: float = 0.0, nsteps: int = 1):
    _check(lib().afe_step_async(m, float(dt), int(nsteps)))


def afe_sync(m, check: bool = True) -> int:
    return _check(lib().afe_sync(m), check)


def afe_get_stats(m) -> afe_stats:
    s = afe_stats()
    _check(lib().afe_get_stats(m, ctypes.byref(s)))
    return s


def afe_set_diagnostics(m, on: bool = True):
    _check(lib().afe_set_diagnostics(m, int(bool(on))))


def afe_get_diagnostics(m, n_cells: int, qbar: bool = True):
    n = afe_num_nodes(m)
    qb = np.empty((n, 5), np.float64) if qbar else None
    it = np.empty(n_cells, np.int32)
    beta = np.empty(n_cells, np.float64)
    mu = np.empty(n_cells, np.float64)
    _check(lib().afe_get_diagnostics(m, None if qb is None else _dptr(qb), it.ctypes.data_as(_I32), _dptr(beta),
                                     _dptr(mu)))
    return qb, it, beta, mu


def afe_device_bytes(m) -> int:
    b = ctypes.c_int64()
    _check(lib().afe_device_bytes(m, ctypes.byref(b)))
    return int(b.value)


def afe_set_profiling(m, on: bool = True):
    _check(lib().afe_set_profiling(m, int(bool(on))))


def afe_stage_times(m, reset: bool = True):
    """Returns (ms[4] summed over the recorded steps, number of steps)."""
    ms = np.zeros(4, np.float64)
    n = ctypes.c_int64()
    _check(lib().afe_stage_times(m, _dptr(ms), ctypes.byref(n), int(bool(reset))))
    return ms, int(n.value)


def afe_plan_info(m) -> afe_plan:
    out = afe_plan()
    _check(lib().afe_plan_info(m, ctypes.byref(out)))
    return out


def afe_set_predictor_variant(m, variant: int):
    _check(lib().afe_set_predictor_variant(m, int(variant)))


def _schedule(cost_order=0, variant=0, ring_cap=0, narrow=0) -> afe_schedule:
    return afe_schedule(int(cost_order), int(variant), int(ring_cap), int(narrow))


def afe_set_schedule(m, cost_order=0, variant=0, ring_cap=0, narrow=0, check: bool = True) -> int:
    s = _schedule(cost_order, variant, ring_cap, narrow)
    return _check(lib().afe_set_schedule(m, ctypes.byref(s)), check)


def afe_get_schedule(m) -> afe_schedule:
    s = afe_schedule()
    _check(lib().afe_get_schedule(m, ctypes.byref(s)))
    return s


def afe_autotune(m, trials: int = 3):
    """Returns (chosen schedule, mean predictor ms with it, with the default; -1 when the choice
    came from the remembered signature)."""
    s = afe_schedule()
    b, d = ctypes.c_double(), ctypes.c_double()
    _check(lib().afe_autotune(m, int(trials), ctypes.byref(s), ctypes.byref(b), ctypes.byref(d)))
    return s, b.value, d.value


def afe_batch_set_schedule(b, cost_order=0, variant=0, ring_cap=0, narrow=0, check: bool = True) -> int:
    s = _schedule(cost_order, variant, ring_cap, narrow)
    return _check(lib().afe_batch_set_schedule(b, ctypes.byref(s)), check)


def afe_batch_autotune(b, trials: int = 3):
    s = afe_schedule()
    x, d = ctypes.c_double(), ctypes.c_double()
    _check(lib().afe_batch_autotune(b, int(trials), ctypes.byref(s), ctypes.byref(x), ctypes.byref(d)))
    return s, x.value, d.value


def afe_cfl_pieces(m, n_cells: int):
    """(largest CFL bracket, smallest characteristic length) over the first n_cells cells."""
    b, h = ctypes.c_double(), ctypes.c_double()
    _check(lib().afe_cfl_pieces(m, int(n_cells), ctypes.byref(b), ctypes.byref(h)))
    return b.value, h.value


def afe_set_wait_limit(m, polls: int):
    _check(lib().afe_set_wait_limit(m, int(polls)))


AFE_NOALLOC_CHUNK = 65536
AFE_NOALLOC_MAX_PARTIALS = 4096
AFE_NOALLOC_MAX_NODES = AFE_NOALLOC_CHUNK * AFE_NOALLOC_MAX_PARTIALS


def afe_conserved_totals_noalloc(m, dq_ptr: int, dtotals_ptr: int, stream: int = 0, check: bool = True) -> int:
    """Conserved totals of a device state into a device array of 5 doubles, with no device
    allocation by the call (for callers that may not allocate at the point of use)."""
    return _check(lib().afe_conserved_totals_noalloc(m, _P(dq_ptr), _P(dtotals_ptr), _P(stream)), check)


AFE_MAX_BATCH = 64


def afe_batch_create(members, stream: int = 0, check: bool = True):
    """Batch of mesh handles stepped by one launch per stage; returns an opaque handle, or
    (None, status) with check=False."""
    arr = (_P * len(members))(*[m.value if isinstance(m, _P) else m for m in members])
    out = _P()
    st = lib().afe_batch_create(arr, len(members), _P(stream), ctypes.byref(out))
    if not check:
        return (out if st == AFE_OK else None), st
    _check(st)
    return out


def afe_batch_step_async(b, dt: float = 0.0, nsteps: int = 1, use_graph: bool = True):
    _check(lib().afe_batch_step_async(b, float(dt), int(nsteps), int(bool(use_graph))))


def afe_batch_sync(b, n_members: int, check: bool = True):
    """Returns (status, per-member statuses as a numpy int32 array)."""
    ms = np.zeros(n_members, np.int32)
    st = lib().afe_batch_sync(b, ms.ctypes.data_as(_I32))
    _check(st, check)
    return st, ms


def afe_batch_info(b):
    """Returns (cells, nodes, kernel launches, graph launches)."""
    v = [ctypes.c_int64() for _ in range(4)]
    _check(lib().afe_batch_info(b, *[ctypes.byref(x) for x in v]))
    return tuple(int(x.value) for x in v)


def afe_batch_destroy(b):
    if b:
        lib().afe_batch_destroy(b)


def afe_mesh_destroy(m):
    if m:
        lib().afe_mesh_destroy(m)


def create_from_polymesh(pm, params: afe_params, stream: int = 0):
    """Convenience: call afe_mesh_create with the arrays of an ``inputs.voronoi.PolyMesh``-like object."""
    if pm.periodic:
        for d in range(3):
            params.period[d] = pm.period[d]
    bc = AFE_BC_PERIODIC if pm.periodic else AFE_BC_TRANSMISSIVE
    return afe_mesh_create(params, pm.xyz, pm.cell_subtet_ptr, pm.subtet_vtx, pm.subtet_shift, bc, stream)
