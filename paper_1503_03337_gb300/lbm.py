"""ctypes binding of liblbm (include/lbm.h): same names, argument marshalling
only.  Every step of the method runs in the CUDA library; there is no
Python or CPU fallback, and loading fails loudly if the library is absent.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblbm.so")

# status codes
LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EUNSTABLE, LBM_ETIMEOUT, LBM_EBUSY = range(7)
# storage
LBM_STORAGE_F64, LBM_STORAGE_F32, LBM_STORAGE_F16, LBM_STORAGE_BF16 = range(4)
# faces
LBM_PERIODIC, LBM_WALL, LBM_MOVING_WALL, LBM_SYMMETRY, LBM_NEQ_VELOCITY, LBM_NEQ_PRESSURE = range(6)
LBM_XM, LBM_XP, LBM_YM, LBM_YP, LBM_ZM, LBM_ZP = range(6)
# fields / dtypes
LBM_FIELD_U, LBM_FIELD_P, LBM_FIELD_POPULATIONS = 1, 2, 4
LBM_DTYPE_F64, LBM_DTYPE_F32 = 0, 1
LBM_ROUND_NEAREST, LBM_ROUND_STOCHASTIC = 0, 1
LBM_RESIDUAL_STEADY, LBM_RESIDUAL_PERIODIC, LBM_RESIDUAL_CAVITY = 0, 1, 2

STORAGE_NAMES = {"f64": LBM_STORAGE_F64, "f32": LBM_STORAGE_F32,
                 "f16": LBM_STORAGE_F16, "bf16": LBM_STORAGE_BF16}


class LBMError(RuntimeError):
    def __init__(self, code, message):
        super().__init__("liblbm error %d (%s): %s" % (code, _strerror(code), message))
        self.code = code


class lbm_desc(ctypes.Structure):
    _fields_ = [("Q", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("nz", ctypes.c_int32), ("storage", ctypes.c_int32)]


class lbm_geom(ctypes.Structure):
    _fields_ = [("face", ctypes.c_int32 * 6), ("u_wall", (ctypes.c_double * 3) * 6),
                ("edge_axis", ctypes.c_int32 * 6), ("edge_scale", (ctypes.c_double * 2) * 6)]


class lbm_params(ctypes.Structure):
    _fields_ = [("nu", ctypes.c_double), ("s_nu", ctypes.c_double), ("s_c", ctypes.c_double),
                ("s_e", ctypes.c_double), ("s_q", ctypes.c_double), ("s_pi", ctypes.c_double),
                ("s_t", ctypes.c_double), ("force", ctypes.c_double * 3),
                ("force_period", ctypes.c_double), ("p_ref", ctypes.c_double),
                ("residual_interval", ctypes.c_int32), ("rounding", ctypes.c_int32),
                ("p_face", ctypes.c_double * 6), ("p_amp", ctypes.c_double * 6),
                ("p_period", ctypes.c_double)]


class lbm_launch(ctypes.Structure):
    _fields_ = [("bx", ctypes.c_int32), ("by", ctypes.c_int32),
                ("cells_per_thread", ctypes.c_int32)]

    def astuple(self):
        return (self.bx, self.by, self.cells_per_thread)


class lbm_stats(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("prev_step", ctypes.c_int64),
                ("sum_abs_du", ctypes.c_double * 3), ("sum_abs_u", ctypes.c_double * 3),
                ("sum_abs_u_prev", ctypes.c_double * 3), ("sum_P", ctypes.c_double),
                ("sum_u", ctypes.c_double * 3), ("max_abs_u", ctypes.c_double),
                ("nonfinite", ctypes.c_int64)]


_lib = None
_lock = threading.Lock()
_VP = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64

# name -> (restype, argtypes); the C-ABI surface of include/lbm.h
SIGNATURES = {
    "lbm_create": (_I, [ctypes.POINTER(lbm_desc), _VP, ctypes.POINTER(_VP)]),
    "lbm_destroy": (None, [_VP]),
    "lbm_set_stream": (_I, [_VP, _VP]),
    "lbm_set_geometry": (_I, [_VP, ctypes.POINTER(lbm_geom)]),
    "lbm_set_params": (_I, [_VP, ctypes.POINTER(lbm_params)]),
    "lbm_init_equilibrium": (_I, [_VP, _VP, _VP, _I]),
    "lbm_set_solid": (_I, [_VP, _VP, _I]),
    "lbm_step": (_I, [_VP, _I64]),
    "lbm_get_step": (_I, [_VP, ctypes.POINTER(_I64)]),
    "lbm_set_step": (_I, [_VP, _I64]),
    "lbm_read_fields": (_I, [_VP, ctypes.c_uint, _VP, _I, _I]),
    "lbm_write_populations": (_I, [_VP, _VP, _I]),
    "lbm_reductions": (_I, [_VP, ctypes.POINTER(lbm_stats)]),
    "lbm_read_stats": (_I, [_VP, ctypes.POINTER(lbm_stats)]),
    "lbm_stats_residual": (_I, [ctypes.POINTER(lbm_stats), ctypes.c_int32, ctypes.c_int32,
                                ctypes.POINTER(ctypes.c_double)]),
    "lbm_residual": (_I, [_VP, ctypes.c_int32, ctypes.c_int32,
                          ctypes.POINTER(ctypes.c_double)]),
    "lbm_memory_bytes": (_I, [_VP, ctypes.POINTER(_I64)]),
    "lbm_device_populations": (_I, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_I64)]),
    "lbm_set_launch": (_I, [_VP, ctypes.POINTER(lbm_launch)]),
    "lbm_set_overlap": (_I, [_VP, ctypes.c_int32]),
    "lbm_get_launch": (_I, [_VP, ctypes.POINTER(lbm_launch)]),
    "lbm_autotune": (_I, [_VP, ctypes.c_int32, ctypes.POINTER(lbm_launch),
                          ctypes.POINTER(ctypes.c_double)]),
    "lbm_reductions_static": (_I, [ctypes.POINTER(lbm_desc), ctypes.POINTER(lbm_geom),
                                   ctypes.POINTER(lbm_params), _I64, _VP, _VP, _I64,
                                   ctypes.POINTER(lbm_stats), _VP]),
    "lbm_batch_create": (_I, [ctypes.c_int32, _I64, _VP, ctypes.POINTER(_VP)]),
    "lbm_batch_destroy": (None, [_VP]),
    "lbm_batch_add": (_I, [_VP, ctypes.POINTER(lbm_desc), ctypes.POINTER(lbm_geom),
                           ctypes.POINTER(lbm_params), ctypes.POINTER(ctypes.c_int32)]),
    "lbm_batch_remove": (_I, [_VP, ctypes.c_int32]),
    "lbm_batch_init_equilibrium": (_I, [_VP, ctypes.c_int32, _VP, _VP, _I]),
    "lbm_batch_step": (_I, [_VP, _I64, ctypes.c_int32]),
    "lbm_batch_get_step": (_I, [_VP, ctypes.c_int32, ctypes.POINTER(_I64)]),
    "lbm_batch_read_fields": (_I, [_VP, ctypes.c_int32, ctypes.c_uint, _VP, _I, _I]),
    "lbm_batch_reductions": (_I, [_VP, ctypes.c_int32, ctypes.POINTER(lbm_stats)]),
    "lbm_batch_reductions_all": (_I, [_VP, ctypes.POINTER(lbm_stats),
                                      ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_int32)]),
    "lbm_batch_residual": (_I, [_VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                ctypes.POINTER(ctypes.c_double)]),
    "lbm_batch_set_launch": (_I, [_VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    "lbm_batch_set_schedule": (_I, [_VP, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64]),
    "lbm_batch_info": (_I, [_VP, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(_I64),
                            ctypes.POINTER(_I64)]),
    "lbm_batch_set_barrier_test": (_I, [_VP, ctypes.c_int32, _I64]),
    "lbm_last_error": (ctypes.c_char_p, []),
    "lbm_strerror": (ctypes.c_char_p, [_I]),
}


def load():
    """Load liblbm.so (built by paper_1503_03337_gb300.build); raises if absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError("liblbm.so is not built (run paper_1503_03337_gb300.build.build())")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _strerror(code):
    try:
        return load().lbm_strerror(code).decode()
    except Exception:  # library not loadable: still report the code
        return "code %d" % code


def _check(rc):
    if rc != LBM_OK:
        raise LBMError(rc, load().lbm_last_error().decode())


def _ptr(x):
    """Address of a torch tensor or numpy array (or an int/None)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


# ---- same-name wrappers ----------------------------------------------------

def lbm_create(Q, nx, ny, nz, storage=LBM_STORAGE_F32, stream=None):
    d = lbm_desc(Q, nx, ny, nz, STORAGE_NAMES.get(storage, storage))
    h = _VP()
    _check(load().lbm_create(ctypes.byref(d), stream, ctypes.byref(h)))
    return h


def lbm_destroy(h):
    load().lbm_destroy(h)


def lbm_set_stream(h, stream):
    _check(load().lbm_set_stream(h, stream))


def make_geom(faces, u_wall=None, edge=None):
    """edge: {face: (axis, scale_first, scale_last)}, edge profiles of moving
    faces (lbm_geom.edge_axis / edge_scale)."""
    g = lbm_geom()
    for i in range(6):
        g.face[i] = int(faces[i])
        for k in range(3):
            g.u_wall[i][k] = 0.0 if u_wall is None else float(u_wall[i][k])
    for face, (axis, first, last) in (edge or {}).items():
        g.edge_axis[face] = int(axis) + 1
        g.edge_scale[face][0], g.edge_scale[face][1] = float(first), float(last)
    return g


def lbm_set_geometry(h, faces, u_wall=None, edge=None):
    _check(load().lbm_set_geometry(h, ctypes.byref(make_geom(faces, u_wall, edge))))


def make_params(nu=0.0, s_nu=0.0, s_c=1.0, s_e=1.19, s_q=1.2, s_pi=1.19, s_t=0.98,
                force=(0.0, 0.0, 0.0), force_period=0.0, p_ref=0.0, residual_interval=0,
                rounding=LBM_ROUND_NEAREST, p_face=None, p_amp=None, p_period=0.0):
    p = lbm_params()
    p.nu, p.s_nu, p.s_c, p.s_e, p.s_q, p.s_pi, p.s_t = nu, s_nu, s_c, s_e, s_q, s_pi, s_t
    for k in range(3):
        p.force[k] = float(force[k])
    p.force_period = float(force_period)
    p.p_ref = float(p_ref)
    p.residual_interval = int(residual_interval)
    p.rounding = int(rounding)
    for f in range(6):
        p.p_face[f] = 0.0 if p_face is None else float(p_face[f])
        p.p_amp[f] = 0.0 if p_amp is None else float(p_amp[f])
    p.p_period = float(p_period)
    return p


def lbm_set_params(h, **kw):
    _check(load().lbm_set_params(h, ctypes.byref(make_params(**kw))))


def lbm_set_solid(h, solid, on_device=None):
    """solid: None, or N bytes (uint8 numpy array or torch tensor, x fastest)."""
    if solid is not None and not hasattr(solid, "data_ptr"):
        solid = np.ascontiguousarray(solid, dtype=np.uint8)
    if on_device is None:
        on_device = int(getattr(solid, "is_cuda", False))
    _check(load().lbm_set_solid(h, _ptr(solid), int(on_device)))


def lbm_init_equilibrium(h, u=None, p=None, on_device=None):
    if on_device is None:
        on_device = int(any(getattr(t, "is_cuda", False) for t in (u, p)))
    _check(load().lbm_init_equilibrium(h, _ptr(u), _ptr(p), int(on_device)))


def lbm_step(h, nsteps):
    _check(load().lbm_step(h, int(nsteps)))


def lbm_get_step(h):
    n = _I64()
    _check(load().lbm_get_step(h, ctypes.byref(n)))
    return n.value


def lbm_set_step(h, n):
    _check(load().lbm_set_step(h, int(n)))


def lbm_read_fields(h, mask, dst, dtype=LBM_DTYPE_F64, dst_on_device=None):
    if dst_on_device is None:
        dst_on_device = int(getattr(dst, "is_cuda", False))
    _check(load().lbm_read_fields(h, int(mask), _ptr(dst), int(dst_on_device), int(dtype)))
    return dst


def lbm_write_populations(h, src, src_on_device=None):
    if src_on_device is None:
        src_on_device = int(getattr(src, "is_cuda", False))
    _check(load().lbm_write_populations(h, _ptr(src), int(src_on_device)))


def lbm_reductions(h):
    s = lbm_stats()
    _check(load().lbm_reductions(h, ctypes.byref(s)))
    return s


def lbm_read_stats(h):
    s = lbm_stats()
    _check(load().lbm_read_stats(h, ctypes.byref(s)))
    return s


def lbm_set_overlap(h, enable):
    _check(load().lbm_set_overlap(h, int(enable)))


def lbm_set_launch(h, bx, by, cells_per_thread=1):
    l = lbm_launch(int(bx), int(by), int(cells_per_thread))
    _check(load().lbm_set_launch(h, ctypes.byref(l)))


def lbm_get_launch(h):
    l = lbm_launch()
    _check(load().lbm_get_launch(h, ctypes.byref(l)))
    return l.astuple()


def lbm_device_populations(h):
    """(device address, bytes) of the handle's population buffer."""
    p, n = _VP(), _I64()
    _check(load().lbm_device_populations(h, ctypes.byref(p), ctypes.byref(n)))
    return p.value, n.value


def lbm_autotune(h, trials=8):
    """Returns ((bx, by, cells_per_thread), ms_per_step) of the fastest launch."""
    l, ms = lbm_launch(), ctypes.c_double()
    _check(load().lbm_autotune(h, int(trials), ctypes.byref(l), ctypes.byref(ms)))
    return l.astuple(), ms.value


def lbm_reductions_static(Q, nx, ny, nz, storage, faces, u_wall, params, step,
                          populations, u_prev=None, prev_step=-1, stream=None, edge=None):
    """Allocation-free FP64 reductions over caller-owned device buffers
    (populations in the storage layout of `step`, optional 3N snapshot)."""
    d = lbm_desc(Q, nx, ny, nz, STORAGE_NAMES.get(storage, storage))
    g = make_geom(faces, u_wall, edge)
    s = lbm_stats()
    _check(load().lbm_reductions_static(ctypes.byref(d), ctypes.byref(g), ctypes.byref(params),
                                        int(step), _ptr(populations), _ptr(u_prev),
                                        int(prev_step), ctypes.byref(s), stream))
    return s


def lbm_memory_bytes(h):
    n = _I64()
    _check(load().lbm_memory_bytes(h, ctypes.byref(n)))
    return n.value


# ---- batches -------------------------------------------------------------------

def lbm_batch_create(capacity, budget_bytes=0, stream=None):
    b = _VP()
    _check(load().lbm_batch_create(int(capacity), int(budget_bytes), stream, ctypes.byref(b)))
    return b


def lbm_batch_destroy(b):
    load().lbm_batch_destroy(b)


def lbm_batch_add(b, Q, nx, ny, nz, storage, faces, u_wall=None, edge=None, **params):
    d = lbm_desc(Q, nx, ny, nz, STORAGE_NAMES.get(storage, storage))
    g = make_geom(faces, u_wall, edge)
    p = make_params(**params)
    slot = ctypes.c_int32()
    _check(load().lbm_batch_add(b, ctypes.byref(d), ctypes.byref(g), ctypes.byref(p),
                                ctypes.byref(slot)))
    return slot.value


def lbm_batch_remove(b, slot):
    _check(load().lbm_batch_remove(b, int(slot)))


def lbm_batch_init_equilibrium(b, slot, u=None, p=None):
    _check(load().lbm_batch_init_equilibrium(b, int(slot), _ptr(u), _ptr(p), 1))


def lbm_batch_step(b, nsteps, chunk=1):
    _check(load().lbm_batch_step(b, int(nsteps), int(chunk)))


def lbm_batch_get_step(b, slot):
    n = _I64()
    _check(load().lbm_batch_get_step(b, int(slot), ctypes.byref(n)))
    return n.value


def lbm_batch_read_fields(b, slot, mask, dst, dtype=LBM_DTYPE_F64):
    _check(load().lbm_batch_read_fields(b, int(slot), int(mask), _ptr(dst), 1, int(dtype)))
    return dst


def lbm_batch_reductions(b, slot):
    s = lbm_stats()
    _check(load().lbm_batch_reductions(b, int(slot), ctypes.byref(s)))
    return s


def lbm_batch_reductions_all(b, capacity):
    """{slot: lbm_stats} for every active domain (one synchronisation)."""
    out = (lbm_stats * capacity)()
    slots = (ctypes.c_int32 * capacity)()
    n = ctypes.c_int32()
    _check(load().lbm_batch_reductions_all(b, out, slots, ctypes.byref(n)))
    return {slots[k]: out[k] for k in range(n.value)}


def lbm_batch_set_launch(b, bx, by, persistent):
    _check(load().lbm_batch_set_launch(b, int(bx), int(by), int(persistent)))


def lbm_batch_set_schedule(b, tiles_per_cta=0, solo_min_cells=0, cluster_bytes=0):
    _check(load().lbm_batch_set_schedule(b, int(tiles_per_cta), int(solo_min_cells),
                                         int(cluster_bytes)))


def lbm_batch_info(b):
    a, u, c = ctypes.c_int32(), _I64(), _I64()
    _check(load().lbm_batch_info(b, ctypes.byref(a), ctypes.byref(u), ctypes.byref(c)))
    return a.value, u.value, c.value


def lbm_batch_set_barrier_test(b, extra_arrivals, spin_limit):
    _check(load().lbm_batch_set_barrier_test(b, int(extra_arrivals), int(spin_limit)))


# ---- convergence criteria (Eq. sc, Eq. cr, Eq. cavity_creterion) --------------

def lbm_stats_residual(s, kind, component=0):
    r = ctypes.c_double()
    _check(load().lbm_stats_residual(ctypes.byref(s), int(kind), int(component),
                                     ctypes.byref(r)))
    return r.value


def lbm_residual(h, kind, component=0):
    r = ctypes.c_double()
    _check(load().lbm_residual(h, int(kind), int(component), ctypes.byref(r)))
    return r.value


def lbm_batch_residual(b, slot, kind, component=0):
    r = ctypes.c_double()
    _check(load().lbm_batch_residual(b, int(slot), int(kind), int(component), ctypes.byref(r)))
    return r.value


def residual_steady(s, k):
    """Eq. sc for component k (earlier time level)."""
    return lbm_stats_residual(s, LBM_RESIDUAL_STEADY, k)


def residual_periodic(s, k):
    """Eq. cr for component k (later time level)."""
    return lbm_stats_residual(s, LBM_RESIDUAL_PERIODIC, k)


def residual_cavity(s):
    """Eq. cavity_creterion: all three components, later time level."""
    return lbm_stats_residual(s, LBM_RESIDUAL_CAVITY)


# ---- host-array helpers (numpy, pageable memory) ------------------------------

def read_u(h, nx, ny, nz):
    out = np.empty((3, nz, ny, nx))
    lbm_read_fields(h, LBM_FIELD_U, out, LBM_DTYPE_F64, 0)
    return out


def read_p(h, nx, ny, nz):
    out = np.empty((nz, ny, nx))
    lbm_read_fields(h, LBM_FIELD_P, out, LBM_DTYPE_F64, 0)
    return out


def read_populations(h, Q, nx, ny, nz):
    out = np.empty((Q, nz, ny, nx))
    lbm_read_fields(h, LBM_FIELD_POPULATIONS, out, LBM_DTYPE_F64, 0)
    return out
