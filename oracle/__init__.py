"""FP64 CPU oracle for the iD3Q14 / iD3Q18 incompressible MRT LBM, and for
the iD3Q26 model built by the same construction (App. B's closing remark).

TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the CPU
baseline leg of the benchmark are the only callers.  The product path (the
CUDA library and its binding) never imports this package.

``lbm_oracle.c`` holds the lattice Boltzmann update (plain C, double
precision, ``-ffp-contract=off``); ``analytic.py`` holds the analytic duct and
pulsatile-channel series and the error/residual norms of Sec. 4.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liblbm_oracle.so")
_lock = threading.Lock()
_lib = None

PERIODIC, WALL, MOVING_WALL, SYMMETRY, NEQ_VELOCITY, NEQ_PRESSURE = 0, 1, 2, 3, 4, 5


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add, OpenMP over z)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC),
                                                   os.path.getmtime(_SRC[:-2] + ".h"))):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-std=c11", "-D_DEFAULT_SOURCE", "-shared", "-fPIC", _SRC,
           "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Grid(ctypes.Structure):
    _fields_ = [("Q", ctypes.c_int), ("nx", ctypes.c_int),
                ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("face", ctypes.c_int * 6),
                ("u_wall", (ctypes.c_double * 3) * 6),
                ("edge_axis", ctypes.c_int * 6),
                ("edge_scale", (ctypes.c_double * 2) * 6),
                ("solid", ctypes.c_void_p)]


class Rates(ctypes.Structure):
    _fields_ = [("sc", ctypes.c_double), ("se", ctypes.c_double),
                ("sq", ctypes.c_double), ("snu", ctypes.c_double),
                ("spi", ctypes.c_double), ("st", ctypes.c_double)]


class Params(ctypes.Structure):
    _fields_ = [("rates", Rates), ("force", ctypes.c_double * 3),
                ("period", ctypes.c_double), ("p_face", ctypes.c_double * 6),
                ("p_amp", ctypes.c_double * 6), ("p_period", ctypes.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            L.oracle_velocities.argtypes = [ctypes.c_int, ip]
            L.oracle_weights.argtypes = [ctypes.c_int, dp, dp]
            L.oracle_transform.argtypes = [ctypes.c_int, dp]
            L.oracle_moment_equilibrium.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp]
            L.oracle_pressure.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp]
            L.oracle_feq.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp]
            L.oracle_collide.argtypes = [ctypes.c_int, ctypes.POINTER(Rates), dp, dp, dp]
            L.oracle_init_equilibrium.argtypes = [ctypes.POINTER(Grid), dp, dp, dp]
            L.oracle_step.argtypes = [ctypes.POINTER(Grid), ctypes.POINTER(Params),
                                      ctypes.c_int64, dp, dp, ctypes.c_int]
            L.oracle_run.argtypes = [ctypes.POINTER(Grid), ctypes.POINTER(Params),
                                     ctypes.c_int64, ctypes.c_int64, dp, ctypes.c_int]
            L.oracle_macroscopic.argtypes = [ctypes.POINTER(Grid), ctypes.POINTER(Params),
                                             ctypes.c_int64, dp, dp, dp]
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(rc):
    if rc != 0:
        raise RuntimeError("oracle call failed with code %d" % rc)


# ---- model tables and one-cell operations -----------------------------------

def velocities(Q: int) -> np.ndarray:
    out = np.zeros(Q * 3, dtype=np.int32)
    _check(lib().oracle_velocities(Q, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))
    return out.reshape(Q, 3).astype(np.int64)


def weights(Q: int):
    w = np.zeros(Q)
    w0 = ctypes.c_double()
    _check(lib().oracle_weights(Q, _dp(w), ctypes.byref(w0)))
    return w, w0.value


def transform(Q: int) -> np.ndarray:
    """T (int64): for Q = 14 and 18 as printed, for Q = 26 the Gram-Schmidt
    rows of Sec. 3's recipe with their denominators cleared."""
    out = np.zeros(Q * Q)
    _check(lib().oracle_transform(Q, _dp(out)))
    return out.reshape(Q, Q).astype(np.int64)


def moment_equilibrium(Q: int, p: float, u) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(Q)
    _check(lib().oracle_moment_equilibrium(Q, float(p), _dp(u), _dp(out)))
    return out


def pressure(Q: int, P: float, u) -> float:
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = ctypes.c_double()
    _check(lib().oracle_pressure(Q, float(P), _dp(u), ctypes.byref(out)))
    return out.value


def feq(Q: int, p: float, u) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(Q)
    _check(lib().oracle_feq(Q, float(p), _dp(u), _dp(out)))
    return out


def s_nu_of(nu: float) -> float:
    """Eq. vis: nu = c_s^2 (tau - 1/2) with c_s^2 = 1/3 and s_nu = 1/tau, so
    s_nu = 1 / (3 nu + 1/2) in lattice units."""
    return 1.0 / (3.0 * nu + 0.5)


def rates(Q: int, snu: float, sc=1.0, se=1.19, sq=1.2, st=0.98, spi=None) -> Rates:
    """Relaxation rates of Sec. 4 (sc=1, se=1.19, sq=1.2, st=0.98, snu=1/tau);
    for Q18 the paper leaves s_pi open and the default reading is s_pi = se."""
    return Rates(sc, se, sq, snu, se if spi is None else spi, st)


def collide(Q: int, r: Rates, f, F=(0.0, 0.0, 0.0)) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.float64)
    out = np.zeros(Q)
    _check(lib().oracle_collide(Q, ctypes.byref(r), _dp(f), _dp(F), _dp(out)))
    return out


# ---- whole-grid operations -----------------------------------------------------

def make_grid(Q, nx, ny, nz, faces=(WALL,) * 6, u_wall=None, edge=None, solid=None) -> Grid:
    """edge: {face: (axis, scale_first, scale_last)}, the edge profile of a
    moving face (see lbm_oracle.h); solid: None or an (nz, ny, nx) array,
    nonzero at solid nodes (kept alive by the returned grid)."""
    g = Grid()
    if solid is not None:
        mask = np.ascontiguousarray(np.asarray(solid).reshape(nz, ny, nx) != 0, dtype=np.uint8)
        g._solid = mask  # the C side holds a pointer into it
        g.solid = mask.ctypes.data
    g.Q, g.nx, g.ny, g.nz = Q, nx, ny, nz
    for i in range(6):
        g.face[i] = int(faces[i])
        for d in range(3):
            g.u_wall[i][d] = 0.0 if u_wall is None else float(u_wall[i][d])
    for face, (axis, lo, hi) in (edge or {}).items():
        g.edge_axis[face] = int(axis) + 1
        g.edge_scale[face][0], g.edge_scale[face][1] = float(lo), float(hi)
    return g


def make_params(r: Rates, force=(0.0, 0.0, 0.0), period=0.0, p_face=None, p_amp=None,
                p_period=0.0) -> Params:
    """p_face / p_amp: pressure of each NEQ_PRESSURE face,
    p_face + p_amp cos(2 pi n / p_period) (constant if p_period <= 0)."""
    p = Params()
    p.rates = r
    for d in range(3):
        p.force[d] = float(force[d])
    p.period = float(period)
    for f in range(6):
        p.p_face[f] = 0.0 if p_face is None else float(p_face[f])
        p.p_amp[f] = 0.0 if p_amp is None else float(p_amp[f])
    p.p_period = float(p_period)
    return p


def init_equilibrium(g: Grid, u=None, p=None) -> np.ndarray:
    N = g.nx * g.ny * g.nz
    f = np.zeros(g.Q * N)
    uu = None if u is None else np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
    pp = None if p is None else np.ascontiguousarray(p, dtype=np.float64).reshape(-1)
    _check(lib().oracle_init_equilibrium(
        ctypes.byref(g), None if uu is None else _dp(uu),
        None if pp is None else _dp(pp), _dp(f)))
    return f.reshape(g.Q, g.nz, g.ny, g.nx)


def step(g: Grid, prm: Params, n: int, f, nthreads: int = 1) -> np.ndarray:
    fin = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty_like(fin)
    _check(lib().oracle_step(ctypes.byref(g), ctypes.byref(prm), int(n),
                             _dp(fin), _dp(out), int(nthreads)))
    return out


def run(g: Grid, prm: Params, f, n0: int, nsteps: int, nthreads: int = None) -> np.ndarray:
    """Advance f (canonical pre-collision populations at step n0) by nsteps."""
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    nthreads = max(1, min(int(nthreads), g.nz))
    out = np.array(f, dtype=np.float64, order="C", copy=True)
    _check(lib().oracle_run(ctypes.byref(g), ctypes.byref(prm), int(n0),
                            int(nsteps), _dp(out), int(nthreads)))
    return out


def macroscopic(g: Grid, prm: Params, n: int, f):
    """u (3, nz, ny, nx) and p (nz, ny, nx) of the populations at step n."""
    fin = np.ascontiguousarray(f, dtype=np.float64)
    N = g.nx * g.ny * g.nz
    u = np.zeros(3 * N)
    p = np.zeros(N)
    _check(lib().oracle_macroscopic(ctypes.byref(g), ctypes.byref(prm), int(n),
                                    _dp(fin), _dp(u), _dp(p)))
    return u.reshape(3, g.nz, g.ny, g.nx), p.reshape(g.nz, g.ny, g.nx)
