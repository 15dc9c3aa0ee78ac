"""CPU checks of the CUDA step's own per-cell code, compiled for the host
(tests/host_emulation.cu), against the FP64 oracle.  They catch arithmetic
and indexing mistakes in the kernel source before it reaches a GPU; the GPU
parity tests then check the device build itself."""
import ctypes
import glob
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_1503_03337_gb300 import build as pkg_build, inputs

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "host_emulation.cu")


@pytest.fixture(scope="module")
def emu():
    out_dir = os.path.join(ROOT, "_build")
    os.makedirs(out_dir, exist_ok=True)
    lib = os.path.join(out_dir, "libhost_emulation.so")
    deps = [SRC] + glob.glob(os.path.join(ROOT, "paper_1503_03337_gb300", "csrc", "*.cuh"))
    if not os.path.exists(lib) or os.path.getmtime(lib) < max(map(os.path.getmtime, deps)):
        tmp = lib + ".tmp%d" % os.getpid()
        subprocess.run([pkg_build.nvcc(), "-std=c++20", "-O2", "--expt-relaxed-constexpr",
                        "-Xcompiler", "-fPIC", "-shared", "-x", "cu", SRC, "-o", tmp], check=True)
        os.replace(tmp, lib)
    L = ctypes.CDLL(lib)
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    L.emu_step.argtypes = [ctypes.c_int, ctypes.c_int, vp, ctypes.c_int, ctypes.c_int,
                           ctypes.c_int, ip, ctypes.c_int, ctypes.c_int, ip, dp, dp, dp, dp,
                           ctypes.c_int64]
    L.emu_canonical.argtypes = [ctypes.c_int, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ip,
                                ctypes.c_int, ctypes.c_int, ip, dp, dp, dp, ctypes.c_int64,
                                ctypes.c_int]
    L.emu_canonical_storage.argtypes = [ctypes.c_int, ctypes.c_int, vp, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int, ip, ctypes.c_int,
                                        ctypes.c_int, ip, dp, dp, dp, ctypes.c_int64,
                                        ctypes.c_int]
    L.emu_collide.argtypes = [ctypes.c_int, dp, dp, dp]
    L.emu_solid_links.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_int, ctypes.c_int, vp, vp]
    L.emu_set_solid.argtypes = [vp]
    L.emu_set_wide.argtypes = [ctypes.c_int]
    L.emu_neq.argtypes = [ctypes.c_int, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ip,
                          ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, dp, dp,
                          ctypes.c_int64]
    return L


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@pytest.mark.parametrize("Q", (14, 18, 26))
def test_collide_matches_oracle(emu, Q):
    rng = np.random.default_rng(21)
    for _ in range(50):
        r = rng.uniform(0.3, 1.9, size=6)
        f = rng.normal(size=Q) * 0.05 + 0.02
        F = rng.normal(size=3) * 1e-3
        got = f.copy()
        assert emu.emu_collide(Q, _d(r), _d(got), _d(F)) == 0
        ref = oracle.collide(Q, oracle.Rates(*r), f, F)
        np.testing.assert_allclose(got, ref, atol=2e-16, rtol=1e-14)


class EmuDomain:
    def __init__(self, emu, case):
        self.emu, self.case = emu, case
        self.per = np.array([int(case.faces[2 * k] == inputs.PERIODIC) for k in range(3)],
                            dtype=np.int32)
        self.moving = sum(1 << f for f in range(6) if case.faces[f] == inputs.MOVING_WALL)
        self.sym = sum(1 << f for f in range(6) if case.faces[f] == inputs.SYMMETRY)
        self.eaxis = np.zeros(6, dtype=np.int32)
        self.escale = np.ones((6, 2))
        for face, (axis, first, last) in (case.edge or {}).items():
            self.eaxis[face] = axis + 1
            self.escale[face] = (first, last)
        self.uw = np.ascontiguousarray(
            np.where(np.array(case.faces)[:, None] == inputs.MOVING_WALL, case.u_wall, 0.0))
        s = oracle.rates(case.Q, oracle.s_nu_of(case.nu))
        self.s = np.array([s.sc, s.se, s.sq, s.snu, s.spi, s.st])
        self.A = np.zeros((case.Q, case.nz, case.ny, case.nx))
        self.n = 0

    def _geom(self):
        """per, moving, sym, edge axes, edge scales, wall velocities"""
        return (self.per.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), self.moving, self.sym,
                self.eaxis.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _d(self.escale),
                _d(self.uw))

    def put(self, f, n):
        self.n = n
        c = self.case
        canon = np.ascontiguousarray(f, dtype=np.float64)
        assert self.emu.emu_canonical(c.Q, self.A.ctypes.data, c.nx, c.ny, c.nz, *self._geom(),
                                      _d(canon), n, 1) == 0

    def get(self):
        c = self.case
        out = np.zeros_like(self.A)
        assert self.emu.emu_canonical(c.Q, self.A.ctypes.data, c.nx, c.ny, c.nz, *self._geom(),
                                      _d(out), self.n, 0) == 0
        return out

    def step(self, k):
        c = self.case
        for _ in range(k):
            amp = np.cos(2 * np.pi * self.n / c.period) if c.period > 0 else 1.0
            F = np.array(c.force, dtype=np.float64) * amp
            assert self.emu.emu_step(c.Q, 0, self.A.ctypes.data, c.nx, c.ny, c.nz, *self._geom(),
                                     _d(self.s), _d(F), self.n) == 0
            self.n += 1


EDGE = [
    ("ragged", (13, 7, 5), (1, 2, 0, 0, 2, 1), None),
    ("periodic", (6, 5, 4), (0, 0, 0, 0, 0, 0), None),
    ("thin_x_periodic", (1, 6, 5), (0, 0, 1, 2, 1, 1), None),
    ("thin_x_walls", (1, 4, 3), (1, 1, 2, 1, 0, 0), None),
    ("two_cells", (2, 2, 2), (2, 2, 2, 2, 2, 2), None),
    ("lid", (5, 6, 4), (1, 1, 1, 2, 1, 1), None),
    # wide enough for whole 32-cell x-ranges away from the x faces, which
    # take the interior offset tables
    ("wide_x", (70, 4, 3), (1, 2, 1, 2, 0, 0), None),
    # symmetry faces (3): against walls, moving walls and each other, on
    # thin axes, and on the x faces of 32-cell x-ranges
    ("sym_lid", (5, 6, 4), (1, 3, 1, 2, 3, 1), None),
    ("sym_corner", (4, 5, 6), (3, 1, 3, 2, 1, 3), None),
    ("sym_periodic", (6, 4, 5), (0, 0, 3, 3, 2, 1), None),
    ("sym_thin", (1, 5, 2), (3, 3, 2, 3, 3, 1), None),
    ("sym_wide_x", (70, 3, 4), (3, 2, 1, 3, 0, 0), None),
    # edge profiles of moving faces (the lid corner velocities of Sec. 4.3),
    # with symmetry faces, on thin axes and on long rows
    ("edge_lid", (5, 6, 4), (1, 1, 1, 2, 1, 3), {3: (0, 0.3, 1.0)}),
    ("edge_multi", (4, 3, 5), (2, 1, 1, 2, 3, 2), {3: (2, 0.2, 0.6), 0: (1, 1.5, -0.5),
                                                   5: (0, 0.0, 2.0)}),
    ("edge_thin", (1, 4, 3), (1, 1, 1, 2, 1, 1), {3: (0, 0.4, 0.9)}),
    ("edge_wide_x", (70, 3, 4), (1, 1, 1, 2, 0, 0), {3: (0, 0.3, 1.0)}),
]


@pytest.mark.parametrize("wide", (False, True))
@pytest.mark.parametrize("Q", (14, 18, 26))
@pytest.mark.parametrize("name,shape,faces,edge", EDGE)
def test_step_matches_oracle(emu, Q, name, shape, faces, edge, wide):
    """The step's per-cell code, with 32-bit and with 64-bit (WIDE)
    population offsets, against the oracle."""
    emu.emu_set_wide(int(wide))
    try:
        _step_matches_oracle(emu, Q, name, shape, faces, edge)
    finally:
        emu.emu_set_wide(0)


def _step_matches_oracle(emu, Q, name, shape, faces, edge):
    rng = np.random.default_rng(5)
    uw = rng.normal(size=(6, 3)) * 0.03
    case = inputs.Case(name, Q, shape[0], shape[1], shape[2], tuple(faces), uw,
                       nu=0.05, force=(1e-4, -2e-4, 5e-5), period=17.0, storage="f64",
                       edge=edge)
    g = oracle.make_grid(Q, *shape, faces=faces, u_wall=uw, edge=edge)
    prm = oracle.make_params(oracle.rates(Q, oracle.s_nu_of(case.nu)), force=case.force, period=case.period)
    u0, p0 = inputs.random_state(case, seed=2)
    f0 = oracle.init_equilibrium(g, u0, p0)
    d = EmuDomain(emu, case)
    d.put(f0, 0)
    np.testing.assert_array_equal(d.get(), f0)
    f = f0
    for k in (1, 1, 5, 30):
        d.step(k)
        f = oracle.run(g, prm, f, d.n - k, k, nthreads=1)
        ref = f
        got = d.get()
        assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref)), (d.n,)


@pytest.mark.parametrize("Q", (14, 18, 26))
def test_restore_at_odd_parity(emu, Q):
    """Canonical populations written at an odd step read back unchanged."""
    faces = (1, 2, 0, 0, 2, 1)
    case = inputs.Case("r", Q, 5, 4, 3, faces, np.full((6, 3), 0.01), nu=0.1)
    d = EmuDomain(emu, case)
    f = inputs.random_populations(Q, (3, 4, 5), seed=1)
    d.put(f, 7)
    np.testing.assert_allclose(d.get(), f, atol=1e-17)


@pytest.mark.parametrize("storage,dtype,tol", ((1, np.float32, 2e-6), (2, np.float16, 3e-3)))
@pytest.mark.parametrize("Q", (14, 18, 26))
@pytest.mark.parametrize("name,shape,faces,edge", [e for e in EDGE if e[0] in
                                                   ("sym_lid", "sym_corner", "edge_multi",
                                                    "sym_wide_x")])
@pytest.mark.parametrize("wide", (False, True))
def test_reduced_storage_step_matches_oracle(emu, Q, name, shape, faces, edge, storage, dtype,
                                             tol, wide):
    """FP32 and FP16 storage (FP32 arithmetic) of the kernel's per-cell code
    with symmetry faces and edge profiles: 7 steps from a seeded state
    against the FP64 oracle, to the storage precision."""
    rng = np.random.default_rng(8)
    uw = rng.normal(size=(6, 3)) * 0.03
    case = inputs.Case(name, Q, shape[0], shape[1], shape[2], tuple(faces), uw,
                       nu=0.05, force=(1e-4, -2e-4, 5e-5), period=17.0, storage="f64",
                       edge=edge)
    g = oracle.make_grid(Q, *shape, faces=faces, u_wall=uw, edge=edge)
    prm = oracle.make_params(oracle.rates(Q, oracle.s_nu_of(case.nu)), force=case.force, period=case.period)
    u0, p0 = inputs.random_state(case, seed=2)
    f0 = oracle.init_equilibrium(g, u0, p0)
    d = EmuDomain(emu, case)
    A = np.zeros(d.A.shape, dtype=dtype)
    canon = np.ascontiguousarray(f0, dtype=np.float64)
    assert emu.emu_canonical_storage(Q, storage, A.ctypes.data, *shape, *d._geom(), _d(canon),
                                     0, 1) == 0
    emu.emu_set_wide(int(wide))
    try:
        for n in range(7):
            amp = np.cos(2 * np.pi * n / case.period)
            F = np.array(case.force, dtype=np.float64) * amp
            assert emu.emu_step(Q, storage, A.ctypes.data, *shape, *d._geom(), _d(d.s),
                                _d(F), n) == 0
    finally:
        emu.emu_set_wide(0)
    out = np.zeros_like(canon)
    assert emu.emu_canonical_storage(Q, storage, A.ctypes.data, *shape, *d._geom(), _d(out),
                                     7, 0) == 0
    ref = oracle.run(g, prm, f0, 0, 7, nthreads=1)
    assert np.max(np.abs(out - ref)) <= tol * np.max(np.abs(ref))


NEQ = [
    # (name, shape, faces): 4 = extrapolation velocity face, 5 = pressure face
    ("duct", (9, 5, 6), (5, 5, 4, 4, 4, 4)),
    ("cavity", (7, 8, 6), (4, 4, 4, 4, 4, 4)),
    ("mixed", (6, 7, 5), (5, 5, 1, 2, 0, 0)),
    ("sym", (5, 6, 7), (0, 0, 4, 4, 1, 3)),
    ("open", (8, 3, 5), (5, 4, 0, 0, 4, 2)),
    ("wide_x", (70, 4, 5), (5, 5, 4, 2, 0, 0)),
]


@pytest.mark.parametrize("oscillate", (False, True))
@pytest.mark.parametrize("Q", (14, 18, 26))
@pytest.mark.parametrize("name,shape,faces", NEQ)
def test_extrapolation_boundaries_match_oracle(emu, Q, name, shape, faces, oscillate):
    """The fused step followed by the kernel's extrapolation pass (the
    per-node code of the boundary kernel, run node after node), FP64,
    random state, wall velocities and face pressures: within 1e-12 of the
    oracle after 1, 2, 7 and 30 steps."""
    rng = np.random.default_rng(len(name) + 10 * Q)
    uw = rng.normal(size=(6, 3)) * 0.02
    pf = rng.normal(size=6) * 0.01
    pa = rng.normal(size=6) * 0.005 if oscillate else np.zeros(6)
    period = 17.0 if oscillate else 0.0
    case = inputs.Case(name, Q, shape[0], shape[1], shape[2], tuple(faces), uw, nu=0.05,
                       force=(1e-4, -5e-5, 2e-5), period=13.0, storage="f64")
    g = oracle.make_grid(Q, *shape, faces=faces, u_wall=uw)
    prm = oracle.make_params(oracle.rates(Q, oracle.s_nu_of(case.nu)), force=case.force,
                             period=case.period, p_face=pf, p_amp=pa, p_period=period)
    u0, p0 = inputs.random_state(case, seed=3)
    f = oracle.init_equilibrium(g, u0, p0)
    d = EmuDomain(emu, case)
    d.put(f, 0)
    vel = sum(1 << k for k in range(6) if faces[k] == 4)
    pre = sum(1 << k for k in range(6) if faces[k] == 5)
    uw_all = np.ascontiguousarray(np.where((np.array(faces) == 4)[:, None] |
                                           (np.array(faces) == 2)[:, None], uw, 0.0))
    for k in (1, 1, 5, 23):
        for _ in range(k):
            d.step(1)
            n = d.n
            amp = np.cos(2 * np.pi * n / case.period)
            F = np.array(case.force) * amp
            pb = pf + pa * (np.cos(2 * np.pi * n / period) if period > 0 else 0.0)
            assert emu.emu_neq(Q, d.A.ctypes.data, *shape, d.per.ctypes.data_as(
                ctypes.POINTER(ctypes.c_int)), d.moving, d.sym, _d(uw_all), vel, pre,
                _d(np.ascontiguousarray(pb)), _d(F), n) == 0
        f = oracle.run(g, prm, f, d.n - k, k, nthreads=1)
        got = d.get()
        assert np.max(np.abs(got - f)) <= 1e-12 * np.max(np.abs(f)), (d.n,)


SOLID = [
    # (name, shape, faces, solid fraction): random solid nodes with every
    # face kind that combines with them, odd and even layouts
    ("periodic", (9, 7, 6), (0, 0, 0, 0, 0, 0), 0.3),
    ("walls", (8, 6, 7), (1, 2, 1, 1, 0, 0), 0.2),
    ("sym", (7, 6, 5), (3, 1, 0, 0, 2, 3), 0.25),
    ("wide_x", (70, 4, 4), (1, 1, 2, 1, 0, 0), 0.15),
    ("dense", (6, 6, 6), (0, 0, 1, 1, 3, 3), 0.6),
]


@pytest.mark.parametrize("wide", (False, True))
@pytest.mark.parametrize("Q", (14, 18, 26))
@pytest.mark.parametrize("name,shape,faces,frac", SOLID)
def test_solid_nodes_match_oracle(emu, Q, name, shape, faces, frac, wide):
    """The kernel's per-cell code with a random solid-node mask (link words
    built by the device builder's per-cell code) against the oracle's solid
    mask: FP64, random state, wall velocities and force, 1, 2, 7 and 30
    steps, fluid and solid nodes alike (solid nodes read zero)."""
    rng = np.random.default_rng(len(name) + Q)
    solid = (rng.random(shape[::-1]) < frac).astype(np.uint8)
    uw = rng.normal(size=(6, 3)) * 0.03
    case = inputs.Case(name, Q, shape[0], shape[1], shape[2], tuple(faces), uw, nu=0.05,
                       force=(1e-4, -2e-4, 5e-5), period=17.0, storage="f64")
    g = oracle.make_grid(Q, *shape, faces=faces, u_wall=uw, solid=solid)
    prm = oracle.make_params(oracle.rates(Q, oracle.s_nu_of(case.nu)), force=case.force,
                             period=case.period)
    u0, p0 = inputs.random_state(case, seed=2)
    f = oracle.init_equilibrium(g, u0, p0)
    d = EmuDomain(emu, case)
    links = np.zeros(shape[::-1], dtype=np.uint32)
    per = int(d.per[0]) | (int(d.per[1]) << 1) | (int(d.per[2]) << 2)
    assert emu.emu_solid_links(Q, *shape, per, d.sym, solid.ctypes.data, links.ctypes.data) == 0
    emu.emu_set_solid(links.ctypes.data)
    emu.emu_set_wide(int(wide))
    try:
        d.put(f, 0)
        for k in (1, 1, 5, 23):
            d.step(k)
            f = oracle.run(g, prm, f, d.n - k, k, nthreads=1)
            got = d.get()
            got[:, solid.astype(bool)] = 0.0  # the read path reports solids as zero
            assert np.max(np.abs(got - f)) <= 1e-12 * np.max(np.abs(f)), (d.n,)
    finally:
        emu.emu_set_solid(None)
        emu.emu_set_wide(0)
