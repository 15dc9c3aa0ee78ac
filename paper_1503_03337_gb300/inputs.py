"""Seeded synthetic workloads shaped like the paper's flows (Sec. 4).

This module only describes inputs: grid sizes, boundary kinds, viscosities,
force amplitudes, seeded random states and request traces.  It contains none
of the method's arithmetic, so both the CUDA path and the oracle can use it.

Recipes (lattice units, c = 1):
  * duct       -- square cross-section n x n with walls on x and y, z periodic,
                  constant body force F_z chosen so the analytic centre-line
                  velocity is u_max: F = u_max nu / (K a^2), a = n/2, with
                  K = 0.29468541 the square-duct constant of the Sec. 4.1 series
                  (pinned against the series in the oracle's tests).
  * cavity     -- cube with the y+ face moving at U along x, other faces walls,
                  nu = U L / Re.
  * half_cavity -- the cavity's z <= 1/2 half, symmetry face on the mid-plane.
  * pulsatile  -- as duct but F_z(t) = A cos(2 pi t / T), nu = b^2 (2 pi/T) / eta^2.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Tuple

import numpy as np

SQUARE_DUCT_K = 0.2946854131

PERIODIC, WALL, MOVING_WALL, SYMMETRY, NEQ_VELOCITY, NEQ_PRESSURE = 0, 1, 2, 3, 4, 5
XM, XP, YM, YP, ZM, ZP = range(6)


@dataclasses.dataclass
class Case:
    """One domain: everything needed to set it up on either side."""
    name: str
    Q: int
    nx: int
    ny: int
    nz: int
    faces: Tuple[int, ...]
    u_wall: np.ndarray            # (6, 3)
    nu: float
    force: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    period: float = 0.0
    storage: str = "f32"
    u_ref: float = 0.0            # velocity scale for error bounds
    init_u: Optional[np.ndarray] = None   # (3, nz, ny, nx) or None (rest)
    init_p: Optional[np.ndarray] = None   # (nz, ny, nx) or None
    rounding: int = 0             # 16-bit stores: 0 nearest, 1 stochastic
    edge: Optional[dict] = None   # {face: (axis, scale_first, scale_last)}
    # pressure of NEQ_PRESSURE faces: p_face + p_amp cos(2 pi n / p_period)
    p_face: Tuple[float, ...] = (0.0,) * 6
    p_amp: Tuple[float, ...] = (0.0,) * 6
    p_period: float = 0.0
    c: float = 1.0  # lattice speed dx/dt of a recipe given in physical units
    p_ref: float = 0.0  # pressure the stored populations are deviations from
    solid: Optional[np.ndarray] = None  # (nz, ny, nx) uint8, nonzero = solid node

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz



def cavity(Q: int, n: int, Re: float, U: float = 0.05, storage: str = "f32",
           ny: Optional[int] = None, nz: Optional[int] = None) -> Case:
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    faces = [WALL] * 6
    faces[YP] = MOVING_WALL
    uw = np.zeros((6, 3))
    uw[YP] = (U, 0.0, 0.0)
    return Case("cavity", Q, n, ny, nz, tuple(faces), uw, nu=U * n / Re,
                storage=storage, u_ref=U)


KU_LID_EDGE = (0.3, 1.0)  # lid velocity / U next to x = 0 and x = 1 (Sec. 4.3)


def half_cavity(Q: int, n: int, Re: float, U: float = 0.05, storage: str = "f32",
                ku_lid: bool = False) -> Case:
    """The z <= 1/2 half of the cavity with a symmetry face on the mid-plane
    z+ (the reduced domain of Sec. 4.3, Eq. z05symmetry): n x n x ceil(n/2)
    nodes, so that the mirrored box is n x n x 2*ceil(n/2).  ku_lid: the lid
    velocity over the first and last x columns is scaled by KU_LID_EDGE (the
    corner setting of Sec. 4.3)."""
    c = cavity(Q, n, Re, U, storage, nz=(n + 1) // 2)
    c.name = "half_cavity"
    c.faces = c.faces[:ZP] + (SYMMETRY,)
    if ku_lid:
        c.edge = {YP: (0,) + KU_LID_EDGE}
    return c


def duct(Q: int, n: int, nz: int, nu: float, u_max: float = 0.02,
         storage: str = "f32") -> Case:
    a = n / 2.0
    F = u_max * nu / (SQUARE_DUCT_K * a * a)
    faces = (WALL, WALL, WALL, WALL, PERIODIC, PERIODIC)
    return Case("duct", Q, n, n, nz, faces, np.zeros((6, 3)), nu=nu,
                force=(0.0, 0.0, F), storage=storage, u_ref=u_max)


def pulsatile(Q: int, n: int, nz: int, period: int, eta: float, amplitude: float,
              storage: str = "f32", u_ref: float = 0.03) -> Case:
    b = n / 2.0
    nu = b * b * (2.0 * np.pi / period) / eta ** 2
    faces = (WALL, WALL, WALL, WALL, PERIODIC, PERIODIC)
    return Case("pulsatile", Q, n, n, nz, faces, np.zeros((6, 3)), nu=nu,
                force=(0.0, 0.0, amplitude), period=float(period),
                storage=storage, u_ref=u_ref)


def pressure_duct(Q: int, dx: float, inv_tau: float, nu: float = 0.03, length: float = 2.0,
                  half_width: float = 0.5, p_in: float = 1.1, p_out: float = 1.0,
                  storage: str = "f64") -> Case:
    """The pressure-driven square duct of Sec. 4.1 on its node grid: nodes on
    the walls y, z = +-a and on the inlet / outlet planes x = 0, l, spacing
    dx (l/dx + 1 by 2a/dx + 1 by 2a/dx nodes), viscosity nu, s_nu = 1/tau,
    inlet and outlet pressures p_in, p_out (the paper's 1.1 and 1.0), all
    converted to lattice units with c = dx / dt, dt = nu_lattice dx^2 / nu,
    nu_lattice = (tau - 1/2) / 3.  Walls use the extrapolation velocity
    boundary, inlet and outlet the extrapolation pressure boundary.  Start
    from rest at the mean pressure, inlet and outlet planes at theirs.
    Stored populations are deviations from the mean pressure (p_ref)."""
    tau = 1.0 / inv_tau
    dt = (tau - 0.5) / 3.0 * dx * dx / nu
    c = dx / dt
    nx, ny = int(round(length / dx)) + 1, int(round(2 * half_width / dx)) + 1
    faces = (NEQ_PRESSURE, NEQ_PRESSURE) + (NEQ_VELOCITY,) * 4
    case = Case("pressure_duct", Q, nx, ny, ny, faces, np.zeros((6, 3)),
                nu=(tau - 0.5) / 3.0, storage=storage, u_ref=0.0)
    case.p_face = (p_in / c ** 2, p_out / c ** 2, 0.0, 0.0, 0.0, 0.0)
    p0 = np.full((ny, ny, nx), 0.5 * (p_in + p_out) / c ** 2)
    p0[:, :, 0] = p_in / c ** 2
    p0[:, :, -1] = p_out / c ** 2
    case.init_p = p0
    case.c = c
    case.p_ref = 0.5 * (p_in + p_out) / c ** 2
    return case


def pressure_pulsatile(Q: int, dx: float, dt: float, tau: float, period: float = 100.0,
                       delta_p: float = 0.001, length: float = 2.0, half_width: float = 0.5,
                       p_out: float = 1.0, storage: str = "f64") -> Case:
    """The pressure-driven pulsatile channel of Sec. 4.2 on its node grid
    (the duct of pressure_duct): outlet pressure p_out, inlet pressure
    p_out - delta_p cos(2 pi t / period), so that dp/dx = G cos(w t) with
    G = delta_p / length (Eq. pbc-pul); spacing dx, time step dt, s_nu =
    1/tau; lattice units with c = dx / dt.  Start from rest at the mean of
    the t = 0 inlet and outlet pressures, the end planes at theirs; stored
    populations are deviations from the outlet pressure (p_ref).  Its
    physical viscosity is (tau - 1/2)/3 dx^2 / dt."""
    c = dx / dt
    nx, ny = int(round(length / dx)) + 1, int(round(2 * half_width / dx)) + 1
    faces = (NEQ_PRESSURE, NEQ_PRESSURE) + (NEQ_VELOCITY,) * 4
    case = Case("pressure_pulsatile", Q, nx, ny, ny, faces, np.zeros((6, 3)),
                nu=(tau - 0.5) / 3.0, storage=storage, u_ref=0.0)
    case.p_face = (p_out / c ** 2, p_out / c ** 2, 0.0, 0.0, 0.0, 0.0)
    case.p_amp = (-delta_p / c ** 2, 0.0, 0.0, 0.0, 0.0, 0.0)
    case.p_period = period / dt
    p0 = np.full((ny, ny, nx), (p_out - 0.5 * delta_p) / c ** 2)
    p0[:, :, 0] = (p_out - delta_p) / c ** 2
    p0[:, :, -1] = p_out / c ** 2
    case.init_p = p0
    case.c = c
    case.p_ref = p_out / c ** 2
    return case


def porous_spheres(Q: int, n: int, radius: float = 6.0, solid_fraction: float = 0.3,
                   seed: int = 0, storage: str = "f32", force: float = 1e-6) -> Case:
    """A periodic n^3 box filled with randomly placed solid spheres (seeded
    centres, overlaps allowed, periodic images) until about solid_fraction
    of the nodes are solid; flow driven by a body force along x.  The
    porous-medium geometry the paper's introduction motivates."""
    rng = np.random.default_rng(seed)
    solid = np.zeros((n, n, n), dtype=bool)
    r = int(np.ceil(radius))
    off = np.arange(-r, r + 1)
    dz, dy, dx = np.meshgrid(off, off, off, indexing="ij")
    ball = dx ** 2 + dy ** 2 + dz ** 2 <= radius ** 2
    bz, by, bx = dz[ball], dy[ball], dx[ball]
    flat = solid.reshape(-1)
    while solid.mean() < solid_fraction:
        # a batch of spheres at a time; the last batch may overshoot a little
        k = max(1, int((solid_fraction - solid.mean()) * n ** 3 / len(bx) * 0.5) + 1)
        x0, y0, z0 = (rng.integers(0, n, size=(3, k, 1)))
        flat[(((z0 + bz) % n) * n + (y0 + by) % n) * n + (x0 + bx) % n] = True
    case = Case("porous", Q, n, n, n, (PERIODIC,) * 6, np.zeros((6, 3)), nu=0.05,
                force=(force, 0.0, 0.0), storage=storage, u_ref=0.0)
    case.solid = solid.astype(np.uint8)
    return case


def random_state(case: Case, seed: int, u_scale: float = 0.02, p_scale: float = 0.01):
    """Seeded smooth-ish random (u, p) fields for equilibrium initialisation."""
    rng = np.random.default_rng(seed)
    shape = (case.nz, case.ny, case.nx)
    u = rng.normal(size=(3,) + shape) * u_scale
    p = rng.normal(size=shape) * p_scale
    return u, p


def random_populations(Q: int, shape, seed: int, scale: float = 0.01, offset: float = 0.02):
    rng = np.random.default_rng(seed)
    return offset + scale * rng.normal(size=(Q,) + tuple(shape))


# ---- batched and serving workloads -----------------------------------------

@dataclasses.dataclass
class BatchDomain:
    kind: str
    Q: int
    L: int
    Re: float
    storage: str


def batch_draw(n_domains: int = 256, seed: int = 0, lmin: int = 24, lmax: int = 160) -> List[BatchDomain]:
    """256 independent cavities/ducts: type and Q with p = 1/2 each, side
    L ~ U{lmin..lmax}, Re ~ U(100, 1000), storage FP32 or FP16 with p = 1/2."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_domains):
        kind = "cavity" if rng.random() < 0.5 else "duct"
        Q = 14 if rng.random() < 0.5 else 18
        L = int(rng.integers(lmin, lmax + 1))
        Re = float(rng.uniform(100.0, 1000.0))
        storage = "f32" if rng.random() < 0.5 else "f16"
        out.append(BatchDomain(kind, Q, L, Re, storage))
    return out


def batch_case(d: BatchDomain) -> Case:
    if d.kind == "cavity":
        return cavity(d.Q, d.L, d.Re, U=0.05, storage=d.storage)
    nu = 0.02 * d.L / d.Re  # duct: Re = U_max L / nu with U_max = 0.02
    return duct(d.Q, d.L, d.L, nu, u_max=0.02, storage=d.storage)


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float      # seconds from trace start
    kind: str
    Q: int
    L: int
    tol: float          # requested accuracy: max |u - u_exact| / U of the delivered field
    max_steps: int

    @property
    def storage(self) -> str:
        """FP16 (stochastic rounding) where its measured error fits the
        request: within 1e-3 U on ducts and oscillating channels, within
        1e-2 U on cavities (whose lid corners amplify storage rounding);
        FP32 (within 1e-5 U) otherwise."""
        fp16_error = 1e-2 if self.kind == "cavity" else 1e-3
        return "f16" if self.tol >= fp16_error else "f32"


def request_trace(n_requests: int, rate: float = 200.0, seed: int = 0, lmin: int = 32,
                  lmax: int = 256, max_steps: int = 2000) -> List[Request]:
    """Poisson arrivals (mean `rate` per second) of cavity/duct/pulsatile
    requests, side uniform in [lmin, lmax], Q uniform in {14, 18}, requested
    tolerance log-uniform in [1e-5, 1e-2]."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n_requests):
        t += rng.exponential(1.0 / rate)
        kind = ("cavity", "duct", "pulsatile")[int(rng.integers(0, 3))]
        Q = 14 if rng.random() < 0.5 else 18
        L = int(rng.integers(lmin, lmax + 1))
        tol = float(10 ** rng.uniform(-5, -2))
        out.append(Request(i, t, kind, Q, L, tol, max_steps))
    return out


def request_case(r: Request) -> Case:
    if r.kind == "cavity":
        c = cavity(r.Q, r.L, 400.0, U=0.05, storage=r.storage)
    elif r.kind == "duct":
        c = duct(r.Q, r.L, max(4, r.L // 4), nu=0.1, u_max=0.02, storage=r.storage)
    else:
        # pulsatile: T = 1000 steps, eta = 4, amplitude from the quasi-steady
        # square-duct relation, so that u stays O(0.02)
        b = r.L / 2.0
        nu = b * b * (2.0 * np.pi / 1000.0) / 16.0
        A = 0.02 * nu / (SQUARE_DUCT_K * b * b)
        c = pulsatile(r.Q, r.L, max(4, r.L // 4), 1000, 4.0, A, storage=r.storage, u_ref=0.02)
    if c.storage == "f16":
        c.rounding = 1  # stochastic
    return c
