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

PERIODIC, WALL, MOVING_WALL, SYMMETRY = 0, 1, 2, 3
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

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def s_nu(self) -> float:
        return 1.0 / (3.0 * self.nu + 0.5)


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
    tol: float          # requested accuracy (picks FP32 below 1e-3, else FP16)
    max_steps: int

    @property
    def storage(self) -> str:
        return "f32" if self.tol < 1e-3 else "f16"


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
        return cavity(r.Q, r.L, 400.0, U=0.05, storage=r.storage)
    if r.kind == "duct":
        return duct(r.Q, r.L, max(4, r.L // 4), nu=0.1, u_max=0.02, storage=r.storage)
    # pulsatile: T = 1000 steps, eta = 4, amplitude from the quasi-steady
    # square-duct relation, so that u stays O(0.02)
    b = r.L / 2.0
    nu = b * b * (2.0 * np.pi / 1000.0) / 16.0
    A = 0.02 * nu / (SQUARE_DUCT_K * b * b)
    return pulsatile(r.Q, r.L, max(4, r.L // 4), 1000, 4.0, A, storage=r.storage, u_ref=0.02)
