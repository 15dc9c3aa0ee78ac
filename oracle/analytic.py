"""Analytic solutions and error norms of Sec. 4 (TEST INFRASTRUCTURE ONLY).

* ``duct_velocity``      -- steady rectangular-duct Poiseuille series (Sec. 4.1)
* ``pulsatile_velocity`` -- oscillating-pressure-gradient rectangular channel
                            series, Eq. wa (Sec. 4.2)
* ``gre_u``              -- global relative L2 velocity error, Eq. ed
* ``residual_*``         -- convergence criteria Eq. sc, Eq. cr and
                            Eq. cavity_creterion

Coordinates follow the paper: the cross-section is -a <= y <= a,
-b <= z <= b and the flow runs along x with dp/dx = -G (steady) or
dp/dx = G cos(w t) (pulsatile).
"""
from __future__ import annotations

import numpy as np


def _cosh_ratio(k, s, h):
    """cosh(k s) / cosh(k h) for |s| <= h, k with Re k >= 0, overflow-free."""
    s = np.abs(s)
    return (np.exp(k * (s - h)) * (1.0 + np.exp(-2.0 * k * s))
            / (1.0 + np.exp(-2.0 * k * h)))


def duct_velocity(y, z, a, b, nu, G, nterms=2001):
    """Steady axial velocity of Sec. 4.1 for pressure gradient dp/dx = -G.

    u = 16 a^2 G / (nu pi^3) sum_{i odd} (-1)^((i-1)/2)
        [1 - cosh(i pi z / 2a) / cosh(i pi b / 2a)] cos(i pi y / 2a) / i^3
    """
    y = np.asarray(y, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    acc = np.zeros(np.broadcast(y, z).shape)
    for i in range(1, 2 * nterms, 2):
        k = i * np.pi / (2.0 * a)
        sign = -1.0 if ((i - 1) // 2) % 2 else 1.0
        acc = acc + sign * (1.0 - _cosh_ratio(k, z, b)) * np.cos(k * y) / i ** 3
    return 16.0 * a * a * G / (nu * np.pi ** 3) * acc


def duct_umax(a, b, nu, G):
    """Centre-line (maximum) velocity of the steady duct flow."""
    return float(duct_velocity(0.0, 0.0, a, b, nu, G))


def pulsatile_amplitude(y, z, a, b, nu, omega, G, tol=1e-17, nmax=200000):
    """Complex amplitude U(y,z) of Eq. wa, so that u = Re{U exp(i w t)}.

    U = i G/w { 1 - 2 sum_n (-1)^n / p_n [ cosh(g_n y/b) cos(p_n z/b) / cosh(g_n a/b)
                                        + cosh(s_n z/b) cos(q_n y/b) / cosh(s_n) ] }
    with g_n = sqrt(p_n^2 + i eta^2), s_n = sqrt(q_n^2 + i eta^2),
    p_n = (2n+1) pi / 2, q_n = (2n+1) pi b / (2a), eta = b sqrt(w/nu).
    The series is summed until a block of 64 terms adds less than ``tol``
    relative to the running sum everywhere (it converges slowly at the walls).
    """
    y = np.asarray(y, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    y, z = np.broadcast_arrays(y, z)
    eta2 = b * b * omega / nu
    acc = np.zeros(y.shape, dtype=np.complex128)
    n = 0
    block = 64
    while n < nmax:
        ns = np.arange(n, n + block, dtype=np.float64)
        pn = (2.0 * ns + 1.0) * np.pi / 2.0
        qn = (2.0 * ns + 1.0) * np.pi * b / (2.0 * a)
        gn = np.sqrt(pn * pn + 1j * eta2)
        sn = np.sqrt(qn * qn + 1j * eta2)
        sign = np.where(ns.astype(np.int64) % 2 == 0, 1.0, -1.0)
        yy = y[..., None]
        zz = z[..., None]
        term = (sign / pn) * (
            _cosh_ratio(gn / b, yy, a) * np.cos(pn * zz / b)
            + _cosh_ratio(sn / b, zz, b) * np.cos(qn * yy / b))
        add = term.sum(axis=-1)
        acc = acc + add
        n += block
        if np.max(np.abs(add)) <= tol * max(1.0, float(np.max(np.abs(acc)))):
            break
    return 1j * G / omega * (1.0 - 2.0 * acc)


def pulsatile_velocity(y, z, t, a, b, nu, omega, G, **kw):
    """Axial velocity of Eq. wa at time t for dp/dx = G cos(w t)."""
    U = pulsatile_amplitude(y, z, a, b, nu, omega, G, **kw)
    return np.real(U * np.exp(1j * omega * t))


def womersley(b, omega, nu):
    """eta = b sqrt(w / nu) (Sec. 4.2)."""
    return b * np.sqrt(omega / nu)


def gre_u(u_num, u_ana):
    """Eq. ed: sqrt(sum |u_n - u_a|^2) / sqrt(sum |u_a|^2) over all nodes and
    components (arrays of any matching shape)."""
    u_num = np.asarray(u_num, dtype=np.float64)
    u_ana = np.asarray(u_ana, dtype=np.float64)
    return float(np.sqrt(np.sum((u_num - u_ana) ** 2)) / np.sqrt(np.sum(u_ana ** 2)))


def residual_steady(u_new, u_old):
    """Eq. sc: sum |u(t+dt) - u(t)| / sum |u(t)| (one velocity component)."""
    return float(np.sum(np.abs(u_new - u_old)) / np.sum(np.abs(u_old)))


def residual_periodic(u_new, u_old):
    """Eq. cr: sum |u(t+T) - u(t)| / sum |u(t+T)|."""
    return float(np.sum(np.abs(u_new - u_old)) / np.sum(np.abs(u_new)))


def residual_cavity(u_new, u_old):
    """Eq. cavity_creterion: as Eq. cr but summed over all three components;
    arrays are (3, ...)."""
    return float(np.sum(np.abs(u_new - u_old)) / np.sum(np.abs(u_new)))


def lattice_coords(n):
    """Node centres of a halfway-walled axis with n fluid nodes, measured from
    the channel centre: i + 1/2 - n/2, so the half-width is n/2."""
    return np.arange(n, dtype=np.float64) + 0.5 - n / 2.0
