"""The oracle's non-equilibrium extrapolation boundaries (Sec. 4: the scheme
the paper applies in all its runs) and its pressure drive (Sec. 4.1, 4.2).

Pins: the boundary nodes carry exactly the prescribed velocity (velocity
faces) or pressure (pressure faces); an equilibrium at rest with equal
pressures is a fixed point; and the whole scheme reproduces the paper's
Table 1 (GRE_u of the pressure-driven Poiseuille duct at dx = 1/8 and 1/16
for 1/tau = 0.8, 1.0, 1.3) to the printed digits, and Table 3's iD3Q14
GRE_u of the pressure-driven pulsatile channel at dp = 0.001 to its two
printed digits."""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import analytic as an
from paper_1503_03337_gb300 import inputs

from lbm_cases import oracle_setup

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "paper_values.json")


def half_unit_of_last_digit(printed):
    """Half a unit in the last of the four significant digits the paper prints."""
    return 0.5 * 10.0 ** (np.floor(np.log10(abs(printed))) - 3)


def steady(case, tol=1e-10, check=10, max_steps=200000):
    """Run to the steady-state criterion of Eq. sc (x velocity, one step
    apart), tested every `check` steps."""
    g, prm = oracle_setup(case)
    f = oracle.init_equilibrium(g, case.init_u, case.init_p)
    n = 0
    while n < max_steps:
        f = oracle.run(g, prm, f, n, check - 1)
        u1, _ = oracle.macroscopic(g, prm, n + check - 1, f)
        f = oracle.run(g, prm, f, n + check - 1, 1)
        n += check
        u2, _ = oracle.macroscopic(g, prm, n, f)
        if an.residual_steady(u2[0], u1[0]) <= tol:
            return g, prm, f, n, u2
    raise AssertionError("no steady state within %d steps" % max_steps)


def duct_gre(case, u, length=2.0, a=0.5, nu=0.03, p_in=1.1, p_out=1.0):
    dx = 2 * a / (case.ny - 1)
    ys = -a + dx * np.arange(case.ny)
    Z, Y = np.meshgrid(ys, ys, indexing="ij")
    ua = np.zeros_like(u)
    ua[0] = (an.duct_velocity(Y, Z, a, a, nu, (p_in - p_out) / length) / case.c)[:, :, None]
    return an.gre_u(u, ua)


@pytest.mark.parametrize("Q", (14, 18))
def test_boundary_nodes_take_prescribed_values(Q):
    """After any step: u = u_wall on velocity-face nodes (p taken from the
    inward neighbour), p = the face pressure on pressure-face nodes (u taken
    from the inward neighbour), and a node where the two meet takes both."""
    case = inputs.pressure_duct(Q, 1.0 / 8, 1.0)
    case.u_wall = np.zeros((6, 3))
    case.u_wall[inputs.YP] = (0.01, 0.0, 0.003)  # a moving velocity face
    case.init_u, _ = inputs.random_state(case, seed=4, u_scale=0.01)
    g, prm = oracle_setup(case)
    f = oracle.run(g, prm, oracle.init_equilibrium(g, case.init_u, case.init_p), 0, 7)
    u, p = oracle.macroscopic(g, prm, 7, f)
    # y+ nodes that are not on the x- / x+ pressure planes or y-: the lid
    lid = u[:, 1:-1, -1, 1:-1]
    assert np.max(np.abs(lid[0] - 0.01)) < 1e-15 and np.max(np.abs(lid[2] - 0.003)) < 1e-15
    assert np.max(np.abs(lid[1])) < 1e-15
    # z- wall nodes off the pressure planes: at rest
    assert np.max(np.abs(u[:, 0, :-1, 1:-1])) < 1e-15
    # pressure planes: p exact, including their edges with the walls
    assert np.max(np.abs(p[:, :, 0] - case.p_face[0])) < 1e-15
    assert np.max(np.abs(p[:, :, -1] - case.p_face[1])) < 1e-15
    # inlet nodes off the walls take their inward neighbour's velocity
    # (the extrapolation sets u_b = u_f exactly)
    assert np.max(np.abs(u[:, 1:-1, 1:-1, 0] - u[:, 1:-1, 1:-1, 1])) < 1e-15


@pytest.mark.parametrize("Q", (14, 18))
def test_rest_state_is_fixed_point(Q):
    case = inputs.pressure_duct(Q, 1.0 / 8, 1.0, p_in=1.0, p_out=1.0)
    g, prm = oracle_setup(case)
    f0 = oracle.init_equilibrium(g, None, case.init_p)
    f = oracle.run(g, prm, f0, 0, 25)
    assert np.max(np.abs(f - f0)) < 1e-15


TABLE1 = [(inv_tau, k) for inv_tau in ("0.8", "1.0", "1.3") for k in (0, 1)]


@pytest.mark.parametrize("inv_tau,k", TABLE1)
def test_table1_reproduced(inv_tau, k):
    """Table 1: the iD3Q14 Poiseuille duct (Sec. 4.1: l = 2, a = b = 0.5,
    nu = 0.03, p_in = 1.1, p_out = 1.0, steady state by Eq. sc at 1e-10)
    gives the printed GRE_u (Eq. ed over every grid point) to the last
    printed digit."""
    gold = json.load(open(GOLDEN))["table1_orders"]
    dx = gold["dx"][k]
    printed = gold["gre_u"][inv_tau][k]
    case = inputs.pressure_duct(14, dx, float(inv_tau))
    _, _, _, _, u = steady(case)
    gre = duct_gre(case, u)
    assert abs(gre - printed) <= half_unit_of_last_digit(printed), (gre, printed)


def pulsatile_gre(case, u, n, delta_p, period=100.0, length=2.0, a=0.5):
    """Eq. ed against Eq. wa at t = n dt on the node grid; on the wall nodes
    the exact solution is the no-slip value 0 (the series only tends to it
    there, and at the duct's edges its partial sums stay at the core value)."""
    dx = 2 * a / (case.ny - 1)
    dt = dx / case.c
    nu = case.nu * dx * dx / dt
    ys = -a + dx * np.arange(case.ny)
    Z, Y = np.meshgrid(ys, ys, indexing="ij")
    omega = 2 * np.pi / period
    ua = an.pulsatile_velocity(Y, Z, n * dt, a, a, nu, omega, delta_p / length) / case.c
    ua[(np.abs(np.abs(Y) - a) < 1e-12) | (np.abs(np.abs(Z) - a) < 1e-12)] = 0.0
    u_ana = np.zeros_like(u)
    u_ana[0] = ua[:, :, None]
    return an.gre_u(u, u_ana)


def test_table3_reproduced_smallest_drop():
    """Table 3, iD3Q14 column, dp = 0.001 (Sec. 4.2: 41x21x21, dt = 0.05,
    c = 1, tau = 0.9, T = 100): the periodic state (Eq. cr over one period
    at 6e-14) gives the printed GRE_u at t = T to the last printed digit."""
    gold = json.load(open(GOLDEN))["table3_gre_u"]
    dp, printed = gold["delta_p"][0], gold["gre_u"][0]
    case = inputs.pressure_pulsatile(14, gold["dx"], gold["dt"], gold["tau"], gold["T"], dp)
    g, prm = oracle_setup(case)
    steps = int(round(case.p_period))
    f = oracle.init_equilibrium(g, None, case.init_p)
    n, u_prev = 0, oracle.macroscopic(g, prm, 0, f)[0]
    for _ in range(20):
        f = oracle.run(g, prm, f, n, steps)
        n += steps
        u = oracle.macroscopic(g, prm, n, f)[0]
        done = an.residual_periodic(u[0], u_prev[0]) <= 6e-14
        u_prev = u
        if done:
            break
    assert done
    gre = pulsatile_gre(case, u, n, dp)
    half = 0.5 * 10.0 ** (np.floor(np.log10(printed)) - 1)  # two printed digits
    assert abs(gre - printed) <= half, (gre, printed)
