"""Convergence criteria of Sec. 4 (Eq. sc, Eq. cr, Eq. cavity_creterion).

The oracle's residual helpers are pinned by a two-field case worked out by
hand; the library's lbm_stats_residual (a host-only C-ABI call, no GPU) is
checked against them on FP64 sums of seeded random fields, and its error
cases are checked."""
import ctypes

import numpy as np
import pytest

from oracle import analytic
from paper_1503_03337_gb300 import build, lbm


@pytest.fixture(scope="module")
def library():
    build.build()
    return lbm.load()


def test_oracle_residuals_hand_worked():
    # one component: u(t) = (1, -2, 3, 0), u(t + dt) = (1.5, -2, 2, -0.5)
    old = np.array([1.0, -2.0, 3.0, 0.0])
    new = np.array([1.5, -2.0, 2.0, -0.5])
    # sum |du| = 0.5 + 0 + 1 + 0.5 = 2; sum |old| = 6; sum |new| = 6
    assert analytic.residual_steady(new, old) == pytest.approx(2.0 / 6.0, rel=1e-15)
    new2 = np.array([1.5, -2.0, 2.5, -0.5])
    # sum |du| = 0.5 + 0 + 0.5 + 0.5 = 1.5; sum |new2| = 6.5, sum |old| = 6
    assert analytic.residual_steady(new2, old) == pytest.approx(1.5 / 6.0, rel=1e-15)
    assert analytic.residual_periodic(new2, old) == pytest.approx(1.5 / 6.5, rel=1e-15)
    # three components on two nodes: later level in the denominator, all
    # components summed together (not the mean of per-component ratios)
    old3 = np.array([[1.0, 0.0], [0.0, 2.0], [0.0, 0.0]])
    new3 = np.array([[1.0, 1.0], [0.0, 2.0], [1.0, 0.0]])
    # sum |du| = 1 + 1 = 2; sum |new3| = 1 + 1 + 2 + 1 = 5
    assert analytic.residual_cavity(new3, old3) == pytest.approx(2.0 / 5.0, rel=1e-15)


def stats_of(u_new, u_old, step=200, prev=100):
    s = lbm.lbm_stats()
    s.step, s.prev_step = step, prev
    for k in range(3):
        s.sum_abs_du[k] = float(np.sum(np.abs(u_new[k] - u_old[k])))
        s.sum_abs_u[k] = float(np.sum(np.abs(u_new[k])))
        s.sum_abs_u_prev[k] = float(np.sum(np.abs(u_old[k])))
    return s


def test_library_matches_oracle_forms(library):
    rng = np.random.default_rng(11)
    u_old = rng.normal(size=(3, 5, 6, 7)) * 0.02
    u_new = u_old + rng.normal(size=u_old.shape) * 1e-4
    s = stats_of(u_new, u_old)
    for k in range(3):
        assert lbm.lbm_stats_residual(s, lbm.LBM_RESIDUAL_STEADY, k) == pytest.approx(
            analytic.residual_steady(u_new[k], u_old[k]), rel=1e-14)
        assert lbm.lbm_stats_residual(s, lbm.LBM_RESIDUAL_PERIODIC, k) == pytest.approx(
            analytic.residual_periodic(u_new[k], u_old[k]), rel=1e-14)
    assert lbm.lbm_stats_residual(s, lbm.LBM_RESIDUAL_CAVITY) == pytest.approx(
        analytic.residual_cavity(u_new, u_old), rel=1e-14)


def test_library_residual_errors_and_zero_fields(library):
    z = np.zeros((3, 2, 2, 2))
    s = stats_of(z, z)
    assert lbm.lbm_stats_residual(s, lbm.LBM_RESIDUAL_CAVITY) == 0.0
    one = z.copy()
    one[0, 0, 0, 0] = 1.0
    s = stats_of(one, z)  # change against a zero earlier level
    assert lbm.lbm_stats_residual(s, lbm.LBM_RESIDUAL_STEADY, 0) == float("inf")
    assert lbm.lbm_stats_residual(s, lbm.LBM_RESIDUAL_PERIODIC, 0) == 1.0
    r = ctypes.c_double()
    s.prev_step = -1  # no earlier snapshot
    assert library.lbm_stats_residual(ctypes.byref(s), lbm.LBM_RESIDUAL_CAVITY, 0,
                                      ctypes.byref(r)) == lbm.LBM_EINVAL
    assert b"prev_step" in library.lbm_last_error()
    s.prev_step = 3
    assert library.lbm_stats_residual(ctypes.byref(s), 7, 0, ctypes.byref(r)) == lbm.LBM_EINVAL
    assert library.lbm_stats_residual(ctypes.byref(s), lbm.LBM_RESIDUAL_STEADY, 3,
                                      ctypes.byref(r)) == lbm.LBM_EINVAL
    assert library.lbm_stats_residual(None, 0, 0, ctypes.byref(r)) == lbm.LBM_EINVAL
    assert library.lbm_residual(None, 0, 0, ctypes.byref(r)) == lbm.LBM_EINVAL
    assert library.lbm_batch_residual(None, 0, 0, 0, ctypes.byref(r)) == lbm.LBM_EINVAL
