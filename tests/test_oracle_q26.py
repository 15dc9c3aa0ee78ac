"""The oracle's iD3Q26 model: the 26 velocities of D3Q27 without c_0, built
by the construction of Sec. 3 (the moment polynomials on the velocity set,
Gram-Schmidt orthogonalised; m_eq = T f_eq), which App. B's closing remark
says also gives a 26-velocity model.  The paper prints no iD3Q26 values, so
the pins are the mathematics the construction must satisfy, the LBGK limit
(the 26-velocity form of He and Luo's incompressible model), and the
hydrodynamics: the duct flow converges to the analytic series at second
order with the viscosity of Eq. vis."""
import itertools

import numpy as np
import pytest

import oracle
import test_oracle_algebra as alg
from test_oracle_analytic import duct_run, duct_steps

Q = 26


def test_velocity_set_is_d3q27_without_rest():
    c = oracle.velocities(Q)
    rows = {tuple(v) for v in c}
    full = {v for v in itertools.product((-1, 0, 1), repeat=3)} - {(0, 0, 0)}
    assert len(c) == 26 and rows == full
    for a in range(0, 6, 2):  # axis directions, each followed by its opposite
        assert tuple(-c[a]) == tuple(c[a + 1])
    # the face and cube diagonals in the order of D3Q18 and D3Q14
    np.testing.assert_array_equal(c[6:18], oracle.velocities(18)[6:18])
    np.testing.assert_array_equal(c[18:26], oracle.velocities(14)[6:14])
    w, w0 = oracle.weights(Q)
    n2 = np.sum(c * c, axis=1)
    assert w0 == pytest.approx(8 / 27, abs=0)
    for k, wk in ((1, 2 / 27), (2, 1 / 54), (3, 1 / 216)):  # D3Q27 weights
        assert np.all(np.abs(w[n2 == k] - wk) < 1e-17)


def test_weights_isotropy():
    alg.test_weights_isotropy(Q)


def test_transform_orthogonal_and_conserved_rows():
    """Integer rows (denominators cleared), exactly orthogonal."""
    T = oracle.transform(Q)
    c = oracle.velocities(Q).astype(float)
    G = T @ T.T
    assert np.count_nonzero(G - np.diag(np.diag(G))) == 0
    assert np.all(np.diag(G) > 0)
    np.testing.assert_array_equal(T[0], np.ones(Q))
    for row, k in ((2, 0), (4, 1), (6, 2)):
        np.testing.assert_array_equal(T[row], c[:, k])
    Tinv = T.T @ np.diag(1.0 / np.diag(G))
    np.testing.assert_allclose(T @ Tinv, np.eye(Q), atol=1e-13)


def test_basis_spans_every_function_of_the_velocities():
    """26 independent rows: T is invertible, so no information is lost (the
    dropped c_x^2 c_y^2 c_z^2 is dependent on these velocities)."""
    T = oracle.transform(Q)
    assert np.linalg.matrix_rank(T) == 26


@pytest.mark.parametrize("fn", [alg.test_equilibrium_moments_match_edf,
                                alg.test_pressure_inverts_equilibrium,
                                alg.test_collision_conserves_P_and_j,
                                alg.test_collision_reduces_to_lbgk,
                                alg.test_equilibrium_is_fixed_point,
                                alg.test_force_adds_exact_momentum,
                                alg.test_force_source_second_moment,
                                alg.test_pressure_shift_invariance])
def test_collision_properties(fn):
    fn(Q)


def test_duct_gre_and_order():
    """Steady duct with body force: GRE_u of a 16x16 cross-section below
    3e-2 and second-order convergence over 8/16/32, with nu from Eq. vis."""
    nu = 0.1
    errs = [duct_run(Q, N, 1, nu, 0.02, duct_steps(N, nu)) for N in (8, 16, 32)]
    assert errs[1] < 3e-2
    slope = np.polyfit(np.log([8, 16, 32]), np.log(errs), 1)[0]
    assert slope < -1.8, errs
