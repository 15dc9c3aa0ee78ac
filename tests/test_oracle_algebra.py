"""Pins of the oracle's model tables and one-cell collision.

Each check compares the oracle against something other than itself: the
paper's Gram-Schmidt basis formulas, textbook lattice isotropy, the printed
velocity-space equilibrium (Eq. edf) and the special cases the paper names.
"""
import itertools

import numpy as np
import pytest

import oracle

QS = (14, 18)


def phi_rows(Q, c):
    """Basis vectors of Sec. 3 (Q14, Eq. m after orthogonalisation) and
    App. B (Q18, Eq. appendix_m18), evaluated on the velocity set c."""
    cx, cy, cz = c[:, 0].astype(float), c[:, 1].astype(float), c[:, 2].astype(float)
    n2 = cx * cx + cy * cy + cz * cz
    one = np.ones_like(cx)
    if Q == 14:
        return np.array([
            one, 7 * n2 / 2 - 15 * one / 2,
            cx, (5 * n2 - 13) * cx / 2,
            cy, (5 * n2 - 13) * cy / 2,
            cz, (5 * n2 - 13) * cz / 2,
            3 * cx ** 2 - n2, cy ** 2 - cz ** 2,
            cx * cy, cy * cz, cx * cz, cx * cy * cz])
    return np.array([
        one, 3 * n2 - 5 * one,
        cx, (5 * n2 - 9) * cx,
        cy, (5 * n2 - 9) * cy,
        cz, (5 * n2 - 9) * cz,
        3 * cx ** 2 - n2, (3 * n2 - 5) * (3 * cx ** 2 - n2),
        cy ** 2 - cz ** 2, (3 * n2 - 5) * (cy ** 2 - cz ** 2),
        cx * cy, cy * cz, cx * cz,
        (cy ** 2 - cz ** 2) * cx, (cz ** 2 - cx ** 2) * cy, (cx ** 2 - cy ** 2) * cz])


@pytest.mark.parametrize("Q", QS)
def test_velocity_set_shape(Q):
    c = oracle.velocities(Q)
    assert c.shape == (Q, 3)
    rows = {tuple(v) for v in c}
    assert len(rows) == Q and (0, 0, 0) not in rows
    axis = {v for v in itertools.product((-1, 0, 1), repeat=3) if sum(map(abs, v)) == 1}
    if Q == 14:
        diag = {v for v in itertools.product((-1, 1), repeat=3)}
    else:
        diag = {v for v in itertools.product((-1, 0, 1), repeat=3) if sum(map(abs, v)) == 2}
    assert rows == axis | diag
    # c_1..c_6 are the axis directions, each followed by its opposite
    for a in range(0, 6, 2):
        assert tuple(-c[a]) == tuple(c[a + 1])


@pytest.mark.parametrize("Q", QS)
def test_transform_equals_gram_schmidt_basis(Q):
    """The printed T (Eq. T14 / App. B) equals the orthogonal basis formulas."""
    T = oracle.transform(Q)
    np.testing.assert_array_equal(T, phi_rows(Q, oracle.velocities(Q)).astype(np.int64))


@pytest.mark.parametrize("Q", QS)
def test_transform_orthogonal_and_inverse(Q):
    T = oracle.transform(Q).astype(float)
    G = T @ T.T
    assert np.count_nonzero(G - np.diag(np.diag(G))) == 0
    Tinv = T.T @ np.diag(1.0 / np.diag(G))
    np.testing.assert_allclose(T @ Tinv, np.eye(Q), atol=1e-15)
    np.testing.assert_allclose(Tinv @ T, np.eye(Q), atol=1e-15)


@pytest.mark.parametrize("Q", QS)
def test_weights_isotropy(Q):
    """With the rest weight w0, the weights satisfy the standard lattice
    isotropy conditions up to fourth order with c_s^2 = 1/3."""
    w, w0 = oracle.weights(Q)
    c = oracle.velocities(Q).astype(float)
    cs2 = 1.0 / 3.0
    assert abs(w0 + w.sum() - 1.0) < 1e-15
    d = np.eye(3)
    for i in range(3):
        assert abs(np.sum(w * c[:, i])) < 1e-15
        for j in range(3):
            assert abs(np.sum(w * c[:, i] * c[:, j]) - cs2 * d[i, j]) < 1e-15
            for k in range(3):
                assert abs(np.sum(w * c[:, i] * c[:, j] * c[:, k])) < 1e-15
                for l in range(3):
                    m4 = np.sum(w * c[:, i] * c[:, j] * c[:, k] * c[:, l])
                    ref = cs2 ** 2 * (d[i, j] * d[k, l] + d[i, k] * d[j, l] + d[i, l] * d[j, k])
                    assert abs(m4 - ref) < 1e-15


def feq_edf(Q, p, u):
    """Eq. edf with lambda_a = w_a p / c_s^2, written out in the test."""
    w, _ = oracle.weights(Q)
    c = oracle.velocities(Q).astype(float)
    cu = c @ u
    cs2 = 1.0 / 3.0
    return w * p / cs2 + w * (cu / cs2 + cu ** 2 / (2 * cs2 ** 2) - u @ u / (2 * cs2))


@pytest.mark.parametrize("Q", QS)
def test_equilibrium_moments_match_edf(Q):
    """Printed closed-form m_eq (Eq. meq / App. B) equals T f_eq (Eq. edf)."""
    rng = np.random.default_rng(1)
    T = oracle.transform(Q).astype(float)
    for _ in range(20):
        u = rng.normal(size=3) * 0.1
        p = rng.normal() * 0.3
        np.testing.assert_allclose(oracle.feq(Q, p, u), feq_edf(Q, p, u), atol=1e-16, rtol=1e-14)
        np.testing.assert_allclose(T @ feq_edf(Q, p, u), oracle.moment_equilibrium(Q, p, u),
                                   atol=1e-15)


@pytest.mark.parametrize("Q", QS)
def test_pressure_inverts_equilibrium(Q):
    """Eq. hgl applied to f_eq(p,u) returns p and u."""
    rng = np.random.default_rng(2)
    c = oracle.velocities(Q).astype(float)
    for _ in range(20):
        u = rng.normal(size=3) * 0.1
        p = rng.normal() * 0.3
        f = feq_edf(Q, p, u)
        np.testing.assert_allclose(c.T @ f, u, atol=1e-16)
        assert abs(oracle.pressure(Q, f.sum(), u) - p) < 1e-15


def random_rates(Q, rng):
    return oracle.Rates(*(rng.uniform(0.3, 1.9, size=6)))


@pytest.mark.parametrize("Q", QS)
def test_collision_conserves_P_and_j(Q):
    """P and j are collision invariants without force (Sec. 3, App. A),
    for any s_c."""
    rng = np.random.default_rng(3)
    c = oracle.velocities(Q).astype(float)
    for _ in range(20):
        f = rng.normal(size=Q) * 0.05 + 0.03
        fp = oracle.collide(Q, random_rates(Q, rng), f)
        assert abs(fp.sum() - f.sum()) < 1e-15
        np.testing.assert_allclose(c.T @ fp, c.T @ f, atol=1e-15)


@pytest.mark.parametrize("Q", QS)
def test_collision_reduces_to_lbgk(Q):
    """S = (1/tau) I turns the MRT step into the LBGK step of Eq. ee."""
    rng = np.random.default_rng(4)
    c = oracle.velocities(Q).astype(float)
    for _ in range(20):
        tau = rng.uniform(0.51, 3.0)
        s = 1.0 / tau
        f = rng.normal(size=Q) * 0.05 + 0.02
        u = c.T @ f
        _, w0 = oracle.weights(Q)
        p = (1.0 / 3.0) / (1.0 - w0) * (f.sum() - w0 * (u @ u) * 1.5)
        ref = f - (f - feq_edf(Q, p, u)) / tau
        got = oracle.collide(Q, oracle.Rates(s, s, s, s, s, s), f)
        np.testing.assert_allclose(got, ref, atol=1e-15)


@pytest.mark.parametrize("Q", QS)
def test_equilibrium_is_fixed_point(Q):
    rng = np.random.default_rng(5)
    for _ in range(10):
        u = rng.normal(size=3) * 0.05
        p = rng.normal() * 0.1
        f = feq_edf(Q, p, u)
        np.testing.assert_allclose(oracle.collide(Q, random_rates(Q, rng), f), f, atol=1e-16)


@pytest.mark.parametrize("Q", QS)
def test_force_adds_exact_momentum(Q):
    """With u = j + F/2 and the (I - S/2) Guo source, j* = j + F for any s_c,
    and P is unchanged (the P row of the Guo source is dropped)."""
    rng = np.random.default_rng(6)
    c = oracle.velocities(Q).astype(float)
    for _ in range(20):
        f = rng.normal(size=Q) * 0.05 + 0.03
        F = rng.normal(size=3) * 1e-3
        fp = oracle.collide(Q, random_rates(Q, rng), f, F)
        np.testing.assert_allclose(c.T @ fp, c.T @ f + F, atol=1e-15)
        assert abs(fp.sum() - f.sum()) < 1e-15


@pytest.mark.parametrize("Q", QS)
def test_force_source_second_moment(Q):
    """Guo's source gives the momentum flux u F + F u.  With the P row of the
    source dropped the deviatoric part is untouched, mass is not
    injected, and the trace loses exactly the P-row share
    3 w0 (u.F) sum|c|^2 / Q.  Checked at S = 0 so that only the source acts."""
    rng = np.random.default_rng(7)
    c = oracle.velocities(Q).astype(float)
    _, w0 = oracle.weights(Q)
    n2sum = float(np.sum(c * c))
    for _ in range(10):
        f = rng.normal(size=Q) * 0.05 + 0.03
        F = rng.normal(size=3) * 1e-3
        zero = oracle.Rates(0, 0, 0, 0, 0, 0)
        fp = oracle.collide(Q, zero, f, F)
        u = c.T @ f + F / 2
        flux = np.einsum('a,ai,aj->ij', fp - f, c, c)
        full = np.outer(u, F) + np.outer(F, u)
        dev = lambda A: A - np.trace(A) / 3.0 * np.eye(3)
        np.testing.assert_allclose(dev(flux), dev(full), atol=1e-15)
        assert abs(np.sum(fp - f)) < 1e-15
        expect_tr = np.trace(full) - 3.0 * w0 * (u @ F) * n2sum / Q
        assert abs(np.trace(flux) - expect_tr) < 1e-15


@pytest.mark.parametrize("Q", QS)
def test_pressure_shift_invariance(Q):
    """f -> f + 3 w dp commutes with the collision."""
    rng = np.random.default_rng(8)
    w, _ = oracle.weights(Q)
    for _ in range(10):
        f = rng.normal(size=Q) * 0.05
        F = rng.normal(size=3) * 1e-3
        dp = rng.normal()
        r = random_rates(Q, rng)
        a = oracle.collide(Q, r, f + 3 * w * dp, F)
        b = oracle.collide(Q, r, f, F) + 3 * w * dp
        np.testing.assert_allclose(a, b, atol=1e-14)
