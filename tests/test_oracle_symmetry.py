"""Symmetry (free-slip) faces of the oracle, pinned against its wall
streaming: a box that is mirror-symmetric about a mid-plane computes, in its
lower half, what the half box computes with a symmetry face on that plane
(the ghost beyond a symmetry face mirrors the node across the plane)."""
import numpy as np
import pytest

import oracle
from paper_1503_03337_gb300 import inputs

W, P, M, S = oracle.WALL, oracle.PERIODIC, oracle.MOVING_WALL, oracle.SYMMETRY


def run(Q, shape, faces, uw, force, steps, u0=None):
    nx, ny, nz = shape
    g = oracle.make_grid(Q, nx, ny, nz, faces=faces, u_wall=uw)
    prm = oracle.make_params(oracle.rates(Q, oracle.s_nu_of(0.05)), force=force)
    f = oracle.run(g, prm, oracle.init_equilibrium(g, u0, None), 0, steps)
    u, p = oracle.macroscopic(g, prm, steps, f)
    return u, p


@pytest.mark.parametrize("Q", (14, 18))
def test_half_cavity_equals_full_cavity(Q):
    """Lid-driven box 10 x 8 x 12 (walls, lid on y+ along x) against its
    half 10 x 8 x 6 with a symmetry face at z+: identical lower halves."""
    uw = np.zeros((6, 3))
    uw[3] = (0.05, 0.0, 0.0)
    full_faces = (W, W, W, M, W, W)
    half_faces = (W, W, W, M, W, S)
    uf, pf = run(Q, (10, 8, 12), full_faces, uw, (0, 0, 0), 60)
    uh, ph = run(Q, (10, 8, 6), half_faces, uw, (0, 0, 0), 60)
    scale = np.max(np.abs(uf))
    assert scale > 1e-3
    np.testing.assert_allclose(uh, uf[:, :6], rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(ph, pf[:6], rtol=0, atol=1e-12)
    # the full box itself is mirror-symmetric: u_z odd, u_x, u_y even
    np.testing.assert_allclose(uf[2, ::-1], -uf[2], atol=1e-12 * scale)
    np.testing.assert_allclose(uf[0, ::-1], uf[0], atol=1e-12 * scale)


@pytest.mark.parametrize("Q", (14, 18))
def test_half_channel_with_symmetry_planes(Q):
    """Body-force channel between walls at y- and y+ (x, z periodic), from a
    random symmetric start, against the half channel with a symmetry face at
    y+; and a symmetry face on a low side (y-) against the upper half."""
    rng = np.random.default_rng(7)
    ny = 8
    u0 = rng.normal(size=(3, 3, ny, 5)) * 0.01
    u0 = 0.5 * (u0 + u0[:, :, ::-1] * np.array([1, -1, 1])[:, None, None, None])
    full = run(Q, (5, ny, 3), (P, P, W, W, P, P), None, (2e-5, 0, 0), 40, u0)[0]
    lo = run(Q, (5, ny // 2, 3), (P, P, W, S, P, P), None, (2e-5, 0, 0), 40,
             np.ascontiguousarray(u0[:, :, : ny // 2]))[0]
    hi = run(Q, (5, ny // 2, 3), (P, P, S, W, P, P), None, (2e-5, 0, 0), 40,
             np.ascontiguousarray(u0[:, :, ny // 2:]))[0]
    scale = np.max(np.abs(full))
    np.testing.assert_allclose(lo, full[:, :, : ny // 2], atol=1e-12 * scale, rtol=0)
    np.testing.assert_allclose(hi, full[:, :, ny // 2:], atol=1e-12 * scale, rtol=0)
