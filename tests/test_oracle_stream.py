"""Pins of the oracle's streaming and boundary rules on tiny grids.

Streaming is isolated by a collision that does nothing (S = 0, F = 0), then
compared with a per-link table built here from the boundary rules: a link whose source node lies beyond a wall carries the cell's
own reflected population plus 6 w (c . u_wall), u_wall scaled by the face's
edge profile in the first and last node columns; across a symmetry face the
source is the node's mirror image and the pulled population the mirror one.
"""
import itertools

import numpy as np
import pytest

import oracle

P, W, M, S = oracle.PERIODIC, oracle.WALL, oracle.MOVING_WALL, oracle.SYMMETRY
ZERO = oracle.Rates(0, 0, 0, 0, 0, 0)


def link_table(Q, n, faces, u_wall, edge=None):
    """Expected pulled value of every (a, node) as ('src', b, node') or
    ('wall', abar, node, correction)."""
    c = oracle.velocities(Q)
    w, _ = oracle.weights(Q)
    find = {tuple(v): b for b, v in enumerate(c)}
    opp = [find[tuple(-c[a])] for a in range(Q)]
    table = {}
    for z, y, x in itertools.product(range(n[2]), range(n[1]), range(n[0])):
        node = (x, y, z)
        for a in range(Q):
            src = [x - c[a][0], y - c[a][1], z - c[a][2]]
            beyond = []
            cm = c[a].copy()  # velocity of the pulled population
            for d in range(3):
                out = 2 * d if src[d] < 0 else 2 * d + 1 if src[d] >= n[d] else None
                if out is None:
                    continue
                if faces[out] == P:
                    src[d] %= n[d]
                elif faces[out] == S:
                    src[d] = node[d]
                    cm[d] = -cm[d]
                else:
                    beyond.append(out)
            if not beyond:
                table[(a, z, y, x)] = ("src", find[tuple(cm)], (src[2], src[1], src[0]))
            else:
                uw = np.zeros(3)
                for face in sorted(beyond):
                    if faces[face] == M:
                        uw = np.asarray(u_wall[face], dtype=float)
                        if edge and face in edge:
                            k, first, last = edge[face]
                            uw = uw * (first if node[k] == 0 else
                                       last if node[k] == n[k] - 1 else 1.0)
                        break
                table[(a, z, y, x)] = ("wall", opp[a], (z, y, x), 6.0 * w[a] * (c[a] @ uw))
    return table


CASES = [
    ((3, 3, 3), (W, W, W, W, W, W), None),
    ((4, 3, 5), (P, P, W, W, P, P), None),
    ((3, 4, 4), (W, W, W, M, W, W), None),
    ((4, 4, 3), (M, W, P, P, W, M), None),
    ((2, 3, 4), (P, P, P, P, P, P), None),
    # symmetry faces against walls, moving walls, periodic axes, each other
    ((3, 4, 4), (W, S, W, M, S, W), None),
    ((4, 3, 3), (S, S, P, P, M, S), None),
    ((1, 3, 2), (S, S, S, M, W, S), None),
    # edge profiles of moving faces (the lid corner velocities of Sec. 4.3)
    ((5, 4, 3), (W, W, W, M, W, W), {3: (0, 0.3, 0.7)}),
    ((4, 3, 5), (M, W, W, M, S, M), {3: (2, 0.2, 0.6), 0: (1, 1.5, -0.5), 5: (0, 0.0, 2.0)}),
    ((1, 4, 3), (W, W, W, M, W, W), {3: (0, 0.4, 0.9)}),
]


@pytest.mark.parametrize("Q", (14, 18))
@pytest.mark.parametrize("n,faces,edge", CASES)
def test_streaming_matches_link_table(Q, n, faces, edge):
    rng = np.random.default_rng(11)
    u_wall = rng.normal(size=(6, 3)) * 0.05
    g = oracle.make_grid(Q, *n, faces=faces, u_wall=u_wall, edge=edge)
    prm = oracle.make_params(ZERO)
    f = rng.normal(size=(Q, n[2], n[1], n[0]))
    out = oracle.step(g, prm, 0, f)
    for key, rule in link_table(Q, n, faces, u_wall, edge).items():
        if rule[0] == "src":
            expect = f[(rule[1],) + rule[2]]
        else:
            expect = f[(rule[1],) + rule[2]] + rule[3]
        assert abs(out[key] - expect) < 1e-15, (key, rule)


@pytest.mark.parametrize("Q", (14, 18))
def test_mass_conserved_with_walls(Q):
    """Collision and stationary bounce-back conserve sum_x P exactly."""
    rng = np.random.default_rng(12)
    g = oracle.make_grid(Q, 5, 4, 6, faces=(W, W, W, W, P, P))
    prm = oracle.make_params(oracle.rates(Q, 1.3))
    f = 0.02 + 0.01 * rng.normal(size=(Q, 6, 4, 5))
    m0 = f.sum()
    f = oracle.run(g, prm, f, 0, 200, nthreads=1)
    assert abs(f.sum() - m0) < 1e-12 * abs(m0)


@pytest.mark.parametrize("Q", (14, 18))
def test_mass_conserved_with_profiled_lid(Q):
    """A tangential lid whose velocity is scaled in its first and last
    columns (the scale belongs to the cell, so every link of a cell sees
    one wall velocity) still conserves sum_x P exactly."""
    rng = np.random.default_rng(13)
    u_wall = np.zeros((6, 3))
    u_wall[3] = (0.08, 0.0, 0.03)
    g = oracle.make_grid(Q, 6, 5, 4, faces=(W, W, W, M, S, W), u_wall=u_wall,
                         edge={3: (0, 0.3, 1.7)})
    prm = oracle.make_params(oracle.rates(Q, 1.3))
    f = 0.02 + 0.01 * rng.normal(size=(Q, 4, 5, 6))
    m0 = f.sum()
    f = oracle.run(g, prm, f, 0, 200, nthreads=1)
    assert abs(f.sum() - m0) < 1e-12 * abs(m0)


@pytest.mark.parametrize("Q", (14, 18))
def test_rest_stays_at_rest(Q):
    g = oracle.make_grid(Q, 4, 5, 3, faces=(W, W, W, W, W, W))
    prm = oracle.make_params(oracle.rates(Q, 1.1))
    p0 = np.full((3, 5, 4), 0.37)
    f = oracle.init_equilibrium(g, None, p0)
    out = oracle.run(g, prm, f, 0, 50, nthreads=1)
    np.testing.assert_allclose(out, f, atol=1e-15)


@pytest.mark.parametrize("Q", (14, 18))
def test_periodic_box_force_closed_form(Q):
    """Fully periodic box from rest with constant F: j^n = n F, so
    u^n = (n + 1/2) F, to round-off."""
    g = oracle.make_grid(Q, 3, 4, 2, faces=(P,) * 6)
    F = np.array([1e-4, -2e-5, 3e-5])
    prm = oracle.make_params(oracle.rates(Q, 0.7), force=F)
    f = oracle.init_equilibrium(g)
    for n in (1, 7, 40):
        fn = oracle.run(g, prm, f, 0, n, nthreads=1)
        u, _ = oracle.macroscopic(g, prm, n, fn)
        for d in range(3):
            np.testing.assert_allclose(u[d], (n + 0.5) * F[d], rtol=1e-12, atol=1e-18)


@pytest.mark.parametrize("Q", (14, 18))
def test_couette_profile_linear(Q):
    """Plane Couette flow between a wall at y = -1/2 and a wall moving at U
    at y = ny - 1/2 (halfway walls): the steady profile is linear,
    u_x = U (y + 1/2) / ny, which halfway bounce-back reproduces exactly."""
    ny, U = 8, 0.01
    u_wall = np.zeros((6, 3))
    u_wall[3] = (U, 0.0, 0.0)
    g = oracle.make_grid(Q, 2, ny, 2, faces=(P, P, W, M, P, P), u_wall=u_wall)
    nu = 0.4
    prm = oracle.make_params(oracle.rates(Q, oracle.s_nu_of(nu)))
    f = oracle.init_equilibrium(g)
    f = oracle.run(g, prm, f, 0, 4000, nthreads=1)
    u, _ = oracle.macroscopic(g, prm, 4000, f)
    y = np.arange(ny) + 0.5
    np.testing.assert_allclose(u[0, 0, :, 0], U * y / ny, rtol=1e-9, atol=1e-14)
    assert np.max(np.abs(u[1:])) < 1e-12


@pytest.mark.parametrize("Q", (14, 18))
def test_duct_mirror_symmetry(Q):
    """A square duct driven along z is symmetric under x -> -x and y -> -y."""
    n = 6
    g = oracle.make_grid(Q, n, n, 2, faces=(W, W, W, W, P, P))
    prm = oracle.make_params(oracle.rates(Q, 1.25), force=(0, 0, 1e-4))
    f = oracle.run(g, prm, oracle.init_equilibrium(g), 0, 300, nthreads=1)
    u, p = oracle.macroscopic(g, prm, 300, f)
    np.testing.assert_allclose(u[2], u[2][:, ::-1, :], rtol=1e-12, atol=1e-18)
    np.testing.assert_allclose(u[2], u[2][:, :, ::-1], rtol=1e-12, atol=1e-18)
    np.testing.assert_allclose(u[0], -u[0][:, :, ::-1], rtol=1e-9, atol=1e-18)
    np.testing.assert_allclose(p, p[:, ::-1, :], rtol=1e-9, atol=1e-18)
