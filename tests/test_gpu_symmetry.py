"""The cavity setups of Sec. 4.3 on the GPU.  Symmetry (free-slip) faces:
the half cavity (Eq. z05symmetry) against the oracle's full, mirror-
symmetric cavity, and the reduced-precision half domains against their own
full boxes.  Edge profiles of moving faces (the lid corner velocities)
against the oracle."""
import zlib

import numpy as np
import pytest

from paper_1503_03337_gb300 import inputs, lbm

from lbm_cases import gpu_run, oracle_run, rel_max

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1503_03337_gb300 import build
    build.build()
    lbm.load()


def full_of(half):
    """The full box whose z < nz half the half case is (wall at z+)."""
    c = inputs.cavity(half.Q, half.nx, 1.0, storage=half.storage, nz=2 * half.nz)
    c.nu, c.u_wall, c.u_ref = half.nu, half.u_wall, half.u_ref
    return c


@pytest.mark.parametrize("Q", (14, 18, 26))
def test_fp64_half_cavity_equals_full_cavity(Q):
    """FP64 half cavity 17 x 17 x 9 on the GPU, 301 steps (odd), against
    the lower half of the oracle's full 17 x 17 x 18 box: populations and
    velocity to 1e-12."""
    half = inputs.half_cavity(Q, 17, 100.0, storage="f64")
    assert half.nz == 9 and half.faces[inputs.ZP] == inputs.SYMMETRY
    g = gpu_run(half, 301)
    o = oracle_run(full_of(half), 301)
    assert rel_max(g["u"], o["u"][:, : half.nz]) <= 1e-12
    assert rel_max(g["f"], o["f"][:, : half.nz]) <= 1e-12
    # and the oracle with the same symmetry face
    oh = oracle_run(half, 301)
    assert rel_max(g["f"], oh["f"]) <= 1e-12


@pytest.mark.parametrize("launch", ((64, 1, 1), (64, 2, 2)))
@pytest.mark.parametrize("storage,tol", (("f32", 1e-5), ("f16", 1e-2), ("bf16", 6e-2)))
@pytest.mark.parametrize("Q", (14, 18, 26))
def test_half_cavity_equals_full_box(Q, storage, tol, launch):
    """32- and 16-bit storage: the half cavity 48 x 48 x 24 and the lower
    half of the full 48 x 48 x 48 box on the GPU, both at the same
    precision, 500 steps: equal to `tol` U (the two differ only by rounding
    order, since neither box is exactly mirror-symmetric in rounded
    arithmetic)."""
    half = inputs.half_cavity(Q, 48, 400.0, storage=storage)
    full = full_of(half)
    h = gpu_run(half, 500, launch=launch)
    f = gpu_run(full, 500, launch=launch)
    assert np.all(np.isfinite(h["u"]))
    err = np.max(np.abs(h["u"] - f["u"][:, : half.nz]))
    assert err <= tol * half.u_ref, err
    assert np.max(np.abs(h["u"])) > 0.1 * half.u_ref


@pytest.mark.parametrize("Q", (14, 18, 26))
def test_half_duct_with_two_symmetry_faces(Q):
    """A quarter of the square duct (symmetry faces at x+ and y+, walls at
    x- and y-, z periodic, body force), FP64, 400 steps, against the oracle's
    full duct: the corner quarter agrees to 1e-12."""
    full = inputs.duct(Q, 12, 8, nu=0.1, u_max=0.02, storage="f64")
    quarter = inputs.duct(Q, 12, 8, nu=0.1, u_max=0.02, storage="f64")
    quarter.nx = quarter.ny = 6
    quarter.faces = (inputs.WALL, inputs.SYMMETRY, inputs.WALL, inputs.SYMMETRY,
                     inputs.PERIODIC, inputs.PERIODIC)
    g = gpu_run(quarter, 400)
    o = oracle_run(full, 400)
    assert rel_max(g["u"], o["u"][:, :, :6, :6]) <= 1e-12
    assert rel_max(g["f"], o["f"][:, :, :6, :6]) <= 1e-12


EDGE_CASES = [
    # (name, shape, faces, edge): a profiled lid over a half cavity, several
    # profiled faces with symmetry faces, a one-column axis, long rows
    ("ku_half", (9, 7, 5), (1, 1, 1, 2, 1, 3), {3: (0, 0.3, 1.0)}),
    ("multi", (6, 5, 7), (2, 1, 1, 2, 3, 2), {3: (2, 0.2, 0.6), 0: (1, 1.5, -0.5),
                                             5: (0, 0.0, 2.0)}),
    ("thin", (1, 6, 4), (1, 1, 1, 2, 1, 1), {3: (0, 0.4, 0.9)}),
    ("long_x", (67, 4, 3), (1, 1, 1, 2, 0, 0), {3: (0, 0.3, 1.0)}),
]


@pytest.mark.parametrize("steps", (1, 2, 37))
@pytest.mark.parametrize("name,shape,faces,edge", EDGE_CASES)
@pytest.mark.parametrize("Q", (14, 18, 26))
def test_fp64_edge_profiles(Q, name, shape, faces, edge, steps):
    """Moving faces with edge profiles (the lid corner velocities of Sec.
    4.3), FP64, from a seeded random state, against the oracle to 1e-12."""
    rng = np.random.default_rng(zlib.crc32(repr((name, Q)).encode()))
    uw = rng.normal(size=(6, 3)) * 0.03
    case = inputs.Case(name, Q, *shape, tuple(faces), uw, nu=0.05, force=(1e-4, -2e-4, 5e-5),
                       period=17.0, storage="f64", u_ref=0.03, edge=edge)
    case.init_u, case.init_p = inputs.random_state(case, seed=3)
    g, o = gpu_run(case, steps), oracle_run(case, steps)
    assert rel_max(g["f"], o["f"]) <= 1e-12
    assert rel_max(g["u"], o["u"]) <= 1e-12


@pytest.mark.parametrize("Q", (14, 18, 26))
def test_ku_half_cavity_fp64_and_fp32(Q):
    """The Sec. 4.3 setup: half cavity 25 x 25 x 13, lid 0.1 with the corner
    velocities, Re 400, 401 steps.  FP64 against the oracle to 1e-12; FP32
    (one and two cells per thread) within 1e-5 U of it; and the profile
    changes the flow next to the lid's first column."""
    c64 = inputs.half_cavity(Q, 25, 400.0, U=0.1, storage="f64", ku_lid=True)
    g = gpu_run(c64, 401)
    o = oracle_run(c64, 401)
    assert rel_max(g["f"], o["f"]) <= 1e-12
    assert rel_max(g["u"], o["u"]) <= 1e-12
    for launch in ((64, 1, 1), (64, 2, 2)):
        c32 = inputs.half_cavity(Q, 25, 400.0, U=0.1, storage="f32", ku_lid=True)
        g32 = gpu_run(c32, 401, launch=launch)
        assert np.max(np.abs(g32["u"] - o["u"])) <= 1e-5 * c32.u_ref
    plain = gpu_run(inputs.half_cavity(Q, 25, 400.0, U=0.1, storage="f64"), 401)
    d = np.abs(plain["u"][0, :, -1, 0] - g["u"][0, :, -1, 0])
    assert np.min(d) > 1e-3 * c64.u_ref
