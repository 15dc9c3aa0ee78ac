"""Symmetry (free-slip) faces on the GPU: the half cavity of Sec. 4.3 (Eq.
z05symmetry) against the oracle's full, mirror-symmetric cavity, and the
reduced-precision half domains against their own full boxes."""
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


@pytest.mark.parametrize("Q", (14, 18))
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
@pytest.mark.parametrize("Q", (14, 18))
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


@pytest.mark.parametrize("Q", (14, 18))
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
