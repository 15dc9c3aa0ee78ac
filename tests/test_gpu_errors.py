"""Argument checks of the single-domain C-ABI on a live handle: every
rejected call returns LBM_EINVAL (raised by the binding as LBMError), leaves
the handle usable, and the next valid call succeeds."""
import numpy as np
import pytest

from paper_1503_03337_gb300 import inputs, lbm

from lbm_cases import gpu_open

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1503_03337_gb300 import build
    build.build()
    lbm.load()


def einval(fn, *a, **kw):
    with pytest.raises(lbm.LBMError) as ei:
        fn(*a, **kw)
    assert ei.value.code == lbm.LBM_EINVAL, ei.value
    assert lbm.load().lbm_last_error().decode()  # a message was left


def test_rejected_calls_leave_handle_usable():
    case = inputs.cavity(18, 16, 100.0, storage="f32")
    h = gpu_open(case)
    try:
        W, P, M = lbm.LBM_WALL, lbm.LBM_PERIODIC, lbm.LBM_MOVING_WALL
        einval(lbm.lbm_set_geometry, h, (P, W, W, W, W, W))      # opposite faces disagree
        einval(lbm.lbm_set_geometry, h, (W, W, W, W, W, 7))      # unknown face kind
        einval(lbm.lbm_set_geometry, h, (P, P, P, W, W, W))      # x fine, y disagrees
        S, lid = lbm.LBM_SYMMETRY, (W, W, W, M, W, W)
        einval(lbm.lbm_set_geometry, h, (P, S, W, W, W, W))      # symmetry facing periodic
        uw = np.zeros((6, 3))
        einval(lbm.lbm_set_geometry, h, lid, uw, {2: (0, 0.3, 1.0)})   # profile on a wall
        einval(lbm.lbm_set_geometry, h, lid, uw, {3: (1, 0.3, 1.0)})   # along the normal
        einval(lbm.lbm_set_geometry, h, lid, uw, {3: (3, 0.3, 1.0)})   # no such axis
        einval(lbm.lbm_set_geometry, h, lid, uw, {3: (0, np.nan, 1.0)})
        uw[0, 1] = np.inf
        einval(lbm.lbm_set_geometry, h, lid, uw)                  # wall velocity not finite
        einval(lbm.lbm_set_params, h, nu=-0.1)                    # nu <= 0
        einval(lbm.lbm_set_params, h, nu=0.1, s_e=2.5)            # rate outside (0, 2)
        einval(lbm.lbm_set_params, h, nu=0.1, s_q=0.0)
        einval(lbm.lbm_set_params, h, nu=0.1, rounding=9)         # unknown rounding mode
        einval(lbm.lbm_set_launch, h, 48, 2, 1)                   # bx not a multiple of 32
        einval(lbm.lbm_set_launch, h, 128, 4, 1)                  # more than 256 threads
        einval(lbm.lbm_set_launch, h, 64, 2, 3)                   # cells per thread
        out = np.zeros(3 * case.cells)
        einval(lbm.lbm_read_fields, h, 0, out)                    # empty field mask
        einval(lbm.lbm_read_fields, h, 64, out)                   # unknown field bit
        einval(lbm.lbm_step, h, -1)
        # the rejected calls changed nothing: stepping now matches a fresh
        # handle with the same geometry and parameters
        lbm.lbm_init_equilibrium(h)
        lbm.lbm_step(h, 20)
        u = lbm.read_u(h, case.nx, case.ny, case.nz)
    finally:
        lbm.lbm_destroy(h)
    h2 = gpu_open(case)
    try:
        lbm.lbm_init_equilibrium(h2)
        lbm.lbm_step(h2, 20)
        np.testing.assert_array_equal(u, lbm.read_u(h2, case.nx, case.ny, case.nz))
    finally:
        lbm.lbm_destroy(h2)


def test_fp64_storage_rejects_two_cells_per_thread():
    case = inputs.cavity(14, 12, 100.0, storage="f64")
    h = gpu_open(case)
    try:
        einval(lbm.lbm_set_launch, h, 64, 1, 2)
        lbm.lbm_set_launch(h, 64, 1, 1)
    finally:
        lbm.lbm_destroy(h)
