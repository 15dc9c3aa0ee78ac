"""The lid-driven cavity at Re = 3200, the case Sec. 4.3 uses to show the
iD3Q14 MRT model's stability (49 x 49 x 25 half cavity, stable to
25000 steps).  Here the full 49^3 cube (the half cavity is its mirror
half), lid 0.1 along x, nu = U L / Re (tau = 0.5046), 25000 steps of the
fused FP32 step: every velocity stays finite and bounded by the lid speed
scale, for both models."""
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


@pytest.mark.parametrize("Q", (14, 18))
def test_cavity_re3200_stays_finite(Q):
    U, n, Re, steps = 0.1, 49, 3200.0, 25000
    case = inputs.cavity(Q, n, Re, U=U, storage="f32")
    assert abs((3 * case.nu + 0.5) - 0.5046) < 1e-4
    h = gpu_open(case, residual_interval=5000)
    try:
        lbm.lbm_init_equilibrium(h)
        lbm.lbm_step(h, steps)  # raises LBMError(LBM_EUNSTABLE) if a check saw a NaN/Inf
        stats = lbm.lbm_reductions(h)
        u = lbm.read_u(h, n, n, n)
    finally:
        lbm.lbm_destroy(h)
    assert stats.nonfinite == 0
    assert np.all(np.isfinite(u))
    assert np.max(np.abs(u)) < 1.5 * U
    # the lid drives a primary vortex: return flow along -x below the lid
    assert u[0, n // 2, n // 4, n // 2] < 0.0
