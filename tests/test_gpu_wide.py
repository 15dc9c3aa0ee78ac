"""Domains with Q*N >= 2^31: the step's 64-bit-offset (wide) kernels.

A box periodic in x and y and started from a field of period 8 in x and y
keeps that period, so every cell of a 512 x 512 x nz box must equal the
cell (x mod 8, y mod 8, z) of the 8 x 8 x nz box stepped the same way with
the 32-bit kernels.  One cell per thread does the same arithmetic in both
(the launch shape never changes results), so the comparison is bit for bit,
at an even and at an odd step count, with walls and a moving lid on z.
The FP64 reductions of the large box are 4096 times those of the small one.
"""
import numpy as np
import pytest

from paper_1503_03337_gb300 import lbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1503_03337_gb300 import build
    build.build()
    lbm.load()
    return torch


FACES = (lbm.LBM_PERIODIC, lbm.LBM_PERIODIC, lbm.LBM_PERIODIC, lbm.LBM_PERIODIC,
         lbm.LBM_WALL, lbm.LBM_MOVING_WALL)


def open_box(torch, Q, n, nz, storage, u, p):
    uw = np.zeros((6, 3))
    uw[5] = (0.05, 0.01, 0.0)
    h = lbm.lbm_create(Q, n, n, nz, storage, torch.cuda.current_stream().cuda_stream)
    lbm.lbm_set_geometry(h, FACES, uw)
    lbm.lbm_set_params(h, nu=0.02, force=(1e-5, -2e-5, 0.0))
    lbm.lbm_init_equilibrium(h, u, p, 1)
    return h


def read_u(torch, h, N):
    u = torch.empty(3 * N, dtype=torch.float64, device="cuda")
    lbm.lbm_read_fields(h, lbm.LBM_FIELD_U, u, lbm.LBM_DTYPE_F64, 1)
    return u


@pytest.mark.parametrize("Q,storage,nz", ((18, "f16", 456), (14, "f32", 600)))
def test_wide_box_equals_tiled_small_box(torch, Q, storage, nz):
    n, m = 512, 8
    N, Ns = n * n * nz, m * m * nz
    assert Q * N >= 2 ** 31 > Q * Ns
    g = torch.Generator(device="cuda").manual_seed(Q)
    us = (torch.rand((3, nz, m, m), generator=g, device="cuda", dtype=torch.float64) - 0.5) * 0.04
    ps = (torch.rand((nz, m, m), generator=g, device="cuda", dtype=torch.float64) - 0.5) * 0.02
    small = open_box(torch, Q, m, nz, storage, us.contiguous(), ps.contiguous())
    big = open_box(torch, Q, n, nz, storage, us.repeat(1, 1, n // m, n // m).contiguous(),
                   ps.repeat(1, n // m, n // m).contiguous())
    try:
        for steps in (3, 1):  # an odd, then an even step count
            lbm.lbm_step(small, steps)
            lbm.lbm_step(big, steps)
            ub = read_u(torch, big, N).view(3, nz, n, n)
            ut = read_u(torch, small, Ns).view(3, nz, m, m).repeat(1, 1, n // m, n // m)
            assert torch.equal(ub, ut), (steps, float((ub - ut).abs().max()))
            del ub, ut
        sb, ss = lbm.lbm_reductions(big), lbm.lbm_reductions(small)
        for k in range(3):
            assert sb.sum_abs_u[k] == pytest.approx(4096 * ss.sum_abs_u[k], rel=1e-10)
        assert sb.max_abs_u == ss.max_abs_u
        assert sb.nonfinite == 0
    finally:
        lbm.lbm_destroy(big)
        lbm.lbm_destroy(small)


def test_cell_limit(torch):
    """nx*ny*nz >= 2^31 is rejected before any allocation."""
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_create(18, 2048, 1024, 1024, "f16", None)
    assert ei.value.code == lbm.LBM_EINVAL
