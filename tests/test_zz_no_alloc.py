"""lbm_reductions_static: the FP64 reductions for callers that cannot call
cudaMalloc.

Such callers include code whose device memory belongs to another allocator
with a fixed budget, and latency-critical loops that must not pay for
cudaMalloc/cudaFree (cudaFree synchronises the whole device).  They pass
buffers they already own; the entry point's only scratch is a static device
array inside the library.  This test checks, on two calls in a row, that it
reports the same statistics as the allocating lbm_reductions for the same
state.  It lives in its own file, collected last, so that a run stopping at
the first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_1503_03337_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu

# the tolerance of the other reduction tests: sums of many terms taken in a
# different order agree to 1e-11 relative
TOL = 1e-11


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1503_03337_gb300 import build
    build.build()
    lbm.load()
    return torch


def close(a, b):
    return abs(a - b) <= TOL * max(abs(a), abs(b)) + 1e-300


def same_stats(s, r, with_du, cells=0):
    for k in range(3):
        assert close(s.sum_abs_u[k], r.sum_abs_u[k])
        # a signed sum that nearly cancels (the net flow of a closed cavity)
        # is accurate relative to the sum of its terms' magnitudes
        assert abs(s.sum_u[k] - r.sum_u[k]) <= TOL * max(s.sum_abs_u[k], r.sum_abs_u[k]) + 1e-300
        if with_du:
            assert close(s.sum_abs_du[k], r.sum_abs_du[k])
            assert close(s.sum_abs_u_prev[k], r.sum_abs_u_prev[k])
    # sum P nearly cancels when the pressure is near its reference: besides
    # the relative bound, allow 1e-16 per cell (the rounding of terms of
    # order 1e-2 summed in a different order)
    assert abs(s.sum_P - r.sum_P) <= TOL * max(abs(s.sum_P), abs(r.sum_P)) + 1e-16 * cells
    assert close(s.max_abs_u, r.max_abs_u)
    assert s.nonfinite == r.nonfinite == 0


def test_static_reductions_match_allocating_path(torch):
    case = inputs.duct(18, 20, 12, nu=0.08, storage="f32")
    Q, N = case.Q, case.cells
    stream = torch.cuda.current_stream()
    h = lbm.lbm_create(Q, case.nx, case.ny, case.nz, "f32", stream.cuda_stream)
    try:
        lbm.lbm_set_geometry(h, case.faces, case.u_wall)
        lbm.lbm_set_params(h, nu=case.nu, force=case.force)
        prm = lbm.make_params(nu=case.nu, force=case.force)
        lbm.lbm_init_equilibrium(h)
        u_prev = torch.empty(3 * N, dtype=torch.float64, device="cuda")
        f64 = torch.empty(Q * N, dtype=torch.float64, device="cuda")
        prev = -1
        for n in (40, 48):  # even steps: the storage layout is canonical
            lbm.lbm_step(h, n - lbm.lbm_get_step(h))
            ref = lbm.lbm_reductions(h)
            lbm.lbm_read_fields(h, lbm.LBM_FIELD_POPULATIONS, f64, lbm.LBM_DTYPE_F64, 1)
            pops = f64.to(torch.float32)  # FP32 storage values, exactly
            got = lbm.lbm_reductions_static(Q, case.nx, case.ny, case.nz, "f32", case.faces,
                                            case.u_wall, prm, n, pops, u_prev, prev,
                                            stream.cuda_stream)
            assert got.step == n and got.prev_step == prev == ref.prev_step
            same_stats(got, ref, with_du=prev >= 0)
            # the snapshot now holds u at step n
            u = torch.empty(3 * N, dtype=torch.float64, device="cuda")
            lbm.lbm_read_fields(h, lbm.LBM_FIELD_U, u, lbm.LBM_DTYPE_F64, 1)
            np.testing.assert_allclose(u_prev.cpu().numpy(), u.cpu().numpy(), rtol=1e-14, atol=1e-18)
            prev = n
    finally:
        lbm.lbm_destroy(h)


WIDE_CASES = {
    # body force along z, walls on x and y, periodic z
    "duct": lambda st: inputs.duct(14, 18, 10, nu=0.08, storage=st),
    # symmetry face on z+, moving lid on y+ with the corner edge profile
    "half_cavity": lambda st: inputs.half_cavity(18, 17, 200.0, U=0.05, storage=st,
                                                 ku_lid=True),
    # the iD3Q26 model on the lid-driven cube
    "cavity_q26": lambda st: inputs.cavity(26, 13, 100.0, storage=st),
}


@pytest.mark.parametrize("name", sorted(WIDE_CASES))
@pytest.mark.parametrize("storage", ("f64", "f32", "f16", "bf16"))
def test_static_reductions_every_layout(torch, name, storage):
    """Every storage type, an even and then an odd step (the in-place
    streaming's two layouts), a forced duct and a half cavity (symmetry face,
    moving lid with an edge profile): lbm_reductions_static on the handle's
    own population buffer gives the statistics of lbm_reductions, on two
    calls in a row."""
    case = WIDE_CASES[name](storage)
    Q, N = case.Q, case.cells
    stream = torch.cuda.current_stream()
    h = lbm.lbm_create(Q, case.nx, case.ny, case.nz, storage, stream.cuda_stream)
    try:
        lbm.lbm_set_geometry(h, case.faces, case.u_wall, case.edge)
        lbm.lbm_set_params(h, nu=case.nu, force=case.force)
        prm = lbm.make_params(nu=case.nu, force=case.force)
        lbm.lbm_init_equilibrium(h)
        pops, nbytes = lbm.lbm_device_populations(h)
        assert nbytes == Q * N * {"f64": 8, "f32": 4, "f16": 2, "bf16": 2}[storage]
        u_prev = torch.empty(3 * N, dtype=torch.float64, device="cuda")
        prev = -1
        for n in (40, 47):
            lbm.lbm_step(h, n - lbm.lbm_get_step(h))
            got = lbm.lbm_reductions_static(Q, case.nx, case.ny, case.nz, storage, case.faces,
                                            case.u_wall, prm, n, pops, u_prev, prev,
                                            stream.cuda_stream, edge=case.edge)
            ref = lbm.lbm_reductions(h)
            assert got.step == n and got.prev_step == prev == ref.prev_step
            same_stats(got, ref, with_du=prev >= 0, cells=N)
            u = torch.empty(3 * N, dtype=torch.float64, device="cuda")
            lbm.lbm_read_fields(h, lbm.LBM_FIELD_U, u, lbm.LBM_DTYPE_F64, 1)
            np.testing.assert_allclose(u_prev.cpu().numpy(), u.cpu().numpy(), rtol=1e-12,
                                       atol=1e-16)
            prev = n
    finally:
        lbm.lbm_destroy(h)


def test_static_reductions_reject_oversized_domain(torch):
    prm = lbm.make_params(nu=0.1)
    dummy = torch.empty(16, dtype=torch.float32, device="cuda")
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_reductions_static(18, 129, 128, 128, "f32", [lbm.LBM_WALL] * 6, None, prm, 0,
                                  dummy)
    assert ei.value.code == lbm.LBM_EINVAL
    assert "at most 2097152 cells" in str(ei.value)
