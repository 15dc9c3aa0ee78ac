"""Solid nodes (lbm_set_solid, general geometry) on the GPU against the
oracle's solid mask, through the C-ABI."""
import zlib

import numpy as np
import pytest

from paper_1503_03337_gb300 import inputs, lbm

from lbm_cases import gpu_open, gpu_run, oracle_run, rel_max

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1503_03337_gb300 import build
    build.build()
    lbm.load()


def seed(*key):
    return zlib.crc32(repr(key).encode())


CASES = [
    ("periodic", (9, 7, 6), (0, 0, 0, 0, 0, 0), 0.3),
    ("walls", (13, 6, 7), (1, 2, 1, 1, 0, 0), 0.2),
    ("sym", (7, 6, 5), (3, 1, 0, 0, 2, 3), 0.25),
    ("wide_x", (131, 5, 4), (1, 1, 2, 1, 0, 0), 0.15),
    ("dense", (6, 6, 6), (0, 0, 1, 1, 3, 3), 0.6),
]


def solid_case(Q, name, shape, faces, frac, storage):
    rng = np.random.default_rng(seed(name, Q))
    uw = rng.normal(size=(6, 3)) * 0.03
    case = inputs.Case(name, Q, shape[0], shape[1], shape[2], tuple(faces), uw, nu=0.05,
                       force=(1e-4, -2e-4, 5e-5), period=17.0, storage=storage, u_ref=0.03)
    case.solid = (rng.random(shape[::-1]) < frac).astype(np.uint8)
    case.init_u, case.init_p = inputs.random_state(case, seed=4)
    return case


@pytest.mark.parametrize("launch", ((64, 1, 1), (32, 4, 1), (128, 2, 1)))
@pytest.mark.parametrize("steps", (1, 2, 37))
@pytest.mark.parametrize("name,shape,faces,frac", CASES)
@pytest.mark.parametrize("Q", (14, 18, 26))
def test_fp64_parity(Q, name, shape, faces, frac, steps, launch):
    """FP64, random solid nodes with every face kind they combine with: the
    populations (zero at solid nodes) and velocity within 1e-12 of the
    oracle, for several block shapes."""
    case = solid_case(Q, name, shape, faces, frac, "f64")
    g, o = gpu_run(case, steps, launch=launch), oracle_run(case, steps)
    assert rel_max(g["f"], o["f"]) <= 1e-12
    assert rel_max(g["u"], o["u"]) <= 1e-12
    assert np.all(g["u"][:, case.solid.astype(bool)] == 0.0)


@pytest.mark.parametrize("Q", (14, 18, 26))
def test_reduced_storage_porous_channel(Q):
    """A channel with random obstacles (periodic, body force), from rest,
    500 steps: FP32 storage within 1e-5 U of the oracle (U = max |u|); FP16
    storage (stochastic rounding) within 1e-3 U or, since the obstacles'
    corners amplify storage rounding as the cavity's lid corners do, within
    three times the FP32 error scaled by the unit-roundoff ratio 2^13."""
    rng = np.random.default_rng(11)
    shape = (48, 20, 16)
    faces = (0, 0, 1, 1, 0, 0)
    ref = inputs.Case("porous", Q, *shape, faces, np.zeros((6, 3)), nu=0.05,
                      force=(2e-5, 0.0, 0.0), storage="f64")
    ref.solid = (rng.random(shape[::-1]) < 0.2).astype(np.uint8)
    o = oracle_run(ref, 500)
    U = float(np.max(np.abs(o["u"])))
    err = {}
    for storage in ("f32", "f16"):
        case = inputs.Case("porous", Q, *shape, faces, np.zeros((6, 3)), nu=0.05,
                           force=(2e-5, 0.0, 0.0), storage=storage)
        case.solid = ref.solid
        if storage == "f16":
            case.rounding = lbm.LBM_ROUND_STOCHASTIC
        g = gpu_run(case, 500)
        err[storage] = float(np.max(np.abs(g["u"] - o["u"])))
        print("Q%d %s: max|u - u_oracle| / U = %.3e" % (Q, storage, err[storage] / U))
    assert err["f32"] <= 1e-5 * U
    assert err["f16"] <= max(1e-3 * U, 3.0 * 2.0 ** 13 * err["f32"])


@pytest.mark.parametrize("Q", (14, 18, 26))
def test_reductions_checkpoint_and_clear(Q):
    """Reductions sum the fluid nodes only (against the oracle's fields);
    a checkpoint written back at an odd step restores the run bit for bit;
    lbm_set_solid(NULL) returns to the plain box."""
    case = solid_case(Q, "walls", (13, 6, 7), (1, 2, 1, 1, 0, 0), 0.2, "f64")
    h = gpu_open(case)
    try:
        lbm.lbm_init_equilibrium(h, np.ascontiguousarray(case.init_u),
                                 np.ascontiguousarray(case.init_p), 0)
        lbm.lbm_step(h, 30)
        lbm.lbm_reductions(h)
        lbm.lbm_step(h, 7)
        st = lbm.lbm_reductions(h)
        o30, o37 = oracle_run(case, 30)["u"], oracle_run(case, 37)["u"]
        for k in range(3):
            assert abs(st.sum_abs_u[k] - np.abs(o37[k]).sum()) <= 1e-11 * np.abs(o37[k]).sum()
            assert abs(st.sum_abs_du[k] - np.abs(o37[k] - o30[k]).sum()) <= \
                1e-11 * np.abs(o37[k]).sum()
        ck = lbm.read_populations(h, Q, case.nx, case.ny, case.nz)  # step 37, odd
        lbm.lbm_step(h, 20)
        fa = lbm.read_populations(h, Q, case.nx, case.ny, case.nz)
        lbm.lbm_set_step(h, 37)
        lbm.lbm_write_populations(h, np.ascontiguousarray(ck), 0)
        lbm.lbm_step(h, 20)
        np.testing.assert_array_equal(lbm.read_populations(h, Q, case.nx, case.ny, case.nz), fa)
        lbm.lbm_set_solid(h, None)
        lbm.lbm_init_equilibrium(h, np.ascontiguousarray(case.init_u),
                                 np.ascontiguousarray(case.init_p), 0)
        lbm.lbm_step(h, 5)
        u = lbm.read_u(h, case.nx, case.ny, case.nz)
    finally:
        lbm.lbm_destroy(h)
    box = solid_case(Q, "walls", (13, 6, 7), (1, 2, 1, 1, 0, 0), 0.2, "f64")
    box.solid = None
    assert rel_max(u, oracle_run(box, 5)["u"]) <= 1e-12


def test_solid_argument_checks():
    case = solid_case(18, "walls", (13, 6, 7), (1, 2, 1, 1, 0, 0), 0.2, "f32")
    h = gpu_open(case)
    try:
        with pytest.raises(lbm.LBMError) as ei:  # extrapolation faces do not combine
            lbm.lbm_set_geometry(h, (4, 4, 1, 1, 0, 0), case.u_wall)
        assert ei.value.code == lbm.LBM_EINVAL
    finally:
        lbm.lbm_destroy(h)
