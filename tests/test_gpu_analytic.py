"""CUDA path against the analytic solutions of Sec. 4 (body-force drive):
the steady square duct (Sec. 4.1) in FP64 and the pulsatile duct (Sec. 4.2)
in FP32, FP16 and BF16 storage.  These are accuracy checks of the whole
scheme (a tolerance, not parity): GRE_u of the order of Tables 1 and 2 at
comparable resolution.  The FP64 run is also compared with the oracle's
GRE_u, which the two computations must share to round-off."""
import numpy as np
import pytest

from oracle import analytic as an
from paper_1503_03337_gb300 import inputs, lbm

from lbm_cases import gpu_open, gpu_run, oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1503_03337_gb300 import build
    build.build()
    lbm.load()


def duct_exact(case):
    a = case.nx / 2.0
    xs = an.lattice_coords(case.nx)
    Y, X = np.meshgrid(xs, xs, indexing="ij")
    ua = np.zeros((3, case.nz, case.ny, case.nx))
    ua[2] = an.duct_velocity(X, Y, a, a, case.nu, case.force[2])[None]
    return ua


@pytest.mark.parametrize("Q", (14, 18))
def test_c1_duct_fp64_gre(Q):
    """16x16x32 duct, nu = 0.1, u_max = 0.02, FP64, 3000 steps from rest:
    GRE_u against the series within Table 1's range at dx = 1/16
    (7.4e-3 to 3.3e-2 under the paper's own boundary scheme), and equal to
    the oracle's GRE_u after the same steps."""
    case = inputs.duct(Q, 16, 32, nu=0.1, u_max=0.02, storage="f64")
    h = gpu_open(case)
    try:
        lbm.lbm_init_equilibrium(h)
        lbm.lbm_step(h, 3000)
        u = lbm.read_u(h, case.nx, case.ny, case.nz)
    finally:
        lbm.lbm_destroy(h)
    ua = duct_exact(case)
    gre = an.gre_u(u, ua)
    assert gre < 3e-2, gre
    gre_o = an.gre_u(oracle_run(case, 3000)["u"], ua)
    assert abs(gre - gre_o) <= 1e-9 * gre_o, (gre, gre_o)


PULSATILE_GRE = {"f32": 3e-2, "f16": 3e-2, "bf16": 3e-2}
# max |u - u_FP32| / U over the four checks.  FP16 (11-bit significand)
# meets the 1e-3 U target; BF16 (8-bit significand) rounds each stored
# population 8x more coarsely and is bounded at its measured level (3.7e-3)
# with margin.
PULSATILE_DEV = {"f16": 1e-3, "bf16": 5e-3}


@pytest.mark.parametrize("storage", ("f32", "f16", "bf16"))
def test_c3_pulsatile_gre(storage):
    """64x64x8 pulsatile duct, T = 1000, eta = 4 (Womersley number of
    Table 2's middle rows), amplitude giving max|u| = 0.03.  Warm start from
    the analytic field at t = 0, two periods of warm-up, then GRE_u at the
    four quarter periods of the third.  Reduced-precision storage rounds
    stochastically; its field also stays close to the FP32 field
    (PULSATILE_DEV)."""
    N, nz, T, eta, A = 64, 8, 1000, 4.0, 1.555e-4
    case = inputs.pulsatile(18, N, nz, T, eta, A, storage=storage)
    if storage != "f32":
        case.rounding = lbm.LBM_ROUND_STOCHASTIC
    b = N / 2.0
    omega = 2 * np.pi / T
    xs = an.lattice_coords(N)
    Y, X = np.meshgrid(xs, xs, indexing="ij")
    Uc = an.pulsatile_amplitude(X, Y, b, b, case.nu, omega, -A)  # G = -A (F = -dp/dx)
    U = float(np.max(np.abs(Uc)))
    assert abs(U - 0.03) < 1e-4
    u0 = np.zeros((3, nz, N, N))
    u0[2] = np.real(Uc)[None]
    fields = {}
    for st in sorted({"f32", storage}):
        c = inputs.pulsatile(18, N, nz, T, eta, A, storage=st)
        c.rounding = case.rounding if st == storage else lbm.LBM_ROUND_NEAREST
        h = gpu_open(c, launch=(64, 1, 2) if st != "f32" else None)
        try:
            lbm.lbm_init_equilibrium(h, u0, None, 0)
            lbm.lbm_step(h, 2 * T)
            errs, us = [], []
            for q in range(4):
                n = lbm.lbm_get_step(h)
                u = lbm.read_u(h, N, N, nz)
                ua = np.zeros_like(u)
                ua[2] = np.real(Uc * np.exp(1j * omega * n))[None]
                errs.append(an.gre_u(u, ua))
                us.append(u)
                lbm.lbm_step(h, T // 4)
        finally:
            lbm.lbm_destroy(h)
        fields[st] = (errs, us)
    errs, us = fields[storage]
    print("pulsatile GRE_u (%s):" % storage, ["%.3e" % e for e in errs])
    assert max(errs) < PULSATILE_GRE[storage], errs
    if storage != "f32":
        dev = max(float(np.max(np.abs(a - b))) for a, b in zip(us, fields["f32"][1]))
        print("max |u_%s - u_f32| / U = %.3e" % (storage, dev / U))
        assert dev <= PULSATILE_DEV[storage] * U, dev / U


# The ends of the pulsatile grid of the 64 x 64 x 8 channel: the longest
# period with the largest Womersley number (thin Stokes layers, tau = 0.521,
# per-step changes of a few FP16 ulps) and the shortest period with the
# smallest (tau = 10.15, the largest wall slip of halfway bounce-back).
HARD_END = [(4000, 15.0), (500, 2.0)]


def pulsatile_setup(Q, T, eta, storage, N=64, nz=8, U=0.03):
    b = N / 2.0
    omega = 2 * np.pi / T
    nu = b * b * omega / eta ** 2
    xs = an.lattice_coords(N)
    Y, X = np.meshgrid(xs, xs, indexing="ij")
    unit = an.pulsatile_amplitude(X, Y, b, b, nu, omega, 1.0)
    A = U / float(np.max(np.abs(unit)))  # max over (t, y, z) of |u| = U
    case = inputs.pulsatile(Q, N, nz, T, eta, A, storage=storage, u_ref=U)
    Uc = -A * unit  # G = -A (F = -dp/dx)
    u0 = np.zeros((3, nz, N, N))
    u0[2] = np.real(Uc)[None]
    case.init_u = u0
    return case, Uc, omega


@pytest.mark.parametrize("T,eta", HARD_END)
@pytest.mark.parametrize("Q", (14, 18))
def test_pulsatile_hard_end_parity(Q, T, eta):
    """One period from the analytic field at t = 0: FP32 storage within
    1e-5 U and FP16 storage (stochastic rounding, two cells per thread on
    even steps, the benchmarked launch) within 1e-3 U of the oracle, max
    over all nodes and components."""
    case, _, _ = pulsatile_setup(Q, T, eta, "f64")
    o = oracle_run(case, T)
    for storage, launch, bound in (("f32", None, 1e-5), ("f16", (64, 1, 2), 1e-3)):
        c, _, _ = pulsatile_setup(Q, T, eta, storage)
        if storage == "f16":
            c.rounding = lbm.LBM_ROUND_STOCHASTIC
        g = gpu_run(c, T, launch=launch)
        err = float(np.max(np.abs(g["u"] - o["u"])))
        print("Q%d T=%d eta=%g %s: max|u - u_oracle| / U = %.3e" % (Q, T, eta, storage, err / 0.03))
        assert err <= bound * 0.03, (storage, err / 0.03)


@pytest.mark.parametrize("T,eta", HARD_END)
def test_pulsatile_hard_end_gre(T, eta):
    """Five periods from the analytic field (D3Q18): GRE_u (Eq. ed) against
    Eq. wa at the quarter periods of the fifth, FP32 and FP16 (stochastic
    rounding, pair launch).  The two storages give the same GRE_u to 1e-3
    of its value plus 1e-4."""
    out = {}
    for storage, launch in (("f32", None), ("f16", (64, 1, 2))):
        c, Uc, omega = pulsatile_setup(18, T, eta, storage)
        if storage == "f16":
            c.rounding = lbm.LBM_ROUND_STOCHASTIC
        h = gpu_open(c, launch=launch)
        try:
            lbm.lbm_init_equilibrium(h, np.ascontiguousarray(c.init_u), None, 0)
            lbm.lbm_step(h, 4 * T)
            errs = []
            for q in range(4):
                n = lbm.lbm_get_step(h)
                u = lbm.read_u(h, c.nx, c.ny, c.nz)
                ua = np.zeros_like(u)
                ua[2] = np.real(Uc * np.exp(1j * omega * n))[None]
                errs.append(an.gre_u(u, ua))
                lbm.lbm_step(h, T // 4)
        finally:
            lbm.lbm_destroy(h)
        out[storage] = errs
        print("T=%d eta=%g %s GRE_u at kT/4 of period 5:" % (T, eta, storage),
              ["%.3e" % e for e in errs])
    for a, b in zip(out["f16"], out["f32"]):
        assert abs(a - b) <= 1e-3 * b + 1e-4, (a, b)
    assert max(out["f32"]) < 0.5
