"""Batched stepping (lbm_batch_*): every domain of a batch computes exactly
what a single-domain handle computes, alone or in any mix, in both launch
modes and under every work split (grouped, solo, tiles per CTA); the
persistent grid barrier's time-out path reports LBM_ETIMEOUT."""
import numpy as np
import pytest

from paper_1503_03337_gb300 import inputs, lbm

from lbm_cases import gpu_open, oracle_run

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


def mix():
    cases = [
        inputs.cavity(18, 40, 400.0, storage="f32"),
        inputs.duct(14, 24, 20, nu=0.05, storage="f16"),
        inputs.cavity(14, 33, 300.0, storage="bf16", ny=17, nz=9),
        inputs.duct(18, 70, 7, nu=0.08, storage="f32"),
        inputs.cavity(18, 20, 100.0, storage="f16"),
    ]
    cases[1].ny = 9  # a non-square duct cross-section
    # a half cavity (symmetry face on the mid-plane z+) with the lid's
    # corner velocities
    cases[2].faces = cases[2].faces[:5] + (inputs.SYMMETRY,)
    cases[2].edge = {inputs.YP: (0,) + inputs.KU_LID_EDGE}
    cases[4].rounding = lbm.LBM_ROUND_STOCHASTIC
    return cases


def add(b, c):
    return lbm.lbm_batch_add(b, c.Q, c.nx, c.ny, c.nz, c.storage, c.faces, c.u_wall,
                             edge=c.edge, nu=c.nu, force=c.force, force_period=c.period, rounding=c.rounding)


def batch_pops(torch, b, slot, c):
    out = torch.empty(c.Q * c.cells, dtype=torch.float64, device="cuda")
    lbm.lbm_batch_read_fields(b, slot, lbm.LBM_FIELD_POPULATIONS, out)
    return out.cpu().numpy().reshape(c.Q, c.nz, c.ny, c.nx)


def single_pops(c, steps):
    h = gpu_open(c, launch=(32, 2, 1))
    try:
        lbm.lbm_init_equilibrium(h)
        lbm.lbm_step(h, steps)
        return lbm.read_populations(h, c.Q, c.nx, c.ny, c.nz)
    finally:
        lbm.lbm_destroy(h)


# (persistent, tiles_per_cta, solo_min_cells, cluster_bytes): the default
# schedule, every domain solo, every domain grouped one tile per CTA in one
# cluster, long runs, and clusters so small that every domain is its own
SCHEDULES = [(1, 0, 0, 0), (0, 0, 0, 0), (0, 3, 1, 0), (0, 1, -1, -1), (0, 7, 2000, 0),
             (0, 0, 0, 1 << 16), (0, 2, -1, 3 << 20)]


@pytest.mark.parametrize("persistent,per,solo,cluster", SCHEDULES)
def test_batch_same_alone_and_in_mix(torch, persistent, per, solo, cluster):
    stream = torch.cuda.current_stream().cuda_stream
    cases = mix()
    b = lbm.lbm_batch_create(8, 0, stream)
    try:
        lbm.lbm_batch_set_launch(b, 64, 2, persistent)
        lbm.lbm_batch_set_schedule(b, per, solo, cluster)
        slots = {}
        steps = {}
        for k in range(4):
            slots[k] = add(b, cases[k])
            lbm.lbm_batch_init_equilibrium(b, slots[k])
            steps[k] = 0
        lbm.lbm_batch_step(b, 10, 4)
        for k in slots:
            steps[k] += 10
        slots[4] = add(b, cases[4])  # admitted later, at its own step 0
        lbm.lbm_batch_init_equilibrium(b, slots[4])
        steps[4] = 0
        lbm.lbm_batch_step(b, 13, 5)
        for k in slots:
            steps[k] += 13
        lbm.lbm_batch_remove(b, slots.pop(1))
        steps.pop(1)
        lbm.lbm_batch_step(b, 7, 7)
        for k in slots:
            steps[k] += 7
        assert lbm.lbm_batch_info(b)[0] == 4
        for k, slot in slots.items():
            assert lbm.lbm_batch_get_step(b, slot) == steps[k]
            got = batch_pops(torch, b, slot, cases[k])
            ref = single_pops(cases[k], steps[k])
            np.testing.assert_array_equal(got, ref, err_msg="domain %d" % k)
    finally:
        lbm.lbm_batch_destroy(b)


@pytest.mark.parametrize("solo", (-1, 1))
def test_batch_pulsatile_matches_oracle(torch, solo):
    """Oscillating force evaluated on the device at each domain's own time
    level, against the oracle, grouped and solo."""
    stream = torch.cuda.current_stream().cuda_stream
    c = inputs.pulsatile(18, 16, 4, 40, 3.0, 2e-4, storage="f32")
    b = lbm.lbm_batch_create(2, 0, stream)
    try:
        lbm.lbm_batch_set_schedule(b, 0, solo)
        s = add(b, c)
        lbm.lbm_batch_init_equilibrium(b, s)
        lbm.lbm_batch_step(b, 61, 8)
        u = torch.empty(3 * c.cells, dtype=torch.float64, device="cuda")
        lbm.lbm_batch_read_fields(b, s, lbm.LBM_FIELD_U, u)
    finally:
        lbm.lbm_batch_destroy(b)
    o = oracle_run(c, 61)
    err = np.max(np.abs(u.cpu().numpy().reshape(o["u"].shape) - o["u"]))
    assert err <= 1e-5 * np.max(np.abs(o["u"]))


def test_batch_schedule_rejects_bad_values(torch):
    stream = torch.cuda.current_stream().cuda_stream
    b = lbm.lbm_batch_create(2, 0, stream)
    try:
        with pytest.raises(lbm.LBMError) as ei:
            lbm.lbm_batch_set_schedule(b, -1, 0)
        assert ei.value.code == lbm.LBM_EINVAL
        with pytest.raises(lbm.LBMError):
            lbm.lbm_batch_set_schedule(b, 5000, 0)
    finally:
        lbm.lbm_batch_destroy(b)


def test_batch_budget_and_slots(torch):
    stream = torch.cuda.current_stream().cuda_stream
    c = inputs.cavity(18, 16, 100.0, storage="f32")
    one = c.Q * c.cells * 4
    b = lbm.lbm_batch_create(2, int(2.5 * one), stream)
    try:
        s0 = add(b, c)
        s1 = add(b, c)
        with pytest.raises(lbm.LBMError) as ei:
            add(b, c)
        assert ei.value.code == lbm.LBM_EBUSY
        lbm.lbm_batch_remove(b, s0)
        assert add(b, c) == s0  # slot reused
        assert lbm.lbm_batch_info(b)[1] == 2 * one
        assert s1 != s0
    finally:
        lbm.lbm_batch_destroy(b)


def test_batch_barrier_timeout_reported(torch):
    """The persistent barrier waits for one CTA that never arrives; its
    bounded wait gives up, the kernel returns, and the host sees
    LBM_ETIMEOUT.  The device stays usable."""
    stream = torch.cuda.current_stream().cuda_stream
    c = inputs.cavity(18, 24, 100.0, storage="f32")
    b = lbm.lbm_batch_create(2, 0, stream)
    try:
        lbm.lbm_batch_set_launch(b, 64, 2, 1)
        s = add(b, c)
        lbm.lbm_batch_init_equilibrium(b, s)
        lbm.lbm_batch_set_barrier_test(b, 1, 20000)
        lbm.lbm_batch_step(b, 4, 4)
        torch.cuda.synchronize()
        with pytest.raises(lbm.LBMError) as ei:
            lbm.lbm_batch_step(b, 1, 1)
        assert ei.value.code == lbm.LBM_ETIMEOUT
    finally:
        lbm.lbm_batch_destroy(b)
    # the context still runs work correctly
    h = gpu_open(c)
    try:
        lbm.lbm_init_equilibrium(h)
        lbm.lbm_step(h, 3)
        assert np.all(np.isfinite(lbm.read_u(h, c.nx, c.ny, c.nz)))
    finally:
        lbm.lbm_destroy(h)
