"""Test helpers: run a Case through the CUDA library (C-ABI) and through the
oracle with identical seeded inputs."""
import numpy as np

import oracle
from paper_1503_03337_gb300 import lbm


def oracle_setup(case):
    g = oracle.make_grid(case.Q, case.nx, case.ny, case.nz, case.faces, case.u_wall,
                         edge=case.edge, solid=case.solid)
    r = oracle.rates(case.Q, oracle.s_nu_of(case.nu))
    prm = oracle.make_params(r, force=case.force, period=case.period, p_face=case.p_face,
                             p_amp=case.p_amp, p_period=case.p_period)
    return g, prm


def oracle_run(case, steps, f0=None, n0=0):
    g, prm = oracle_setup(case)
    if f0 is None:
        f0 = oracle.init_equilibrium(g, case.init_u, case.init_p)
    f = oracle.run(g, prm, f0, n0, steps)
    u, p = oracle.macroscopic(g, prm, n0 + steps, f)
    return {"f": f, "u": u, "p": p}


def gpu_open(case, stream=None, residual_interval=0, launch=None):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    h = lbm.lbm_create(case.Q, case.nx, case.ny, case.nz, case.storage, stream)
    lbm.lbm_set_geometry(h, case.faces, case.u_wall, case.edge)
    lbm.lbm_set_params(h, nu=case.nu, force=case.force, force_period=case.period,
                       residual_interval=residual_interval, rounding=case.rounding,
                       p_face=case.p_face, p_amp=case.p_amp, p_period=case.p_period,
                       p_ref=case.p_ref)
    if case.solid is not None:
        lbm.lbm_set_solid(h, case.solid)
    if launch is not None:
        lbm.lbm_set_launch(h, *launch)
    return h


def gpu_run(case, steps, keep=False, launch=None):
    h = gpu_open(case, launch=launch)
    try:
        u0 = None if case.init_u is None else np.ascontiguousarray(case.init_u, dtype=np.float64)
        p0 = None if case.init_p is None else np.ascontiguousarray(case.init_p, dtype=np.float64)
        lbm.lbm_init_equilibrium(h, u0, p0, 0)
        lbm.lbm_step(h, steps)
        out = {"u": lbm.read_u(h, case.nx, case.ny, case.nz),
               "p": lbm.read_p(h, case.nx, case.ny, case.nz),
               "f": lbm.read_populations(h, case.Q, case.nx, case.ny, case.nz)}
    finally:
        if not keep:
            lbm.lbm_destroy(h)
    if keep:
        out["h"] = h
    return out


def rel_max(a, b):
    """max |a - b| / max |b|"""
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))
