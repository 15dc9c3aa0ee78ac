"""Host-side checks of the face geometry (no GPU): lbm_geom validation,
shared by handles, batches and the static reductions, answered by
lbm_reductions_static before any CUDA call; and the half-cavity recipe."""
import ctypes

import numpy as np
import pytest

from paper_1503_03337_gb300 import build, inputs, lbm

W, P, M, S = lbm.LBM_WALL, lbm.LBM_PERIODIC, lbm.LBM_MOVING_WALL, lbm.LBM_SYMMETRY


@pytest.fixture(scope="module")
def library():
    build.build()
    return lbm.load()


def static_call(library, faces, u_wall=None, edge=None):
    d = lbm.lbm_desc(18, 16, 8, 8, lbm.LBM_STORAGE_F32)
    g = lbm.make_geom(faces, u_wall, edge)
    prm = lbm.make_params(nu=0.1)
    out = lbm.lbm_stats()
    rc = library.lbm_reductions_static(ctypes.byref(d), ctypes.byref(g), ctypes.byref(prm), 0,
                                       ctypes.c_void_p(256), None, -1, ctypes.byref(out), None)
    return rc, library.lbm_last_error().decode()


@pytest.mark.parametrize("faces,u_wall,edge,msg", [
    ((W, W, W, W, W, 7), None, None, "unknown face kind"),
    ((P, S, W, W, W, W), None, None, "periodic"),
    ((W, W, P, W, W, W), None, None, "periodic"),
    ((W, W, W, M, W, W), None, {2: (0, 0.3, 1.0)}, "moving face"),
    ((W, W, W, M, W, W), None, {3: (1, 0.3, 1.0)}, "in-plane"),
    ((W, W, W, M, W, W), None, {3: (3, 0.3, 1.0)}, "edge_axis"),
    ((W, W, W, M, W, W), None, {3: (0, float("nan"), 1.0)}, "edge scale"),
    ((W, W, W, M, W, W), np.full((6, 3), np.inf), None, "wall velocity"),
])
def test_geometry_rejected_before_cuda(library, faces, u_wall, edge, msg):
    rc, err = static_call(library, faces, u_wall, edge)
    assert rc == lbm.LBM_EINVAL and msg in err, err


def test_half_cavity_recipe():
    """Sec. 4.3's reduced domain: n x n x ceil(n/2), symmetry face at z+,
    lid on y+ along x; the corner setting scales the lid over the first and
    last x columns by 0.3 and 1.0."""
    c = inputs.half_cavity(18, 97, 3200.0, U=0.1, ku_lid=True)
    assert (c.nx, c.ny, c.nz) == (97, 97, 49)
    assert c.faces[inputs.ZP] == inputs.SYMMETRY and c.faces[inputs.ZM] == inputs.WALL
    assert c.faces[inputs.YP] == inputs.MOVING_WALL and tuple(c.u_wall[inputs.YP]) == (0.1, 0, 0)
    assert c.edge == {inputs.YP: (0, 0.3, 1.0)}
    assert abs(c.nu - 0.1 * 97 / 3200.0) < 1e-15
    assert inputs.half_cavity(14, 48, 100.0).nz == 24 and inputs.half_cavity(14, 48, 100.0).edge is None
