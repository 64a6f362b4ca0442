"""The library's forward run against the free-space Green's function (see tests/green.py): the
receiver pressure of a Ricker point source in a homogeneous medium approaches
f'(t - r/c) / (4 pi c^2 r) as the mesh is refined and the order raised, in FP64 and FP32."""

import numpy as np
import pytest

from paper_1506_00907_gb300 import ridg
from tests import green

pytestmark = pytest.mark.gpu


def _receiver_pressure(n, N, dtype):
    xyz, tets = green.cube(n)
    K = len(tets)
    mesh = ridg.Mesh(xyz, tets, default_bc=ridg.BC_TRANSPARENT)
    s = ridg.Solver(mesh, N, np.full(K, green.C), np.full(K, green.RHO), dtype=dtype, n_levels_max=1)
    tr, _, _ = s.rtm_shot(tuple(green.SOURCE), green.F0, green.T_PEAK, 1.0, green.RECEIVER[None, :], green.t_end(),
                          want_images=False)
    t = s.info.dt_global * np.arange(tr.shape[1])
    return tr[0], green.pressure(t)


def test_point_source_converges_to_greens_function():
    errs = {}
    for n, N in ((8, 3), (16, 4)):
        p64, pa = _receiver_pressure(n, N, "f64")
        p32, _ = _receiver_pressure(n, N, "f32")
        errs[(n, N)] = np.linalg.norm(p64 - pa) / np.linalg.norm(pa)
        assert np.linalg.norm(p32 - p64) / np.linalg.norm(p64) < 1e-5
    assert errs[(8, 3)] < 0.1, errs
    assert errs[(16, 4)] < errs[(8, 3)] / 4, errs
