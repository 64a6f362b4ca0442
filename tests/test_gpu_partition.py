"""Domain decomposition in the library (ridg_group_*, Sec. 4.2): a shot over a mesh split into parts,
one solver per part (here all on one GPU, each with its own stream), interface traces copied between
the parts after every fine step.

* The union of the parts' traces and images equals the single solver's shot over the whole mesh bit
  for bit (every element computes from the same inputs), and the oracle's at the stated tolerances.
* On the box whose finest elements are isolated, the steps that advance the finest level only copy
  nothing; on the tiny mesh, whose finest level is most of the mesh, every step copies.
* Malformed partitions are refused."""

import numpy as np
import pytest

from oracle.partition import partition
from oracle.rtm import make_problem, rtm_shot
from paper_1506_00907_gb300 import ridg
from synth import inclusion_box, tiny_layered_rtm
from tests.parity_cases import TOL, rel_l2

pytestmark = pytest.mark.gpu


def _case(name):
    w = inclusion_box() if name == "inclusions" else tiny_layered_rtm(N=3, t_final=0.003)
    prob = make_problem(w.xyz, w.tets, w.c, w.rho, w.N, default_bc=w.default_bc, cfl=w.cfl,
                        n_levels_max=w.n_levels_max)
    return w, prob


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("name,n_parts", [("inclusions", 2), ("tiny", 3)])
def test_group_shot_equals_single_solver_and_oracle(name, n_parts, dtype):
    w, prob = _case(name)
    part = partition(prob.geo, prob.levels, prob.n_levels, n_parts)
    mesh = ridg.Mesh(w.xyz, w.tets, default_bc=w.default_bc)
    args = (w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final)
    g = ridg.Group(mesh, w.N, w.c, w.rho, part, dtype=dtype, cfl=w.cfl, n_levels_max=w.n_levels_max)
    tr, ip, iq = g.rtm_shot(*args)
    s = ridg.Solver(mesh, w.N, w.c, w.rho, dtype=dtype, cfl=w.cfl, n_levels_max=w.n_levels_max)
    tr1, ip1, iq1 = s.rtm_shot(*args)
    assert np.abs(tr1).max() > 0 and np.abs(ip1).max() > 0
    assert np.array_equal(tr, tr1) and np.array_equal(ip, ip1) and np.array_equal(iq, iq1)
    info = g.info()
    assert info.n_parts == n_parts
    assert sum(info.elements[:n_parts]) == w.K
    assert all(info.interface_faces[p] > 0 for p in range(n_parts))
    assert info.transfer_bytes > 0 and info.transfer_steps > 0
    st = s.shot_stats()
    assert info.dof_updates == st.dof_updates_forward + st.dof_updates_backward
    # steps that advance the finest level only copy nothing exactly when lumping kept it inside
    assert (info.silent_steps > 0) == (name == "inclusions")
    ref = rtm_shot(prob, *args)
    assert rel_l2(tr, ref.traces) < TOL[dtype]
    assert rel_l2(ip, ref.image_p) < TOL[dtype] and rel_l2(iq, ref.image_q) < TOL[dtype]


def test_group_shot_with_observed_data_and_window():
    """Observed data that are not the modelled traces and an image window starting half-way, FP32, the
    partition of the library's own partitioner."""
    w, prob = _case("tiny")
    mesh = ridg.Mesh(w.xyz, w.tets, default_bc=w.default_bc)
    part = ridg.partition(mesh, w.N, w.c, 2, cfl=w.cfl, n_levels_max=w.n_levels_max)
    g = ridg.Group(mesh, w.N, w.c, w.rho, part, cfl=w.cfl, n_levels_max=w.n_levels_max)
    n_t = g.trace_len(w.t_final)
    obs = np.random.default_rng(23).standard_normal((len(w.receivers), n_t))
    args = (w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final, 0.5 * w.t_final)
    tr, ip, iq = g.rtm_shot(*args, observed=obs)
    s = ridg.Solver(mesh, w.N, w.c, w.rho, cfl=w.cfl, n_levels_max=w.n_levels_max)
    tr1, ip1, iq1 = s.rtm_shot(*args, observed=obs)
    assert np.array_equal(tr, tr1) and np.array_equal(ip, ip1) and np.array_equal(iq, iq1)
    assert np.abs(ip).max() > 0


def test_group_rejects_malformed_partitions():
    w, prob = _case("inclusions")
    mesh = ridg.Mesh(w.xyz, w.tets, default_bc=w.default_bc)
    bad = np.zeros(w.K, dtype=np.int32)
    bad[0] = 5  # parts 1..4 empty
    with pytest.raises(ridg.RidgError) as e:
        ridg.Group(mesh, w.N, w.c, w.rho, bad, cfl=w.cfl, n_levels_max=w.n_levels_max)
    assert e.value.code == -1
    neg = np.zeros(w.K, dtype=np.int32)
    neg[3] = -1
    with pytest.raises(ridg.RidgError):
        ridg.Group(mesh, w.N, w.c, w.rho, neg, cfl=w.cfl, n_levels_max=w.n_levels_max)
