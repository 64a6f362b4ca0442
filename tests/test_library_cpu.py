"""C-ABI library on the CPU: it loads, exports every function declared in include/ridg.h, and its
host-side setup (reference operators, mesh checks, error codes) agrees with the oracle.  No
kernel runs here."""

import os
import re

import numpy as np
import pytest

from oracle.reference_element import ReferenceElement
from paper_1506_00907_gb300 import ridg
from synth import tiny_layered_rtm, unit_cube_mesh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open("include/ridg.h").read()
    return sorted(set(re.findall(r"\b(ridg_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = ridg.lib()
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(ridg.EXPORTED)
    assert b"sm_103a" in lib.ridg_version()


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
def test_reference_operators_match_oracle(N):
    ops = ridg.reference_operators(N)
    re_ = ReferenceElement(N)
    scale = 10.0 ** (N - 3)
    assert np.allclose(ops["rst"], re_.rst, atol=1e-14)
    assert np.array_equal(ops["fmask"], re_.Fmask)
    assert np.allclose(ops["D"], re_.D, atol=1e-12 * scale)
    assert np.allclose(ops["M"], re_.M, atol=1e-13)
    assert np.allclose(ops["LIFT"], re_.LIFT, atol=1e-10 * scale)


def test_mesh_counts():
    xyz, tets = unit_cube_mesh(4)
    m = ridg.Mesh(xyz, tets, default_bc=3)
    nb, ni = m.counts()
    assert nb == 192 and 2 * ni + nb == 4 * len(tets)


def test_mesh_errors():
    xyz, tets = unit_cube_mesh(2)
    bad = tets.copy()
    bad[0, [2, 3]] = bad[0, [3, 2]]  # inverted element
    with pytest.raises(ridg.RidgError) as e:
        ridg.Mesh(xyz, bad)
    assert e.value.code == -2
    with pytest.raises(ridg.RidgError) as e:
        ridg.Mesh(xyz, tets + 10 ** 6)
    assert e.value.code == -2
    fb = np.zeros((len(tets), 4), dtype=np.int8)
    fb[:, :] = 1  # boundary code on interior faces
    with pytest.raises(ridg.RidgError) as e:
        ridg.Mesh(xyz, tets, face_bc=fb)
    assert e.value.code == -2
    with pytest.raises(ridg.RidgError) as e:
        ridg.Mesh(xyz, tets, default_bc=7)
    assert e.value.code == -1
    with pytest.raises(ridg.RidgError):
        ridg.reference_operators(9)


def test_layered_mesh_boundary_faces():
    w = tiny_layered_rtm()
    m = ridg.Mesh(w.xyz, w.tets, default_bc=2)
    nb, ni = m.counts()
    assert nb > 0 and 2 * ni + nb == 4 * w.K


def test_point_location_matches_the_oracle():
    """Host point location (grid index) against the oracle's brute-force rule: the lowest element
    index whose barycentric coordinates are all >= -1e-12, and the reference coordinates in it; at
    random points, at mesh vertices, edge midpoints and face centroids (points on several elements)
    and outside the mesh."""
    from oracle.mesh_geometry import MeshGeometry
    from oracle.reference_element import reference_element

    w = tiny_layered_rtm(N=1)
    m = ridg.Mesh(w.xyz, w.tets, default_bc=w.default_bc)
    g = MeshGeometry(w.xyz, w.tets, reference_element(1), default_bc=w.default_bc)
    rng = np.random.default_rng(7)
    lo, hi = w.xyz.min(axis=0), w.xyz.max(axis=0)
    pts = [lo + (hi - lo) * rng.uniform(size=3) for _ in range(60)]
    tets = w.tets[rng.choice(len(w.tets), 20, replace=False)]
    for t in tets:
        v = w.xyz[t]
        pts += [v[0], 0.5 * (v[0] + v[1]), v[:3].mean(axis=0)]
    pts += [hi + 1.0, lo - np.array([0.0, 0.0, 5.0]), np.array([np.nan, 0.0, 0.0])]
    pts = np.array(pts)
    elem, rst = m.locate(pts)
    for x, k, r in zip(pts, elem, rst):
        if not np.all(np.isfinite(x)):
            assert k == -1
            continue
        k_ref, r_ref = g.locate(x)
        assert k == k_ref
        if k >= 0:
            assert np.allclose(r, r_ref, atol=1e-10)


def test_fault_points_arm_and_disarm():
    """Host-side failure points: armed by ridg_inject_fault or by RIDG_FAULT when the library loads,
    disarmed by "none"; unknown names and negative counts are refused (no GPU involved)."""
    import subprocess
    import sys

    ridg.inject_fault("arena", 3)
    assert ridg.fault_armed() == 2
    ridg.inject_fault("none")
    assert ridg.fault_armed() == 0
    with pytest.raises(ridg.RidgError):
        ridg.inject_fault("disk")
    with pytest.raises(ridg.RidgError):
        ridg.inject_fault("alloc", -1)
    code = ("from paper_1506_00907_gb300 import ridg; print(ridg.fault_armed())")
    env = dict(os.environ, RIDG_FAULT="exchange:5")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == "4"
