"""Named synthetic workloads (meshes, media, sources, receivers) and seeded states.

The workloads are shaped like the paper's experiments:

* ``config1_cube`` -- unit cube, 4x4x4 hexahedra x 6 tetrahedra = 384 tetrahedra, N=3,
  c = rho = 1, rigid walls, the standing mode cos(pi x) cos(pi y) cos(pi z) as the
  initial pressure, one rate level, 200 steps, FP64.  The stated "CFL 0.5" is unstable
  for AB3 with Delta t = C l_k/((N+1)^2 c_k); the paper's own C = 0.15 is used.
* ``config2_layered_rtm`` -- a 2 km x 2 km x 1 km box (z = depth) with 1500 m/s over
  2500 m/s (interface at 500 m), rho = 1000 kg/m^3, about 2e5 tetrahedra refined 2x
  near the interface and 2x/4x around the source so that three rate levels occur,
  N=4, 10 Hz Ricker at (1000, 1000, 8) m, 201 receivers on x = 0..2000 m at y = 1000 m,
  z = 10 m, a 1.5 s record, transparent boundaries, FP32.  It stands in for the
  paper's salt-dome survey (whose mesh and model are not available).
* ``small_layered_rtm`` -- the same recipe on a box small enough for the oracle.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .meshes import BC_RIGID, BC_TRANSPARENT, graded_axis, HexGrid, unit_cube_mesh


def standing_mode(x, y, z, t, c=1.0, rho=1.0):
    """Closed-form standing mode in the unit cube with rigid walls:
    p = cos(pi x) cos(pi y) cos(pi z) cos(w t), v_i = (pi/(rho w)) sin(pi x_i) prod_{j!=i} cos(pi x_j) sin(w t),
    w = c pi sqrt(3).  Returns (p, vx, vy, vz)."""
    w = c * np.pi * np.sqrt(3.0)
    cx, cy, cz = np.cos(np.pi * x), np.cos(np.pi * y), np.cos(np.pi * z)
    sx, sy, sz = np.sin(np.pi * x), np.sin(np.pi * y), np.sin(np.pi * z)
    a = np.pi / (rho * w) * np.sin(w * t)
    return cx * cy * cz * np.cos(w * t), a * sx * cy * cz, a * cx * sy * cz, a * cx * cy * sz


def random_state(K, Np, seed, scale=1.0):
    """Seeded smooth-free random state [K, 4, Np] (p, vx, vy, vz), standard normal * scale."""
    rng = np.random.default_rng(seed)
    return scale * rng.standard_normal((K, 4, Np))


@dataclass
class Workload:
    name: str
    xyz: np.ndarray
    tets: np.ndarray
    c: np.ndarray
    rho: np.ndarray
    N: int
    default_bc: int
    face_bc: np.ndarray | None = None
    cfl: float = 0.5
    n_levels_max: int = 3
    dtype: str = "f32"
    source_xyz: tuple = (0.0, 0.0, 0.0)
    f0: float = 10.0
    t_peak: float = 0.13524
    amplitude: float = 1.0
    receivers: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    t_final: float = 0.0
    t_image_start: float = 0.0
    e_up: tuple = (0.0, 0.0, -1.0)
    n_steps: int = 0

    @property
    def K(self):
        return self.tets.shape[0]


def config1_cube() -> Workload:
    xyz, tets = unit_cube_mesh(4)
    K = tets.shape[0]
    return Workload("cube384_N3_rigid_fp64", xyz, tets, np.ones(K), np.ones(K), N=3, default_bc=BC_RIGID,
                    cfl=0.15, n_levels_max=1, dtype="f64", n_steps=200)


def _layered(lx, ly, lz, h, src, interface, c_top, c_bottom, rho, xb, yb, zb):
    g = HexGrid(graded_axis(0.0, lx, h, xb), graded_axis(0.0, ly, h, yb), graded_axis(0.0, lz, h, zb))
    xyz, tets = g.mesh()
    zc = xyz[tets][:, :, 2].mean(axis=1)
    c = np.where(zc < interface, c_top, c_bottom).astype(np.float64)
    return g, xyz, tets, c, np.full(tets.shape[0], rho, dtype=np.float64)


def config2_layered_rtm() -> Workload:
    """About 2e5 tetrahedra, three rate levels (see module docstring)."""
    lx, ly, lz, h = 2000.0, 2000.0, 1000.0, 62.5
    xs_src, ys_src = 1000.0, 1000.0
    xb = [(xs_src - 125.0, xs_src + 125.0, 2), (xs_src - 31.25, xs_src + 31.25, 2)]
    yb = [(ys_src - 125.0, ys_src + 125.0, 2), (ys_src - 31.25, ys_src + 31.25, 2)]
    zb = [(0.0, 62.5, 2), (400.0, 600.0, 2), (0.0, 31.25, 2)]
    g, xyz, tets, c, rho = _layered(lx, ly, lz, h, (xs_src, ys_src), 500.0, 1500.0, 2500.0, 1000.0, xb, yb, zb)
    rec = np.stack([np.arange(0.0, 2000.0 + 1e-9, 10.0), np.full(201, 1000.0), np.full(201, 10.0)], axis=1)
    return Workload("layered2km_N4_3lev_rtm_fp32", xyz, tets, c, rho, N=4, default_bc=BC_TRANSPARENT,
                    cfl=0.15, n_levels_max=3, dtype="f32", source_xyz=(xs_src, ys_src, 8.0), f0=10.0,
                    t_peak=0.1127 * 12.0 / 10.0, receivers=rec, t_final=1.5, t_image_start=0.0)


def config3_crop(N=5, f0=50.0, t_final=0.04) -> Workload:
    """The 1/8-volume crop [500, 1500]^2 x [250, 750] m of the layered bench model (its elements whose
    centroids lie inside, transparent faces on the cut; it holds the interface at 500 m and the
    refined bands), order N (5 or 6), source at (1000, 1000, 250) m on the crop's top, 50 receivers on
    z = 260 m along y = 1000 m; a Ricker pulse of f0 (50 Hz by default, t_peak = 0.1127 * 12 / f0) so
    that the whole pulse lies inside a short record."""
    w = config2_layered_rtm()
    cen = w.xyz[w.tets].mean(axis=1)
    keep = ((cen[:, 0] > 500.0) & (cen[:, 0] < 1500.0) & (cen[:, 1] > 500.0) & (cen[:, 1] < 1500.0)
            & (cen[:, 2] > 250.0) & (cen[:, 2] < 750.0))
    tets = w.tets[keep]
    used = np.unique(tets)
    remap = np.full(w.xyz.shape[0], -1, dtype=np.int64)
    remap[used] = np.arange(used.size)
    rec = np.stack([np.arange(510.0, 1490.0 + 1e-9, 20.0), np.full(50, 1000.0), np.full(50, 260.0)], axis=1)
    return Workload(f"layered_crop_N{N}", w.xyz[used], remap[tets], w.c[keep], w.rho[keep], N=N,
                    default_bc=BC_TRANSPARENT, cfl=0.15, n_levels_max=3, dtype="f32", source_xyz=(1000.0, 1000.0, 250.0),
                    f0=f0, t_peak=0.1127 * 12.0 / f0, receivers=rec, t_final=t_final)


def small_layered_rtm(N=3, t_final=0.12) -> Workload:
    """A 400 x 400 x 200 m version of the layered RTM recipe for oracle-sized checks."""
    lx, ly, lz, h = 400.0, 400.0, 200.0, 50.0
    xb = [(150.0, 250.0, 2), (190.0, 210.0, 2)]
    yb = [(150.0, 250.0, 2), (190.0, 210.0, 2)]
    zb = [(80.0, 120.0, 2), (0.0, 12.5, 2)]
    g, xyz, tets, c, rho = _layered(lx, ly, lz, h, (200.0, 200.0), 100.0, 1500.0, 2500.0, 1000.0, xb, yb, zb)
    rec = np.stack([np.linspace(20.0, 380.0, 19), np.full(19, 200.0), np.full(19, 10.0)], axis=1)
    return Workload("layered400m_small_rtm", xyz, tets, c, rho, N=N, default_bc=BC_TRANSPARENT, cfl=0.15,
                    n_levels_max=3, dtype="f32", source_xyz=(200.0, 200.0, 8.0), f0=25.0,
                    t_peak=0.1127 * 12.0 / 25.0, receivers=rec, t_final=t_final, t_image_start=0.0)


def adjoint_box(seed=0) -> Workload:
    """6x6x3 hexahedra x 6 = 648 tetrahedra on 600 x 600 x 300 m with a smooth seeded velocity."""
    ax = np.linspace(0.0, 600.0, 7)
    g = HexGrid(ax, ax.copy(), np.linspace(0.0, 300.0, 4))
    xyz, tets = g.mesh()
    cen = xyz[tets].mean(axis=1)
    rng = np.random.default_rng(seed)
    u = rng.standard_normal(tets.shape[0])
    d2 = ((cen[:, None, :] - cen[None, :, :]) ** 2).sum(axis=2)
    Wt = np.exp(-d2 / (2 * 150.0 ** 2))
    s = Wt @ u
    s = (s - s.min()) / (s.max() - s.min())
    c = 1500.0 + 1500.0 * s
    rec = np.stack(np.meshgrid(np.linspace(100, 500, 5), np.linspace(100, 500, 5), indexing="ij"), axis=-1).reshape(-1, 2)
    rec = np.concatenate([rec, np.full((25, 1), 10.0)], axis=1)
    return Workload("box648_N3_adjoint", xyz, tets, c, np.full(tets.shape[0], 1000.0), N=3,
                    default_bc=BC_TRANSPARENT, cfl=0.15, n_levels_max=1, dtype="f32", source_xyz=(300.0, 300.0, 8.0),
                    f0=10.0, t_peak=0.13524, receivers=rec, t_final=0.5)


def inclusion_box(seed=3, n_fast=3) -> Workload:
    """The 648-tetrahedron box (6x6x3 hexahedra, 600 x 600 x 300 m) at 1500 m/s with ``n_fast``
    isolated elements (seeded, none sharing a vertex) at 6000 m/s, N = 2: the fast elements are
    the only ones of the finest of three rate levels, as in the paper's survey where the finest
    elements are few and isolated; for checks of the domain decomposition."""
    ax = np.linspace(0.0, 600.0, 7)
    g = HexGrid(ax, ax.copy(), np.linspace(0.0, 300.0, 4))
    xyz, tets = g.mesh()
    K = tets.shape[0]
    rng = np.random.default_rng(seed)
    fast = []
    for k in rng.permutation(K):
        if all(not (set(tets[k]) & set(tets[j])) for j in fast):
            fast.append(int(k))
        if len(fast) == n_fast:
            break
    c = np.full(K, 1500.0)
    c[fast] = 6000.0
    rec = np.stack([np.linspace(50.0, 550.0, 11), np.full(11, 300.0), np.full(11, 10.0)], axis=1)
    return Workload("box648_N2_inclusions", xyz, tets, c, np.full(K, 1000.0), N=2, default_bc=BC_TRANSPARENT,
                    cfl=0.15, n_levels_max=3, dtype="f64", source_xyz=(300.0, 300.0, 8.0), f0=25.0,
                    t_peak=0.1127 * 12.0 / 25.0, receivers=rec, t_final=0.004)


def adjoint_observed_velocity(w: Workload, amplitude=0.05, sigma=100.0) -> np.ndarray:
    """Velocity of the observed data: c (1 + amplitude g), g a Gaussian bump of width sigma at the
    centre of the box."""
    cen = w.xyz[w.tets].mean(axis=1)
    mid = 0.5 * (w.xyz.min(axis=0) + w.xyz.max(axis=0))
    g = np.exp(-((cen - mid) ** 2).sum(axis=1) / (2 * sigma ** 2))
    return w.c * (1.0 + amplitude * g)


def adjoint_box_small() -> Workload:
    """2 x 2 x 1 hexahedra x 6 = 24 tetrahedra on 200 x 200 x 100 m, N = 2, a velocity that
    varies per element, one level; for checks the oracle's gradient can run on the CPU."""
    ax = np.linspace(0.0, 200.0, 3)
    g = HexGrid(ax, ax.copy(), np.linspace(0.0, 100.0, 2))
    xyz, tets = g.mesh()
    K = tets.shape[0]
    c = 1500.0 + 1000.0 * np.random.default_rng(1).uniform(size=K)
    rec = np.array([[50.0, 50.0, 10.0], [150.0, 60.0, 10.0], [100.0, 150.0, 20.0]])
    w = Workload("box24_N2_adjoint", xyz, tets, c, np.full(K, 1000.0), N=2, default_bc=BC_TRANSPARENT, cfl=0.15,
                 n_levels_max=1, dtype="f64", source_xyz=(100.0, 100.0, 8.0), f0=40.0,
                 t_peak=0.1127 * 12.0 / 40.0, receivers=rec, t_final=0.08)
    w.c_observed = adjoint_observed_velocity(w, sigma=60.0)
    return w


def adjoint_box_two_level() -> Workload:
    """The 24-tetrahedron box of ``adjoint_box_small`` at N = 1 with a velocity contrast across
    x = 100 m (about 1500 and 3600 m/s, each varied by up to 10 % per element), so that the
    elements fall on two rate levels (12 each); for checks of the oracle's multi-rate gradient."""
    w = adjoint_box_small()
    cen = w.xyz[w.tets].mean(axis=1)
    c = np.where(cen[:, 0] < 100.0, 1500.0, 3600.0) * (1.0 + 0.1 * np.random.default_rng(1).uniform(size=w.K))
    v = Workload("box24_N1_two_level", w.xyz, w.tets, c, w.rho.copy(), N=1, default_bc=w.default_bc, cfl=w.cfl,
                 n_levels_max=2, dtype="f64", source_xyz=w.source_xyz, f0=w.f0, t_peak=w.t_peak,
                 receivers=w.receivers, t_final=w.t_final)
    v.c_observed = adjoint_observed_velocity(v, sigma=60.0)
    return v


def adjoint_box_three_level() -> Workload:
    """The 24-tetrahedron box at N = 1 with three velocity zones (about 1500 m/s for x < 100 m,
    3400 m/s for x > 100 m and y < 100 m, 7200 m/s elsewhere, each varied by up to 10 % per
    element), so that the elements fall on three rate levels; for checks of the oracle's
    multi-rate gradient."""
    w = adjoint_box_small()
    cen = w.xyz[w.tets].mean(axis=1)
    c = np.where(cen[:, 0] < 100.0, 1500.0, np.where(cen[:, 1] < 100.0, 3400.0, 7200.0))
    c = c * (1.0 + 0.1 * np.random.default_rng(1).uniform(size=w.K))
    v = Workload("box24_N1_three_level", w.xyz, w.tets, c, w.rho.copy(), N=1, default_bc=w.default_bc, cfl=w.cfl,
                 n_levels_max=3, dtype="f64", source_xyz=w.source_xyz, f0=w.f0, t_peak=w.t_peak,
                 receivers=w.receivers, t_final=w.t_final)
    v.c_observed = adjoint_observed_velocity(v, sigma=60.0)
    return v


def serving_model(size: str, seed=6) -> Workload:
    """One of the three models of the shot-serving stream: a 2 x 2 x 1 km box with three layers
    (1500, 2000, 2500 m/s; interface depths drawn with ``seed``), the surface refined 8x in depth and
    2x around each interface (three rate levels), transparent boundaries.  ``size``: "50k" (N = 3),
    "200k" (N = 4) or "800k" (N = 5) elements, approximately."""
    h, N = {"50k": (100.0, 3), "200k": (2000.0 / 36, 4), "800k": (100.0 / 3, 5)}[size]
    rng = np.random.default_rng(seed)
    z1 = float(rng.uniform(250.0, 450.0))
    z2 = float(rng.uniform(550.0, 800.0))
    zb = [(0.0, h, 2), (0.0, h / 2, 2), (0.0, h / 4, 2), (z1 - h, z1 + h, 2), (z2 - h, z2 + h, 2)]
    g = HexGrid(graded_axis(0.0, 2000.0, h), graded_axis(0.0, 2000.0, h), graded_axis(0.0, 1000.0, h, zb))
    xyz, tets = g.mesh()
    zc = xyz[tets][:, :, 2].mean(axis=1)
    c = np.where(zc < z1, 1500.0, np.where(zc < z2, 2000.0, 2500.0))
    return Workload(f"serving_{size}_N{N}", xyz, tets, c, np.full(tets.shape[0], 1000.0), N=N,
                    default_bc=BC_TRANSPARENT, cfl=0.15, n_levels_max=3, dtype="f32", f0=10.0,
                    t_peak=0.1127 * 12.0 / 10.0)


def serving_requests(n, seed=5):
    """Request stream of the serving benchmark: per request the model index (0..2), a surface source
    position and a receiver line (101..401 receivers at y = 1000 m, z = 10 m)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        m = int(rng.integers(0, 3))
        src = (float(rng.uniform(200.0, 1800.0)), float(rng.uniform(200.0, 1800.0)), 8.0)
        nr = int(rng.integers(101, 402))
        rec = np.stack([np.linspace(0.0, 2000.0, nr), np.full(nr, 1000.0), np.full(nr, 10.0)], axis=1)
        out.append((m, src, rec))
    return out


def tiny_layered_rtm(N=3, t_final=0.03) -> Workload:
    """200 x 200 x 100 m, two layers (interface at 50 m), refined bands around the source:
    three rate levels on 1440 tetrahedra.  Small enough for the oracle to run a whole shot."""
    lx, ly, lz, h = 200.0, 200.0, 100.0, 50.0
    xb = [(75.0, 125.0, 2), (95.0, 105.0, 2)]
    yb = [(75.0, 125.0, 2)]
    zb = [(0.0, 12.5, 2), (0.0, 6.25, 2), (0.0, 3.0, 2)]
    g, xyz, tets, c, rho = _layered(lx, ly, lz, h, (100.0, 100.0), 50.0, 1500.0, 2500.0, 1000.0, xb, yb, zb)
    rec = np.stack([np.linspace(10.0, 190.0, 7), np.full(7, 100.0), np.full(7, 5.0)], axis=1)
    return Workload("layered200m_tiny_rtm", xyz, tets, c, rho, N=N, default_bc=BC_TRANSPARENT, cfl=0.15,
                    n_levels_max=3, dtype="f32", source_xyz=(100.0, 100.0, 4.0), f0=60.0,
                    t_peak=0.1127 * 12.0 / 60.0, receivers=rec, t_final=t_final, t_image_start=0.0)
