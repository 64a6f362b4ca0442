"""Closed-form pressure of a point source in a homogeneous medium, shared by the CPU pin of the
oracle and the GPU check of the library (nothing here is part of the method).

The system dp/dt + rho c^2 div v = f(t) delta(x - x0), rho dv/dt + grad p = 0 gives
p_tt - c^2 lap p = f'(t) delta(x - x0), whose solution in free space is
p(r, t) = f'(t - r/c) / (4 pi c^2 r): independent of rho.  The source scaling that would follow
from adding the source to the weak form scaled by 1/(rho c^2) is rho c^2 times larger."""

import numpy as np

from synth.meshes import HexGrid

C, RHO, F0 = 1.5, 2.0, 2.5  # rho c^2 = 4.5, so the two source scalings differ plainly
T_PEAK = 1.2 / F0
SOURCE = np.array([0.013, 0.021, 0.017])  # inside an element near the centre of the cube
RECEIVER = np.array([0.5, 0.0, 0.0])


def cube(n):
    """[-1, 1]^3 cut into n^3 hexahedra x 6 tetrahedra (homogeneous C, RHO)."""
    ax = np.linspace(-1.0, 1.0, n + 1)
    xyz, tets = HexGrid(ax, ax.copy(), ax.copy()).mesh()
    return xyz, tets


def t_end():
    """End of the direct pulse at the receiver; reflections from the transparent walls come later
    (the nearest wall, at normal incidence, reflects almost nothing)."""
    return T_PEAK + np.linalg.norm(RECEIVER - SOURCE) / C + 1.2 / F0


def pressure(t):
    """f'(t - r/c) / (4 pi c^2 r) for the unit Ricker pulse f(t) = (1 - 2a tau^2) exp(-a tau^2),
    a = (pi f0)^2, tau = t - t_peak."""
    r = np.linalg.norm(RECEIVER - SOURCE)
    a = (np.pi * F0) ** 2
    tau = np.asarray(t, dtype=np.float64) - r / C - T_PEAK
    fprime = np.exp(-a * tau**2) * (-6.0 * a * tau + 4.0 * a * a * tau**3)
    return fprime / (4.0 * np.pi * C * C * r)
