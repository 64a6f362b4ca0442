"""A plane pressure pulse travelling along a bar, shared by the CPU pin of the oracle and the GPU
check of the library (nothing here is part of the method).

p = g(x - c t), v = (p / (rho c), 0, 0) solves the system exactly; rigid side walls (n.v = 0)
leave it undisturbed.  The pulse reaches the end x = 2 and either leaves through a transparent
face (Eq. ABC, p - rho c n.v = 0, exact for this wave at normal incidence) or is reflected by a
rigid one."""

import numpy as np

from synth.meshes import HexGrid, classify_boundary_faces

C, RHO, WIDTH, X0 = 2.0, 1.5, 0.12, 0.7
T_END = 1.8 / C  # the pulse has left x = 2 (or come back, reflected)


def bar(end_code, n=16):
    """[0, 2] x [0, 0.25]^2, n x 2 x 2 hexahedra x 6; transparent at x = 0, end_code at x = 2,
    rigid sides."""
    ax, ay = np.linspace(0.0, 2.0, n + 1), np.linspace(0.0, 0.25, 3)
    xyz, tets = HexGrid(ax, ay, ay.copy()).mesh()
    rules = [(0, 0.0, 2), (0, 2.0, end_code), (1, 0.0, 3), (1, 0.25, 3), (2, 0.0, 3), (2, 0.25, 3)]
    return xyz, tets, classify_boundary_faces(xyz, tets, rules)


def state(x, t):
    """Fields [K, 4, Np] of the right-going pulse at time t on nodes x [K, Np, 3]."""
    g = np.exp(-(((x[..., 0] - X0 - C * t) / WIDTH) ** 2))
    q = np.zeros((x.shape[0], 4, x.shape[1]))
    q[:, 0] = g
    q[:, 1] = g / (RHO * C)
    return q
