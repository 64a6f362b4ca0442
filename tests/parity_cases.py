"""Shared set-up for the GPU parity tests: the same seeded inputs are given to the oracle and to
the CUDA library; nothing here computes any part of the method."""

import numpy as np

from synth import classify_boundary_faces


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


# stated tolerances (relative L2 against the FP64 oracle)
TOL = {"f64": 1e-10, "f32": 1e-5}


def mixed_bc(w):
    """Free surface on top (z = 0), rigid bottom, transparent sides."""
    zmax = float(w.xyz[:, 2].max())
    xmax, ymax = float(w.xyz[:, 0].max()), float(w.xyz[:, 1].max())
    rules = [(2, 0.0, 1), (2, zmax, 3), (0, 0.0, 2), (0, xmax, 2), (1, 0.0, 2), (1, ymax, 2)]
    return classify_boundary_faces(w.xyz, w.tets, rules)
