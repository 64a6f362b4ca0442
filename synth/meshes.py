"""Conforming tetrahedral meshes from tensor-product hexahedral grids.

Every hexahedron is cut into six tetrahedra along its main diagonal (the Kuhn, or
"path", subdivision).  All hexahedra use the same diagonal direction, so the
triangulation is conforming across the whole grid.  Tetrahedra are emitted with
positive orientation: det[v1-v0, v2-v0, v3-v0] > 0.

Local face numbering is an interface convention of the C ABI (``include/ridg.h``):
local face f of tetrahedron (v0, v1, v2, v3) has the vertices LOCAL_FACE_VERTICES[f].
It is used here only to label boundary faces with a boundary-condition code.
"""

from __future__ import annotations

from dataclasses import dataclass
from itertools import permutations

import numpy as np

# Local face f of a tetrahedron (v0,v1,v2,v3): the vertex triple that spans it.
# Face 0 is opposite v3, face 1 opposite v2, face 2 opposite v0, face 3 opposite v1.
LOCAL_FACE_VERTICES = ((0, 1, 2), (0, 1, 3), (1, 2, 3), (0, 2, 3))

BC_AUTO, BC_FREE, BC_TRANSPARENT, BC_RIGID = 0, 1, 2, 3


def graded_axis(lo: float, hi: float, h: float, bands=()) -> np.ndarray:
    """Cell edges of a 1-D axis: uniform cells of size ``h`` on [lo, hi], then each
    band ``(a, b, factor)`` splits every cell that overlaps (a, b) into ``factor``
    equal cells.  Bands are applied in order, so a later band nests inside an earlier one.
    """
    n = int(round((hi - lo) / h))
    if n < 1 or abs(n * h - (hi - lo)) > 1e-9 * max(1.0, abs(hi - lo)):
        raise ValueError("h must divide the axis length")
    edges = list(lo + h * np.arange(n + 1))
    for a, b, factor in bands:
        new = [edges[0]]
        for x0, x1 in zip(edges[:-1], edges[1:]):
            if min(x1, b) - max(x0, a) > 1e-12 * (hi - lo):
                for i in range(1, factor):
                    new.append(x0 + (x1 - x0) * i / factor)
            new.append(x1)
        edges = new
    return np.asarray(edges, dtype=np.float64)


def kuhn_tets(nx: int, ny: int, nz: int) -> np.ndarray:
    """Vertex indices [6*nx*ny*nz, 4] of the Kuhn split of an nx x ny x nz hex grid whose
    grid vertex (i, j, k) has index i + (nx+1)*(j + (ny+1)*k).  Orientation is positive
    provided the grid coordinates increase along each axis."""
    sx, sy = 1, nx + 1
    sz = (nx + 1) * (ny + 1)
    step = np.array([sx, sy, sz], dtype=np.int64)
    i, j, k = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    base = (i * sx + j * sy + k * sz).transpose(2, 1, 0).reshape(-1)  # x fastest
    tets = []
    for perm in permutations(range(3)):
        v0 = base
        v1 = v0 + step[perm[0]]
        v2 = v1 + step[perm[1]]
        v3 = v2 + step[perm[2]]
        # sign of the permutation decides the orientation of (v0, v1, v2, v3)
        inversions = sum(1 for a in range(3) for b in range(a + 1, 3) if perm[a] > perm[b])
        if inversions % 2 == 0:
            tets.append(np.stack([v0, v1, v2, v3], axis=1))
        else:
            tets.append(np.stack([v0, v1, v3, v2], axis=1))
    # interleave so that the six tetrahedra of one hexahedron are consecutive
    t = np.stack(tets, axis=1).reshape(-1, 4)
    return t


@dataclass
class HexGrid:
    xs: np.ndarray
    ys: np.ndarray
    zs: np.ndarray

    @property
    def shape(self):
        return len(self.xs) - 1, len(self.ys) - 1, len(self.zs) - 1

    def vertices(self) -> np.ndarray:
        X, Y, Z = np.meshgrid(self.xs, self.ys, self.zs, indexing="ij")
        return np.stack(
            [X.transpose(2, 1, 0).reshape(-1), Y.transpose(2, 1, 0).reshape(-1), Z.transpose(2, 1, 0).reshape(-1)],
            axis=1,
        ).astype(np.float64)

    def tets(self) -> np.ndarray:
        return kuhn_tets(*self.shape)

    def mesh(self):
        return self.vertices(), self.tets()


def unit_cube_mesh(n: int = 4):
    """[0,1]^3 cut into n^3 hexahedra x 6 tetrahedra."""
    ax = np.linspace(0.0, 1.0, n + 1)
    return HexGrid(ax, ax.copy(), ax.copy()).mesh()


def layered_box_mesh(lx, ly, lz, h, xbands=(), ybands=(), zbands=()):
    """Box [0,lx] x [0,ly] x [0,lz] (z = depth) with graded tensor-product spacing."""
    g = HexGrid(graded_axis(0.0, lx, h, xbands), graded_axis(0.0, ly, h, ybands), graded_axis(0.0, lz, h, zbands))
    return g


def classify_boundary_faces(xyz: np.ndarray, tets: np.ndarray, rules) -> np.ndarray:
    """Boundary-condition code per (element, local face), int8 [K, 4].

    ``rules`` is a list of ``(axis, value, code)``: a local face whose three vertices all
    lie on the plane x_axis == value gets ``code``.  Other faces get 0 (automatic:
    interior where a neighbour exists, else the solver's default boundary condition).
    """
    K = tets.shape[0]
    out = np.zeros((K, 4), dtype=np.int8)
    for f, fv in enumerate(LOCAL_FACE_VERTICES):
        pts = xyz[tets[:, list(fv)]]  # [K, 3, 3]
        for axis, value, code in rules:
            tol = 1e-9 * max(1.0, float(np.max(np.abs(xyz[:, axis]))))
            on = np.all(np.abs(pts[:, :, axis] - value) < tol, axis=1)
            out[on, f] = code
    return out
