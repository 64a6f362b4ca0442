"""Per-element geometry and connectivity (oracle, FP64, test infrastructure).

Appendix of the paper: the affine map Psi_k from the reference tetrahedron to D_k,
its Jacobian J_k, the volume factors (the chain rule needs the inverse Jacobian
d r_j / d x_i; the appendix prints d Psi_i / d r_j, read here as its inverse), the face
factors g^sur = J_{k,f} / J_k, and outward unit normals.  Faces are matched by their
vertex triples; face nodes by their physical coordinates.  Also: the time-step bound
of Sec. 5.1 (smallest face-to-opposite-vertex distance), point location and the
L2-projected point source of Eq. sourceTerm.
"""

from __future__ import annotations

import numpy as np

from .reference_element import FACE_VERTICES, OPPOSITE, ReferenceElement

BC_INTERIOR, BC_FREE, BC_TRANSPARENT, BC_RIGID = 0, 1, 2, 3


class MeshGeometry:
    def __init__(self, xyz, tets, ref: ReferenceElement, face_bc=None, default_bc=BC_TRANSPARENT):
        xyz = np.asarray(xyz, dtype=np.float64)
        tets = np.asarray(tets, dtype=np.int64)
        self.xyz, self.tets, self.ref = xyz, tets, ref
        K = tets.shape[0]
        self.K = K
        P = xyz[tets]  # [K, 4, 3]
        self.P = P
        # affine map x(r) = sum_i lambda_i(r) P_i; columns dx/dr, dx/ds, dx/dt
        A = 0.5 * np.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]], axis=2)  # [K,3(x),3(r)]
        self.A = A
        self.J = np.linalg.det(A)
        if np.any(self.J <= 0):
            raise ValueError("non-positive element Jacobian")
        # rx[k, i, j] = d r_j / d x_i
        self.rx = np.transpose(np.linalg.inv(A), (0, 2, 1))
        # physical node coordinates
        lam = np.stack([-(1 + ref.rst[:, 0] + ref.rst[:, 1] + ref.rst[:, 2]) / 2, (1 + ref.rst[:, 0]) / 2,
                        (1 + ref.rst[:, 1]) / 2, (1 + ref.rst[:, 2]) / 2], axis=1)
        self.x = np.einsum("ni,kid->knd", lam, P)  # [K, Np, 3]
        # outward normals, face areas, face factor
        self.normal = np.zeros((K, 4, 3))
        self.area = np.zeros((K, 4))
        for f, (a, b, c) in enumerate(FACE_VERTICES):
            o = OPPOSITE[f]
            n = np.cross(P[:, b] - P[:, a], P[:, c] - P[:, a])
            flip = np.einsum("kd,kd->k", n, P[:, o] - P[:, a]) > 0
            n[flip] *= -1.0
            nn = np.linalg.norm(n, axis=1)
            self.area[:, f] = 0.5 * nn
            self.normal[:, f] = n / nn[:, None]
        self.Jf = self.area / 2.0  # 2-D reference triangle has area 2
        self.Fscale = self.Jf / self.J[:, None]
        self.volume = self.J * 4.0 / 3.0
        # smallest distance between a face and its opposite vertex = 3 V / (largest face area)
        self.min_height = 3.0 * self.volume / self.area.max(axis=1)
        self._connect(face_bc, default_bc)

    # ------------------------------------------------------------------ connectivity
    def _connect(self, face_bc, default_bc):
        K, ref = self.K, self.ref
        Nfp = ref.Nfp
        self.nbr = -np.ones((K, 4), dtype=np.int64)
        self.nbr_face = -np.ones((K, 4), dtype=np.int64)
        self.bc = np.zeros((K, 4), dtype=np.int64)
        table = {}
        for k in range(K):
            for f, fv in enumerate(FACE_VERTICES):
                key = tuple(sorted(int(self.tets[k, i]) for i in fv))
                table.setdefault(key, []).append((k, f))
        for key, lst in table.items():
            if len(lst) > 2:
                raise ValueError("non-manifold face")
            if len(lst) == 2:
                (k1, f1), (k2, f2) = lst
                self.nbr[k1, f1], self.nbr_face[k1, f1] = k2, f2
                self.nbr[k2, f2], self.nbr_face[k2, f2] = k1, f1
        fb = np.zeros((K, 4), dtype=np.int64) if face_bc is None else np.asarray(face_bc, dtype=np.int64)
        interior = self.nbr >= 0
        if np.any(interior & (fb != 0)):
            raise ValueError("boundary code on a matched face")
        self.bc = np.where(interior, BC_INTERIOR, np.where(fb != 0, fb, default_bc))
        # face-node matching by physical coordinates (brute force per face, in chunks)
        self.nbr_node = -np.ones((K, 4, Nfp), dtype=np.int64)  # index into the neighbour face's node list
        h = float(self.min_height.min())
        ks, fs = np.nonzero(self.nbr >= 0)
        Fm = ref.Fmask
        for lo in range(0, len(ks), 20000):
            k1, f1 = ks[lo:lo + 20000], fs[lo:lo + 20000]
            k2, f2 = self.nbr[k1, f1], self.nbr_face[k1, f1]
            xa = self.x[k1[:, None], Fm[f1]]  # [F, Nfp, 3]
            xb = self.x[k2[:, None], Fm[f2]]
            d = np.linalg.norm(xa[:, :, None, :] - xb[:, None, :, :], axis=3)
            j = np.argmin(d, axis=2)
            if np.max(np.take_along_axis(d, j[:, :, None], axis=2)) > 1e-9 * max(h, 1.0):
                raise ValueError("face nodes do not match")
            self.nbr_node[k1, f1] = j

    # ------------------------------------------------------------------ time step bound
    def dt_bound(self, N, c, cfl):
        """Sec. 5.1: Delta t_k = C l_k / ((N+1)^2 c_k), l_k the smallest face-vertex height."""
        return cfl * self.min_height / ((N + 1) ** 2 * np.asarray(c, dtype=np.float64))

    # ------------------------------------------------------------------ points
    def locate(self, x0):
        """Element containing x0: lowest index whose barycentrics are all >= -1e-12;
        returns (k, reference coordinates) or (-1, None)."""
        x0 = np.asarray(x0, dtype=np.float64)
        if not hasattr(self, "_Binv"):
            B = np.stack([self.P[:, 1] - self.P[:, 0], self.P[:, 2] - self.P[:, 0], self.P[:, 3] - self.P[:, 0]], axis=2)
            self._Binv = np.linalg.inv(B)
        l123 = np.einsum("kij,kj->ki", self._Binv, x0[None, :] - self.P[:, 0])
        lam = np.concatenate([1.0 - l123.sum(axis=1, keepdims=True), l123], axis=1)
        inside = np.nonzero(np.all(lam >= -1e-12, axis=1))[0]
        if len(inside) == 0:
            return -1, None
        k = int(inside[0])
        return k, 2.0 * l123[k] - 1.0

    def source_weights(self, k, rst):
        """Eq. sourceTerm: coefficients w of the L2 projection of delta(x - x0) on element k,
        M_k w = l(x0) with M_k = J_k M."""
        ell = self.ref.lagrange_at(rst)[0]
        return np.linalg.solve(self.J[k] * self.ref.M, ell)

    def interpolation_row(self, rst):
        return self.ref.lagrange_at(rst)[0]
