"""FP64 CPU oracle for the nodal-DG acoustic RTM hot path (test infrastructure only).

This package is the slow, plain reference the CUDA library is checked against.  It is
test infrastructure: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
and reference legs of ``bench.py`` may import it.  It shares no code with the CUDA
library (``paper_1506_00907_gb300``) and imports nothing from it; the two meet only in
the seeded inputs of the ``synth`` package.

Modules follow the paper (Modave, St-Cyr, Mulder, Warburton, "Nodal discontinuous
Galerkin simulations for reverse-time migration on GPU clusters"):

* ``reference_element`` -- nodes, differentiation, mass, face-mass and lifting
  matrices of the reference tetrahedron (Sec. 3.1 and the appendix).
* ``mesh_geometry`` -- affine maps, geometric factors g^vol, g^sur, outward normals,
  face connectivity, point location and the L2-projected Dirac (Eq. sourceTerm).
* ``dg_rhs`` -- the semi-discrete right-hand side (Eqs. dgLocalSchemeP/U) with the
  penalty fluxes of Eqs. weakFormP/V and the boundary conditions of Sec. 2.
* ``mrab`` -- levels and the multi-rate Adams-Bashforth procedure (Sec. 3.2,
  Eqs. updateAB / updateABcoarse, Algorithm 1), forward and backward in time.
* ``imaging`` -- the AB3-exact image increments (Sec. 3.3, Eq. updateABcorr) for
  the classical (Eq. imageP) and characteristic (Eqs. imageQ, charact) conditions.
* ``rtm`` -- one RTM shot: forward run with boundary-trace recording, backward
  source re-simulation with replay, backward receiver run, image accumulation
  (Sec. 2, Sec. 4.3); forward modelling alone.
* ``wavelet`` -- the Ricker pulse, sampled source signals and the cubic interpolation of
  receiver data in time.
* ``adjoint`` -- the least-squares trace misfit and its gradient with respect to the
  per-element velocity (discrete adjoint of the single-rate scheme; the operator is
  assembled from ``dg_rhs`` and transposed as a sparse matrix; with several rate levels,
  reverse accumulation over the fine steps of Algorithm 1, their matrices assembled from
  ``mrab``).

Every function is FP64 and follows the paper's steps in the paper's order; matrix
products from numpy serve as single steps.  Readings of places where the paper is
silent or garbled are stated in the docstrings where they apply.

Every function is pinned by CPU tests against closed forms, invariants, printed
coefficients or brute force.  Parity unpinned: the absolute images of a whole shot on
a large model (the paper publishes no image values); they are held only by this
oracle's agreement with the CUDA path on the shots it can run and by the invariants
of the image increments.
"""
