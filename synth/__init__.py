"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This package only *generates inputs*: tetrahedral meshes built from tensor-product
hexahedral grids, piecewise-constant velocity/density models, source and receiver
layouts, seeded random wavefield states and the closed-form standing-mode initial
condition.  It holds none of the discontinuous-Galerkin arithmetic (no reference
element, no geometric factors, no fluxes, no time stepping): the oracle and the CUDA
library each compute those on their own from what is generated here.
"""

from .meshes import (  # noqa: F401
    HexGrid,
    kuhn_tets,
    unit_cube_mesh,
    layered_box_mesh,
    graded_axis,
    LOCAL_FACE_VERTICES,
    classify_boundary_faces,
)
from .workloads import (  # noqa: F401
    standing_mode,
    random_state,
    Workload,
    config1_cube,
    config2_layered_rtm,
    config3_crop,
    small_layered_rtm,
    tiny_layered_rtm,
    adjoint_box,
    adjoint_box_small,
    adjoint_box_two_level,
    adjoint_box_three_level,
    adjoint_observed_velocity,
    inclusion_box,
    serving_model,
    serving_requests,
)
