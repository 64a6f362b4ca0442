"""The allocation-free energy entry point (ridg_energy_noalloc) against ridg_energy.

Some callers cannot allocate device memory when they need the energy check (for instance while a
stream is being captured into a CUDA graph); ridg_energy_noalloc serves them from a fixed static
scratch array and writes into a device buffer the caller owns.  This file is collected last so that
a failure here leaves every other test already run; it passes alone and after the others."""

import numpy as np
import pytest

from paper_1506_00907_gb300 import ridg
from synth import random_state, tiny_layered_rtm

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_energy_noalloc_matches_energy_on_two_calls(dtype):
    import torch

    w = tiny_layered_rtm(N=3)
    mesh = ridg.Mesh(w.xyz, w.tets, default_bc=w.default_bc)
    s = ridg.Solver(mesh, w.N, w.c, w.rho, dtype=dtype, cfl=w.cfl, n_levels_max=w.n_levels_max)
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    for seed in (21, 22):  # two calls in a row, different fields
        s.set_state(random_state(w.K, s.Np, seed=seed))
        e_ref = s.energy()
        s.energy_noalloc(out[seed - 21:])
        torch.cuda.synchronize()
        e_new = float(out[seed - 21].item())
        assert np.isfinite(e_new) and e_ref > 0
        # same FP64 accumulation, different summation order
        assert abs(e_new - e_ref) <= 1e-12 * abs(e_ref)
