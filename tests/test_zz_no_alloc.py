"""The allocation-free energy entry point (ridg_energy_noalloc) against ridg_energy.

Some callers cannot allocate device memory when they need the energy check (an application that
owns a fixed device-memory budget, or a time-critical loop in which cudaMalloc must not run because
it can block and synchronise the device); ridg_energy_noalloc serves them from a fixed static
scratch array and writes into a device buffer the caller owns.  This file is collected last so that
a failure here leaves every other test already run; it passes alone and after the others."""

import numpy as np
import pytest

from oracle.rtm import make_problem
from oracle.dg_rhs import energy
from paper_1506_00907_gb300 import ridg
from synth import random_state, tiny_layered_rtm

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_energy_noalloc_matches_energy_on_two_calls(dtype):
    import torch

    w = tiny_layered_rtm(N=3)
    mesh = ridg.Mesh(w.xyz, w.tets, default_bc=w.default_bc)
    s = ridg.Solver(mesh, w.N, w.c, w.rho, dtype=dtype, cfl=w.cfl, n_levels_max=w.n_levels_max)
    geo = make_problem(w.xyz, w.tets, w.c, w.rho, w.N, default_bc=w.default_bc, cfl=w.cfl,
                       n_levels_max=w.n_levels_max).geo
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    for seed in (21, 22):  # two calls in a row, different fields
        q = random_state(w.K, s.Np, seed=seed)
        s.set_state(q)
        e_ref = s.energy()
        # both entry points against the oracle's energy of the same (working-precision) fields; the
        # FP32 solver's material factors are FP32 too (2^-24 each), hence 1e-6 there
        e_oracle = energy(q.astype(np.float32).astype(np.float64) if dtype == "f32" else q, geo)
        tol = 1e-6 if dtype == "f32" else 1e-12
        assert abs(e_ref - e_oracle) <= tol * e_oracle
        s.energy_noalloc(out[seed - 21:])
        torch.cuda.synchronize()
        e_new = float(out[seed - 21].item())
        assert np.isfinite(e_new) and e_ref > 0
        # same FP64 accumulation, different summation order
        assert abs(e_new - e_ref) <= 1e-12 * abs(e_ref)
        assert abs(e_new - e_oracle) <= tol * e_oracle
