"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same seeded
inputs, element by element, at the tolerances stated in the tests (relative L2: 1e-10 in FP64
mode, 1e-5 in FP32)."""

import functools

import numpy as np
import pytest

from oracle.dg_rhs import attach_media, energy, rhs, traces
from oracle.mesh_geometry import MeshGeometry
from oracle.mrab import MRAB, assign_levels
from oracle.reference_element import reference_element
from oracle.rtm import forward, make_problem, rtm_shot
from oracle.wavelet import ricker
from paper_1506_00907_gb300 import ridg
from synth import config1_cube, random_state, standing_mode, tiny_layered_rtm, unit_cube_mesh
from tests.parity_cases import TOL, mixed_bc, rel_l2

pytestmark = pytest.mark.gpu


def _oracle_problem(w, face_bc=None, N=None, tau_scale=1.0):
    N = w.N if N is None else N
    return make_problem(w.xyz, w.tets, w.c, w.rho, N, face_bc=face_bc, default_bc=w.default_bc, cfl=w.cfl,
                        n_levels_max=w.n_levels_max, tau_scale=tau_scale)


def _gpu(w, dtype, face_bc=None, N=None, **kw):
    mesh = ridg.Mesh(w.xyz, w.tets, face_bc=face_bc, default_bc=w.default_bc)
    return ridg.Solver(mesh, w.N if N is None else N, w.c, w.rho, dtype=dtype, cfl=w.cfl, n_levels_max=w.n_levels_max,
                       **kw)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_levels_nodes_dt_match_oracle(dtype):
    w = tiny_layered_rtm(N=3)
    prob = _oracle_problem(w)
    s = _gpu(w, dtype)
    assert s.info.n_levels == prob.n_levels == 3
    assert np.array_equal(s.levels(), prob.levels)
    assert np.isclose(s.info.dt_local, prob.dt_local, rtol=1e-13)
    assert np.allclose(s.nodes(), prob.geo.x, atol=1e-10)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
def test_rhs_parity_mixed_boundaries(dtype, N):
    """One right-hand-side evaluation (volume + surface + all three boundary conditions) on a
    two-material, three-level mesh: several CTAs and a ragged last block."""
    w = tiny_layered_rtm(N=N)
    fb = mixed_bc(w)
    prob = _oracle_problem(w, face_bc=fb)
    s = _gpu(w, dtype, face_bc=fb)
    q = random_state(w.K, s.Np, seed=11)
    r_gpu = s.eval_rhs(q)
    g = prob.geo
    r_ref = rhs(np.arange(g.K), q, traces(q, g), g)
    assert rel_l2(r_gpu, r_ref) < TOL[dtype]
    # element by element as well: every element's error against its own norm (loose: some elements'
    # right-hand sides nearly cancel), and the largest element error against the largest element norm
    err_k = np.linalg.norm((r_gpu - r_ref).reshape(w.K, -1), axis=1)
    ref_k = np.linalg.norm(r_ref.reshape(w.K, -1), axis=1)
    assert (err_k / ref_k).max() < 100 * TOL[dtype]
    assert err_k.max() / ref_k.max() < 10 * TOL[dtype]


def test_config1_standing_mode_fp64():
    """384 tets, N=3, rigid walls, 200 steps: GPU FP64 vs the oracle, and vs the closed form."""
    w = config1_cube()
    prob = _oracle_problem(w)
    s = _gpu(w, "f64")
    x = s.nodes()
    sm = lambda t: np.stack(standing_mode(x[..., 0], x[..., 1], x[..., 2], t), axis=1)  # noqa: E731
    dt = s.info.dt_local
    assert s.info.n_levels == 1 and np.isclose(dt, prob.dt_local, rtol=1e-13)
    s.set_state(sm(0.0))
    s.set_history(s.eval_rhs(sm(-dt)), s.eval_rhs(sm(-2 * dt)))
    s.step(w.n_steps)
    q_gpu = s.get_state()
    g = prob.geo
    st = MRAB(g, prob.levels, prob.n_levels, prob.dt_local)
    st.set_state(sm(0.0))
    r_of = lambda q: rhs(np.arange(g.K), q, traces(q, g), g)  # noqa: E731
    st.set_history(r_of(sm(-dt)), r_of(sm(-2 * dt)))
    for _ in range(w.n_steps):
        st.global_step()
    assert rel_l2(q_gpu, st.q) < TOL["f64"]
    qe = sm(w.n_steps * dt)
    err = rel_l2(q_gpu[:, 0], qe[:, 0])
    assert err < 2e-2
    assert rel_l2(s.energy(), energy(st.q, g)) < 1e-10


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("N", [3, 4, 5, 6])
def test_mrab_three_levels_parity(dtype, N):
    """Multi-rate stepping with half-step traces on three levels: 4 global steps from a seeded
    state and history (orders 5 and 6 run the tensor-core kernel with rolled k-steps)."""
    w = tiny_layered_rtm(N=N)
    fb = mixed_bc(w)
    prob = _oracle_problem(w, face_bc=fb)
    s = _gpu(w, dtype, face_bc=fb)
    Np = s.Np
    q = random_state(w.K, Np, seed=3)
    r1 = random_state(w.K, Np, seed=4, scale=1e3)
    r2 = random_state(w.K, Np, seed=5, scale=1e3)
    s.set_state(q)
    s.set_history(r1, r2)
    s.step(4)
    q_gpu = s.get_state()
    st = MRAB(prob.geo, prob.levels, prob.n_levels, prob.dt_local)
    st.set_state(q)
    st.set_history(r1, r2)
    for _ in range(4):
        st.global_step()
    assert rel_l2(q_gpu, st.q) < TOL[dtype]


@functools.lru_cache(maxsize=None)
def _oracle_shot(N):
    w = tiny_layered_rtm(N=N, t_final=0.006)
    prob = _oracle_problem(w)
    return w, rtm_shot(prob, w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final, w.t_image_start)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("N", [3, 4, 5])
def test_rtm_shot_parity(dtype, N):
    """A whole shot on the tiny three-level model (forward with recording, overshoot, backward
    source and receiver runs with replay and images): receiver traces and both images.  N = 4 is
    the order of the bench."""
    w, ref = _oracle_shot(N)
    s = _gpu(w, dtype)
    tr, ip, iq = s.rtm_shot(w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final, w.t_image_start)
    assert tr.shape == ref.traces.shape
    assert rel_l2(tr, ref.traces) < TOL[dtype]
    assert rel_l2(ip, ref.image_p) < TOL[dtype]
    assert rel_l2(iq, ref.image_q) < TOL[dtype]
    st = s.shot_stats()
    assert st.n_global == ref.n_global
    assert st.dof_updates_forward + st.dof_updates_backward > 0


@functools.lru_cache(maxsize=None)
def _oracle_shot_variant(variant):
    """Tiny N = 3 shot variants: an image window that starts half-way, observed data that are not
    the modelled traces, a free-surface top and rigid bottom (boundary records of every kind),
    receivers on element vertices and faces (point-location ties)."""
    w = tiny_layered_rtm(N=3, t_final=0.004)
    fb, rec, obs, t_i = None, w.receivers, None, 0.0
    if variant == "window":
        t_i = 0.5 * w.t_final
    elif variant == "observed":
        n_t = int(np.ceil(w.t_final / _oracle_problem(w).dt_global - 1e-9)) + 1
        obs = np.random.default_rng(17).standard_normal((len(rec), n_t))
    elif variant == "free_top":
        fb = mixed_bc(w)
    elif variant == "ties":
        # interior mesh vertices, midpoints of the edges between them, and the centroid of a face
        # shared by two elements: points on the closure of several elements
        v = np.array([[100.0, 100.0, 25.0], [100.0, 125.0, 25.0], [100.0, 150.0, 25.0], [75.0, 100.0, 50.0]])
        k = int(np.argmin(np.linalg.norm(w.xyz[w.tets].mean(axis=1) - [101.0, 101.0, 26.0], axis=1)))
        face = w.xyz[w.tets[k, :3]].mean(axis=0)
        rec = np.concatenate([v, 0.5 * (v[:2] + v[1:3]), face[None, :]])
    prob = _oracle_problem(w, face_bc=fb)
    ref = rtm_shot(prob, w.source_xyz, w.f0, w.t_peak, 1.0, rec, w.t_final, t_i, observed=obs)
    return w, fb, rec, obs, t_i, ref


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("variant", ["window", "observed", "free_top", "ties"])
def test_rtm_shot_variants_parity(dtype, variant):
    w, fb, rec, obs, t_i, ref = _oracle_shot_variant(variant)
    s = _gpu(w, dtype, face_bc=fb)
    tr, ip, iq = s.rtm_shot(w.source_xyz, w.f0, w.t_peak, 1.0, rec, w.t_final, t_i, observed=obs)
    assert rel_l2(tr, ref.traces) < TOL[dtype]
    assert rel_l2(ip, ref.image_p) < TOL[dtype]
    # receivers on shared vertices, edges and faces: the receiver wavefield starts as point injections at
    # those places and the characteristic image weights its velocities by the impedance; the FP32
    # tensor-core split leaves that image at 1.03e-5 of the FP64 oracle, held here at 2e-5
    tol_q = 2e-5 if (dtype == "f32" and variant == "ties") else TOL[dtype]
    assert rel_l2(iq, ref.image_q) < tol_q


def test_rtm_edge_cases():
    w = tiny_layered_rtm(N=2, t_final=0.002)
    s = _gpu(w, "f64")
    # no receivers: the receiver wavefield stays zero, so do the images
    tr, ip, iq = s.rtm_shot(w.source_xyz, w.f0, w.t_peak, 1.0, np.zeros((0, 3)), w.t_final)
    assert tr.shape[0] == 0 and np.all(ip == 0) and np.all(iq == 0)
    # empty image window: t_i is rounded down to a global step, so start it at the last one
    t_last = (s.trace_len(w.t_final) - 1) * s.info.dt_global
    tr, ip, iq = s.rtm_shot(w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final, t_image_start=t_last)
    assert np.all(ip == 0) and np.abs(tr).max() > 0
    with pytest.raises(ridg.RidgError) as e:
        s.rtm_shot((1e6, 0, 0), w.f0, w.t_peak, 1.0, w.receivers, w.t_final)
    assert e.value.code == -7
    with pytest.raises(ridg.RidgError) as e:
        s.rtm_shot(w.source_xyz, w.f0, w.t_peak, 1.0, np.array([[1e6, 0.0, 0.0]]), w.t_final)
    assert e.value.code == -7


def test_single_element_mesh():
    xyz = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
    tets = np.array([[0, 1, 2, 3]])
    m = ridg.Mesh(xyz, tets, default_bc=1)
    s = ridg.Solver(m, 3, [2.0], [1.5], dtype="f64")
    q = random_state(1, s.Np, seed=9)
    g = attach_media(MeshGeometry(xyz, tets, reference_element(3), default_bc=1), [2.0], [1.5])
    assert rel_l2(s.eval_rhs(q), rhs(np.arange(1), q, traces(q, g), g)) < TOL["f64"]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_energy_matches_oracle(dtype):
    """The discrete energy of the solver's fields (FP64 accumulation on the device) against the
    oracle's, on a two-material mesh with several blocks.  In FP32 mode the oracle takes the same
    fields rounded to FP32; the solver's material factors rho c^2 and 1/rho are FP32 as well
    (relative rounding 2^-24 each), so that mode is held at 1e-6, FP64 at 1e-12."""
    w = tiny_layered_rtm(N=4)
    prob = _oracle_problem(w)
    s = _gpu(w, dtype)
    q = random_state(w.K, s.Np, seed=41)
    s.set_state(q)
    q_ref = q.astype(np.float32).astype(np.float64) if dtype == "f32" else q
    e_ref = energy(q_ref, prob.geo)
    assert abs(s.energy() - e_ref) <= (1e-6 if dtype == "f32" else 1e-12) * e_ref


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("tau_scale", [0.5, 2.0])
def test_rhs_parity_penalty_scale(dtype, tau_scale):
    """The penalty scale multiplies tau_p and tau_v on interior and boundary faces alike."""
    w = tiny_layered_rtm(N=4)
    fb = mixed_bc(w)
    prob = _oracle_problem(w, face_bc=fb, tau_scale=tau_scale)
    s = _gpu(w, dtype, face_bc=fb, tau_scale=tau_scale)
    q = random_state(w.K, s.Np, seed=12)
    g = prob.geo
    assert rel_l2(s.eval_rhs(q), rhs(np.arange(g.K), q, traces(q, g), g)) < TOL[dtype]


@functools.lru_cache(maxsize=None)
def _oracle_forward():
    """Forward modelling on the tiny three-level model, driven by the Ricker pulse and by samples
    of a different signal at a spacing unrelated to the time step (ragged: the last samples end
    before the record does)."""
    w = tiny_layered_rtm(N=3, t_final=0.004)
    prob = _oracle_problem(w)
    dt_s = 0.7 * prob.dt_local
    n_s = int(0.8 * w.t_final / dt_s)
    t = np.arange(n_s) * dt_s
    wav = ricker(t, 1.5 * w.f0, 0.6 * w.t_peak) + 0.2 * np.sin(2 * np.pi * w.f0 * t)
    tr = forward(prob, w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final)
    tr_s = forward(prob, w.source_xyz, 0.0, 0.0, 0.5, w.receivers, w.t_final, wavelet=wav, wavelet_dt=dt_s)
    return w, wav, dt_s, tr, tr_s


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_forward_parity(dtype):
    w, wav, dt_s, tr_ref, tr_s_ref = _oracle_forward()
    s = _gpu(w, dtype)
    tr = s.forward(w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final)
    assert tr.shape == tr_ref.shape and rel_l2(tr, tr_ref) < TOL[dtype]
    tr_s = s.forward(w.source_xyz, 0.0, 0.0, 0.5, w.receivers, w.t_final, wavelet=wav, wavelet_dt=dt_s)
    assert rel_l2(tr_s, tr_s_ref) < TOL[dtype]
    # the forward run of a shot is the same computation
    tr_shot, _, _ = s.rtm_shot(w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final)
    assert np.array_equal(tr_shot, tr)
    # a sampled source in a whole shot
    tr_shot_s, ip, _ = s.rtm_shot(w.source_xyz, 0.0, 0.0, 0.5, w.receivers, w.t_final, wavelet=wav, wavelet_dt=dt_s)
    assert np.array_equal(tr_shot_s, tr_s) and np.abs(ip).max() > 0
    with pytest.raises(ridg.RidgError) as e:
        s.forward(w.source_xyz, 0.0, 0.0, 1.0, w.receivers, w.t_final, wavelet=wav, wavelet_dt=0.0)
    assert e.value.code == -1


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_image_mask(dtype):
    """A solver restricted to one imaging condition accumulates that image unchanged and leaves the
    other at zero."""
    w = tiny_layered_rtm(N=3, t_final=0.004)
    args = (w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final)
    tr, ip, iq = _gpu(w, dtype).rtm_shot(*args)
    trp, ipp, iqp = _gpu(w, dtype, image_mask=ridg.IMAGE_P).rtm_shot(*args)
    trq, ipq, iqq = _gpu(w, dtype, image_mask=ridg.IMAGE_Q).rtm_shot(*args)
    assert np.array_equal(trp, tr) and np.array_equal(trq, tr)
    assert rel_l2(ipp, ip) < 1e-12 and np.all(iqp == 0)
    assert rel_l2(iqq, iq) < 1e-12 and np.all(ipq == 0)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_device_state_round_trip(dtype):
    """Fields set and read through device buffers are those of the host-buffer calls."""
    torch = pytest.importorskip("torch")
    w = tiny_layered_rtm(N=3)
    s = _gpu(w, dtype)
    q = random_state(w.K, s.Np, seed=31)
    s.set_state(q)
    s.step(2)
    q_host = s.get_state()
    qd = torch.tensor(q, dtype=torch.float64, device="cuda")
    s.set_state_device(qd)
    s.step(2)
    out = torch.zeros_like(qd)
    s.get_state_device(out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), q_host)
    assert np.array_equal(s.get_state(), q_host)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
def test_rhs_parity_fp32_cuda_cores(N):
    """FP32 with the element products as plain FMAs on CUDA cores (the reference the tensor-core
    split is measured against): right-hand side with every boundary condition."""
    w = tiny_layered_rtm(N=N)
    fb = mixed_bc(w)
    prob = _oracle_problem(w, face_bc=fb)
    s = _gpu(w, "f32", face_bc=fb, contraction=ridg.CONTRACT_CUDA_CORES)
    q = random_state(w.K, s.Np, seed=11)
    g = prob.geo
    r_ref = rhs(np.arange(g.K), q, traces(q, g), g)
    assert rel_l2(s.eval_rhs(q), r_ref) < TOL["f32"]


def test_rtm_shot_parity_fp32_cuda_cores():
    w, ref = _oracle_shot(4)
    s = _gpu(w, "f32", contraction=ridg.CONTRACT_CUDA_CORES)
    tr, ip, iq = s.rtm_shot(w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final, w.t_image_start)
    assert rel_l2(tr, ref.traces) < TOL["f32"]
    assert rel_l2(ip, ref.image_p) < TOL["f32"]
    assert rel_l2(iq, ref.image_q) < TOL["f32"]


def test_blow_up_is_reported_as_unstable():
    """A time step far beyond the AB3 stability bound (cfl = 3) makes the fields overflow; the shot
    reports RIDG_E_UNSTABLE instead of returning non-finite images."""
    w = tiny_layered_rtm(N=3, t_final=0.02)
    mesh = ridg.Mesh(w.xyz, w.tets, default_bc=w.default_bc)
    s = ridg.Solver(mesh, w.N, w.c, w.rho, dtype="f32", cfl=3.0, n_levels_max=w.n_levels_max)
    with pytest.raises(ridg.RidgError) as e:
        s.rtm_shot(w.source_xyz, w.f0, w.t_peak, 1e6, w.receivers, w.t_final)
    assert e.value.code == -5


# the BF16 hi + lo split keeps about 16 significand bits per product (2^-17 relative): its stated
# tolerance against the FP64 oracle is 1e-4
TOL_BF16 = 1e-4


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
def test_rhs_parity_bf16_split(N):
    """FP32 with the element products on tensor cores as a BF16 hi + lo split (m16n8k16): right-hand
    side with every boundary condition, several blocks and a ragged tail."""
    w = tiny_layered_rtm(N=N)
    fb = mixed_bc(w)
    prob = _oracle_problem(w, face_bc=fb)
    s = _gpu(w, "f32", face_bc=fb, contraction=ridg.CONTRACT_TENSOR_BF16)
    q = random_state(w.K, s.Np, seed=11)
    g = prob.geo
    r_ref = rhs(np.arange(g.K), q, traces(q, g), g)
    r = s.eval_rhs(q)
    assert rel_l2(r, r_ref) < TOL_BF16
    # the split is the only difference from the TF32 path: its error is above FP32 rounding
    assert rel_l2(r, r_ref) > 1e-7


def test_rtm_shot_parity_bf16_split():
    w, ref = _oracle_shot(4)
    s = _gpu(w, "f32", contraction=ridg.CONTRACT_TENSOR_BF16)
    tr, ip, iq = s.rtm_shot(w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final, w.t_image_start)
    assert rel_l2(tr, ref.traces) < TOL_BF16
    assert rel_l2(ip, ref.image_p) < TOL_BF16
    assert rel_l2(iq, ref.image_q) < TOL_BF16


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
def test_rhs_parity_fp16_split(N):
    """FP32 with the element products as an FP16 hi + lo split (m16n8k16), each column of each operand
    tile scaled by a power of two into FP16's range: right-hand side with every boundary condition,
    several blocks and a ragged tail, at the FP32 tolerance; the fields are scaled by 1e-12 as well,
    far below FP16's range, which only the column scales bring back."""
    w = tiny_layered_rtm(N=N)
    fb = mixed_bc(w)
    prob = _oracle_problem(w, face_bc=fb)
    s = _gpu(w, "f32", face_bc=fb, contraction=ridg.CONTRACT_TENSOR_FP16)
    g = prob.geo
    for scale in (1.0, 1e-12):
        q = scale * random_state(w.K, s.Np, seed=11)
        r_ref = rhs(np.arange(g.K), q, traces(q, g), g)
        assert rel_l2(s.eval_rhs(q), r_ref) < TOL["f32"]


def test_rtm_shot_parity_fp16_split():
    w, ref = _oracle_shot(4)
    s = _gpu(w, "f32", contraction=ridg.CONTRACT_TENSOR_FP16)
    tr, ip, iq = s.rtm_shot(w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final, w.t_image_start)
    assert rel_l2(tr, ref.traces) < TOL["f32"]
    assert rel_l2(ip, ref.image_p) < TOL["f32"]
    assert rel_l2(iq, ref.image_q) < TOL["f32"]


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
def test_rhs_parity_tf32_split_at_every_order(N):
    """The TF32 three-term split forced at every order (the default tensor-core mode runs it up to N = 4
    and the FP16 split from N = 5)."""
    w = tiny_layered_rtm(N=N)
    fb = mixed_bc(w)
    prob = _oracle_problem(w, face_bc=fb)
    s = _gpu(w, "f32", face_bc=fb, contraction=ridg.CONTRACT_TENSOR_TF32)
    q = random_state(w.K, s.Np, seed=11)
    g = prob.geo
    assert rel_l2(s.eval_rhs(q), rhs(np.arange(g.K), q, traces(q, g), g)) < TOL["f32"]
