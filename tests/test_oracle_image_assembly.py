"""Image assembly of the oracle's RTM shot, pinned by an independent time quadrature.

Eq. imageP and Eq. imageQ define the images as time integrals over [t_i, t_f] of products of the
backward source and receiver fields; the oracle's shot accumulates them step by step with the
AB3-exact increment of Eq. updateABcorr, evaluated from the fields and histories before each
update, over the window tau > tau_i, with the sign of a backward sweep, and with q^-_S paired with
q^+_R.  Here the backward fields are taken from the shot itself at every step of each element's
level (the shot's test hook), and the images are integrated again with composite Simpson on those
step values, without the increment formula.  Both converge to the same integral; their difference
shrinks at third order in the time step (the AB3 interpolant between steps against a quadrature
of the step values).  Each of these mistakes breaks that: imaging after the update or with the
previous step's receiver history (first order), a window one step off, the wrong sign, or S and R
exchanged in the characteristic image (O(1))."""

import numpy as np

from oracle.rtm import make_problem, rtm_shot
from synth import HexGrid, adjoint_box_three_level

E_UP = np.array([0.0, 0.0, -1.0])


def simpson(f, h):
    """Composite Simpson along axis 0 of equally spaced samples f (an odd tail takes the 3/8 rule)."""
    n = f.shape[0] - 1
    if n == 0:
        return np.zeros(f.shape[1:])
    if n % 2 == 0:
        return h / 3.0 * (f[0] + f[-1] + 4.0 * f[1:-1:2].sum(axis=0) + 2.0 * f[2:-1:2].sum(axis=0))
    if n == 1:
        return 0.5 * h * (f[0] + f[1])
    return simpson(f[:-3], h) + 3.0 * h / 8.0 * (f[-4] + 3.0 * f[-3] + 3.0 * f[-2] + f[-1])


def uniform_box(N, cfl):
    """200 x 200 x 100 m, 2 x 2 x 1 hexahedra x 6 = 24 tetrahedra, c = 1500 m/s: one rate level."""
    g = HexGrid(np.linspace(0.0, 200.0, 3), np.linspace(0.0, 200.0, 3), np.linspace(0.0, 100.0, 2))
    xyz, tets = g.mesh()
    K = tets.shape[0]
    return make_problem(xyz, tets, np.full(K, 1500.0), np.full(K, 1000.0), N, default_bc=2, cfl=cfl,
                        n_levels_max=1)


def quadrature_images(prob, res, obs, t_i, e_up=E_UP, swap=False):
    """I_P = int p_S p_R dt and I_Q = int q^-_S q^+_R dt over [t_i, t_f] by Simpson, per element on
    the step times of its own level (multiples of its stride in units of Delta t_local).  With
    ``swap`` the two wavefields exchange roles."""
    nl, dtl = prob.n_local, prob.dt_local
    tau_f = res.n_global * nl
    tau_i = int(np.floor(t_i / prob.dt_global + 1e-9)) * nl
    Z = prob.geo.Z
    I_p = np.zeros_like(res.image_p)
    I_q = np.zeros_like(res.image_q)
    for l in range(1, prob.n_levels + 1):
        E = np.nonzero(prob.levels == l)[0]
        d = 2 ** (prob.n_levels - l)
        taus = range(tau_i, tau_f + 1, d)
        S = np.array([obs[t][1 if swap else 0][E] for t in taus])
        R = np.array([obs[t][0 if swap else 1][E] for t in taus])
        up_S = np.einsum("d,tkdn->tkn", e_up, S[:, :, 1:4])
        up_R = np.einsum("d,tkdn->tkn", e_up, R[:, :, 1:4])
        q_minus_S = S[:, :, 0] - Z[E][None, :, None] * up_S
        q_plus_R = R[:, :, 0] + Z[E][None, :, None] * up_R
        I_p[E] = simpson(S[:, :, 0] * R[:, :, 0], d * dtl)
        I_q[E] = simpson(q_minus_S * q_plus_R, d * dtl)
    return I_p, I_q


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def shot_and_quadrature(prob, source, f0, t_peak, rec, t_final, t_i, swap=False):
    obs = {}
    res = rtm_shot(prob, source, f0, t_peak, 1.0, rec, t_final, t_i,
                   observe=lambda tau, qs, qr: obs.__setitem__(tau, (qs, qr)))
    return res, quadrature_images(prob, res, obs, t_i, swap=swap), obs


REC = np.array([[50.0, 100.0, 10.0], [150.0, 100.0, 10.0], [100.0, 60.0, 20.0]])
F0 = 50.0
T_PEAK = 0.1127 * 12.0 / F0


def test_single_rate_images_converge_at_third_order_to_the_quadrature():
    """One rate level, the whole window and one starting half-way: the shot's images against
    Simpson on the step values, at two time steps (C = 0.15, 0.075)."""
    for t_i in (0.0, 0.025):
        errs = []
        for cfl in (0.15, 0.075):
            prob = uniform_box(2, cfl)
            res, (qp, qq), _ = shot_and_quadrature(prob, (100.0, 100.0, 30.0), F0, T_PEAK, REC, 0.05, t_i)
            assert np.abs(qp).max() > 0 and np.abs(qq).max() > 0
            errs.append((rel(res.image_p, qp), rel(res.image_q, qq)))
        (ep1, eq1), (ep2, eq2) = errs
        assert ep1 < 2e-3 and eq1 < 2e-3
        assert ep2 < 2.5e-4 and eq2 < 2.5e-4
        # third order: halving the step divides the difference by about 8 (a first-order mistake by 2)
        assert ep1 / ep2 > 6.0 and eq1 / eq2 > 6.0


def test_characteristic_image_pairs_q_minus_of_the_source_with_q_plus_of_the_receivers():
    """Exchanging the roles of the two wavefields leaves the classical image unchanged and changes
    the characteristic one at O(1): the shot's I_Q is the integral of q^-_S q^+_R (Eq. imageQ)."""
    prob = uniform_box(2, 0.075)
    obs = {}
    res = rtm_shot(prob, (100.0, 100.0, 30.0), F0, T_PEAK, 1.0, REC, 0.05, 0.0,
                   observe=lambda tau, qs, qr: obs.__setitem__(tau, (qs, qr)))
    qp, qq = quadrature_images(prob, res, obs, 0.0)
    sp, sq = quadrature_images(prob, res, obs, 0.0, swap=True)
    assert rel(sp, qp) < 1e-14
    assert rel(sq, qq) > 0.5
    assert rel(res.image_q, qq) < 2.5e-4 and rel(res.image_q, sq) > 0.5


def test_multi_rate_images_converge_at_third_order_to_the_quadrature():
    """Three rate levels (the 24-element box with three velocity zones, 10 + 8 + 6 elements): every
    element is imaged at the steps of its own level, coarse elements with their long steps."""
    w = adjoint_box_three_level()
    errs = []
    for cfl in (0.15, 0.075):
        prob = make_problem(w.xyz, w.tets, w.c, w.rho, 1, default_bc=w.default_bc, cfl=cfl, n_levels_max=3)
        assert prob.n_levels == 3 and np.all(np.bincount(prob.levels)[1:] > 0)
        res, (qp, qq), _ = shot_and_quadrature(prob, w.source_xyz, w.f0, w.t_peak, w.receivers, 0.06, 0.0)
        errs.append((rel(res.image_p, qp), rel(res.image_q, qq)))
    (ep1, eq1), (ep2, eq2) = errs
    assert ep1 < 4e-3 and eq1 < 4e-3
    assert ep1 / ep2 > 6.0 and eq1 / eq2 > 6.0
