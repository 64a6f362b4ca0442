"""Source signal and trace interpolation in time (oracle, test infrastructure).

* Ricker pulse (Sec. 5.1, Sec. 5.2): f(t) = A (1 - 2 pi^2 f0^2 tau^2) exp(-pi^2 f0^2 tau^2),
  tau = t - t_p (unit peak at t_p).
* Receiver traces are sampled at the global steps t_n = n Delta t_global.  When they are
  re-injected in the backward receiver run (Sec. 2), values between samples come from
  the cubic Lagrange interpolant on the four samples around t (samples outside the
  record count as zero).  Times are integers in units of Delta t_local, so the stencil
  is chosen with exact integer arithmetic.
* A source may also be given as samples s_n of its signal at t_n = n dt (any dt > 0, the
  first sample at t = 0): f(t) is then the same cubic Lagrange interpolant, on the samples
  floor(t/dt) - 1 .. floor(t/dt) + 2, again with missing samples counted as zero, times
  the amplitude.  The paper's sources are Ricker pulses; the sampled form is the reading
  used for a wavelet known only by its samples.
"""

from __future__ import annotations

import numpy as np


def ricker(t, f0, t_peak, amplitude=1.0):
    a = (np.pi * f0 * (np.asarray(t, dtype=np.float64) - t_peak)) ** 2
    return amplitude * (1.0 - 2.0 * a) * np.exp(-a)


def cubic_weights(tau: int, n_local: int):
    """Samples and weights for the value at integer fine time ``tau``: returns
    (n_lo - 1, [w_-1, w_0, w_1, w_2]) with the samples n_lo-1 .. n_lo+2."""
    n_lo = tau // n_local
    u = (tau - n_lo * n_local) / n_local
    xs = (-1.0, 0.0, 1.0, 2.0)
    w = []
    for i, xi in enumerate(xs):
        li = 1.0
        for j, xj in enumerate(xs):
            if j != i:
                li *= (u - xj) / (xi - xj)
        w.append(li)
    return n_lo - 1, w


def interpolate_trace(trace: np.ndarray, tau: int, n_local: int) -> float:
    n0, w = cubic_weights(tau, n_local)
    out = 0.0
    for i in range(4):
        n = n0 + i
        if 0 <= n < len(trace):
            out += w[i] * trace[n]
    return out


def lagrange4(x: float):
    """Weights of the cubic Lagrange interpolant on the nodes -1, 0, 1, 2 at x."""
    xs = (-1.0, 0.0, 1.0, 2.0)
    w = []
    for i, xi in enumerate(xs):
        li = 1.0
        for j, xj in enumerate(xs):
            if j != i:
                li *= (x - xj) / (xi - xj)
        w.append(li)
    return w


def sampled(t: float, samples, dt: float, amplitude=1.0) -> float:
    """Sampled source signal at time t (samples at t_n = n dt, zero outside)."""
    u = t / dt
    n_lo = int(np.floor(u))
    w = lagrange4(u - n_lo)
    out = 0.0
    for i in range(4):
        n = n_lo - 1 + i
        if 0 <= n < len(samples):
            out += w[i] * samples[n]
    return amplitude * out
