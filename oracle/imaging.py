"""Imaging conditions and their AB3-exact time integration (oracle, test infrastructure).

Sec. 3.3 ("Evaluation of Imaging Condition"): over one local step of level l the fields
follow the Adams-Bashforth interpolant

    x(T + tau h) = x(T) + h sum_s A_s(tau) r^{(s)},   A_s(tau) = int_0^tau l_s,

with l_s the Lagrange polynomials on the nodes 0, -1, -2 (Eqs. ABrepS/ABrepR).  The
product of two such interpolants integrates exactly to (Eq. updateABcorr)

    h xS xR + h^2 sum_s c_s (xS rR_s + rS_s xR) + h^3 sum_{s1,s2} C_{s1 s2} rS_{s1} rR_{s2}

with c_s = int_0^1 A_s and C_ij = int_0^1 A_i A_j.  Readings: the paper prints a_s where
the h^2 weights must be c_s = (19/24, -5/12, 1/8) (needed for exactness already for
fields linear in time), pairs the terms as xS rR_s + rS_s xR, and its printed C equals
int_0^1 A_i A_j exactly; a factor h is dropped in Eqs. ABrepS/ABrepR.

Backward runs use h < 0, so the increment above is int_T^{T+h} = -int_{T+h}^T; the image
accumulates the negated increments so that it equals the forward-oriented integral.

The classical condition (Eq. imageP) correlates pressures; the characteristic condition
(Eqs. imageQ, charact) correlates q^-_S with q^+_R, q^{+/-} = p +/- c rho (e_up . v),
e_up the upward unit vector (the equation's pairing; z is depth, so e_up = (0,0,-1)).
"""

from __future__ import annotations

from fractions import Fraction

import numpy as np


def _poly_l(s):
    """Exact coefficients (ascending) of the Lagrange polynomial on nodes 0,-1,-2 that is 1 at -(s-1)."""
    nodes = [Fraction(0), Fraction(-1), Fraction(-2)]
    coeffs = [Fraction(1)]
    denom = Fraction(1)
    for j, xj in enumerate(nodes):
        if j == s - 1:
            continue
        new = [Fraction(0)] * (len(coeffs) + 1)
        for i, ci in enumerate(coeffs):
            new[i + 1] += ci
            new[i] -= xj * ci
        coeffs = new
        denom *= nodes[s - 1] - xj
    return [ci / denom for ci in coeffs]


def _integrate(coeffs):
    return [Fraction(0)] + [ci / (i + 1) for i, ci in enumerate(coeffs)]


def _mul(a, b):
    out = [Fraction(0)] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] += x * y
    return out


def _eval01(coeffs):
    return sum(coeffs, Fraction(0))


A_POLY = [_integrate(_poly_l(s)) for s in (1, 2, 3)]  # A_s(tau) as exact polynomials
C_VEC = tuple(_eval01(_integrate(A)) for A in A_POLY)
C_MAT = tuple(tuple(_eval01(_integrate(_mul(A_POLY[i], A_POLY[j]))) for j in range(3)) for i in range(3))


def step_increment(h, xS, rS, xR, rR):
    """Exact integral over [T, T+h] of the product of the two AB3 interpolants.

    xS, xR: values at T (any shape); rS, rR: sequences of the three right-hand sides
    r^{(1)}, r^{(2)}, r^{(3)} (at T, T-h, T-2h)."""
    c = [float(x) for x in C_VEC]
    C = [[float(x) for x in row] for row in C_MAT]
    out = h * xS * xR
    for s in range(3):
        out = out + h * h * c[s] * (xS * rR[s] + rS[s] * xR)
    for i in range(3):
        for j in range(3):
            out = out + h ** 3 * C[i][j] * rS[i] * rR[j]
    return out


def characteristic(p, v, Z, e_up, sign):
    """q^{+/-} = p +/- Z (e_up . v) for sign = +1 / -1 (Eq. charact); v [..., 3, Np], Z per element."""
    ev = np.einsum("d,...dn->...n", np.asarray(e_up, dtype=np.float64), v)
    return p + sign * Z[:, None] * ev
