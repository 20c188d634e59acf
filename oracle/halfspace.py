"""Oracle: closed-form step-off dB_z/dt at the centre of a loop on a half-space.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Textbook result for a circular loop of radius a carrying I, switched off at
t = 0, on a homogeneous half-space of conductivity sigma, quasi-static, field
at the loop centre on the surface:
    dB_z/dt = -(I / (sigma a^3)) [3 erf(theta a)
                                   - 2/sqrt(pi) theta a (3 + 2 theta^2 a^2) exp(-theta^2 a^2)],
    theta = sqrt(mu0 sigma / (4 t)).
A square loop of half-side s is a sheet of vertical dipoles of unit moment
density; integrating the circular result over angle gives
    (4/pi) int_0^{pi/4} F(s / cos(phi), t) dphi
with F(a, t) the circular formula above.  This pins the sign and scale of the
whole chain (source, solve, residue sum, observation) against physics; it is
not a parity check (mesh and boundary truncation errors are present).
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

MU0 = 4e-7 * np.pi


def circular(a, t, sigma, current=1.0):
    th = np.sqrt(MU0 * sigma / (4.0 * t))
    x = th * a
    return -(current / (sigma * a ** 3)) * (
        3.0 * erf(x) - 2.0 / np.sqrt(np.pi) * x * (3.0 + 2.0 * x * x) * np.exp(-x * x))


def square(s, t, sigma, current=1.0, n_quad=64):
    xg, wg = np.polynomial.legendre.leggauss(n_quad)
    phi = (xg + 1.0) * (np.pi / 8.0)
    w = wg * (np.pi / 8.0)
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    out = np.array([np.sum(w * circular(s / np.cos(phi), tt, sigma, current)) for tt in t])
    return 4.0 / np.pi * out
