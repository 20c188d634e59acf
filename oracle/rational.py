"""Oracle: shared-pole rational approximation of exp(-t z) (Section 2.3).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper approximates exp(-t_j M^-1 K) b by r_j(M^-1 K) b with
    r_j(z) = 2 Re sum_{i=1}^m alpha_i^[j] / (z - xi_i),
poles xi_i shared by every time t_j and coefficients alpha_i^[j] per time, and
obtains them with RKFIT.  The poles the paper used are not printed, so they
are fitted here once on the host in FP64: the poles by variable projection
(for fixed poles the alpha are a linear least-squares problem; the poles then
minimise the stacked residual over a grid of times), the coefficients for the
requested observation times by linear least squares with the poles fixed.
Both least-squares problems carry a small Tikhonov term mu * alpha_i/|xi_i|:
max_z |alpha_i/(z - xi_i)| = |alpha_i|/|xi_i| for Re xi_i < 0, so the term bounds
the size of the individual partial fractions.  Without it the fit drifts to
nearly coincident poles with huge opposite residues, and the residue sum of
the response then cancels by ten orders of magnitude in FP64.
Each xi_i stands for the conjugate pair {xi_i, conj(xi_i)}; Re xi_i < 0 keeps
every pole off the non-negative real axis, where the spectrum of M^-1 K lies.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import least_squares


def sample_points(n=2200, zmin=1e-2, zmax=1e9):
    return np.concatenate([[0.0], np.logspace(np.log10(zmin), np.log10(zmax), n)])


def check_points(n=20000, zmin=1e-3, zmax=1e11):
    return np.concatenate([[0.0], np.logspace(np.log10(zmin), np.log10(zmax), n)])


def basis(z, xi):
    """Real basis of 2 Re sum_i alpha_i/(z - xi_i) in (Re alpha, Im alpha)."""
    c = 1.0 / (np.asarray(z, dtype=np.float64)[:, None] - np.asarray(xi)[None, :])
    return np.hstack([2.0 * c.real, -2.0 * c.imag])


def evaluate(z, xi, alpha):
    """r(z) = 2 Re sum_i alpha_i / (z - xi_i) for one coefficient vector."""
    c = 1.0 / (np.asarray(z, dtype=np.float64)[:, None] - np.asarray(xi)[None, :])
    return 2.0 * np.real(c @ np.asarray(alpha))


MU = 1e-4


def _augmented(z, xi, E, mu):
    B = basis(z, xi)
    sc = np.concatenate([np.abs(xi), np.abs(xi)])
    Ba = np.vstack([B, mu * np.diag(1.0 / sc)])
    Ea = np.vstack([E, np.zeros((B.shape[1], E.shape[1]))])
    return Ba, Ea


def fit_alpha(xi, times, z=None, mu=MU):
    """alpha[i][j] by (penalised) linear least squares of r_j to exp(-t_j z) on z."""
    z = sample_points() if z is None else z
    m = len(xi)
    E = np.exp(-np.outer(z, times))                       # [Z, K]
    Ba, Ea = _augmented(z, xi, E, mu)
    coef, *_ = np.linalg.lstsq(Ba, Ea, rcond=None)        # [2m, K]
    return coef[:m] + 1j * coef[m:]


def _xi_of(p, m):
    return -np.exp(p[:m]) + 1j * np.exp(p[m:])


def seed_poles(m, t0=1e-5, t1=1e-2, seed_angle=0.7):
    """Starting poles of the fit: moduli log-spaced over [0.3 / t1, 30 / t0]
    (the decay rates the time range resolves) at the angle seed_angle * pi
    from the positive real axis (Re < 0 < Im)."""
    rho = np.logspace(np.log10(0.3 / t1), np.log10(30.0 / t0), m)
    th = np.pi * seed_angle
    return rho * np.cos(th) + 1j * rho * np.sin(th)


def vp_objective(xi, times, z=None, mu=MU):
    """Variable-projection objective of a pole set: sum over the times of the
    squared residual of the penalised least-squares residue fit."""
    z = sample_points() if z is None else z
    Ba, Ea = _augmented(z, xi, np.exp(-np.outer(z, times)), mu)
    coef, *_ = np.linalg.lstsq(Ba, Ea, rcond=None)
    return float(np.sum((Ba @ coef - Ea) ** 2))


def fit_poles(m, t0=1e-5, t1=1e-2, n_times=40, seed_angle=0.7, max_nfev=300, mu=MU):
    """Shared poles for t in [t0, t1] by variable projection."""
    z = sample_points()
    ts = np.logspace(np.log10(t0), np.log10(t1), n_times)
    E = np.exp(-np.outer(z, ts))

    def resid(p):
        Ba, Ea = _augmented(z, _xi_of(p, m), E, mu)
        coef, *_ = np.linalg.lstsq(Ba, Ea, rcond=None)
        return (Ba @ coef - Ea).ravel()

    x0 = seed_poles(m, t0, t1, seed_angle)
    p0 = np.concatenate([np.log(-x0.real), np.log(x0.imag)])
    sol = least_squares(resid, p0, method="trf", max_nfev=max_nfev, x_scale=1.0)
    xi = _xi_of(sol.x, m)
    return xi[np.argsort(np.abs(xi))]


def cancellation(xi, alpha, z=None):
    """max_j max_z sum_i |2 alpha_ij/(z - xi_i)|: size of the largest partial
    fraction sum relative to exp's bound of 1."""
    z = check_points() if z is None else z
    c = np.abs(1.0 / (z[:, None] - np.asarray(xi)[None, :]))
    return float(np.max(2.0 * (c @ np.abs(alpha))))


def max_error(xi, alpha, times, z=None):
    """eps_j = max_z |exp(-t_j z) - r_j(z)| on the check grid."""
    z = check_points() if z is None else z
    eps = []
    for j, t in enumerate(times):
        eps.append(np.max(np.abs(np.exp(-t * z) - evaluate(z, xi, alpha[:, j]))))
    return np.array(eps)
