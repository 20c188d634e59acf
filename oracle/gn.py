"""Oracle: the Gauss-Newton iteration of Section 3.3, on the oracle's own products.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

phi(m) = 1/2 ||W_d (d(m) - d_obs)||^2 + lambda/2 ||W (m - m_ref)||^2  (W^T W = L)
grad phi = J^T W_d^2 (d - d_obs) + lambda W^T W (m - m_ref)
dm: LSQR on eq. (lsqr) for a fixed number of iterations.
Line search: eta = 1, then halving (or the minimiser of the quadratic through
phi(m), grad . dm, phi(m + eta dm) when it lies in [eta_min, eta/2]) until
Armijo with c1 holds, never below eta_min (taken there).  lambda halves when
the relative decrease of phi falls below conv_tol while chi^2 > 1.05; the
iteration stops once chi^2 <= 1.05.
"""
from __future__ import annotations

import numpy as np

from .inversion import gn_operator, gn_rhs, lsqr


def _phi(o, W, d_obs, wd, m, m_ref, lam):
    d = o.forward()
    r = wd * (d - d_obs).ravel()
    reg = 0.5 * float(np.sum((W @ (m - m_ref)) ** 2))
    return 0.5 * float(r @ r) + lam * reg, float(r @ r) / r.size, d


def gauss_newton(o, W, d_obs, wd, m_ref, m0, lam, n_lsqr, n_iter, c1=1e-4, eta_min=1.0 / 16,
                 cool=0.5, conv_tol=0.05):
    wd = np.asarray(wd).ravel()
    m = np.array(m0, dtype=np.float64)
    hist = []
    o.set_model(m)
    for it in range(n_iter):
        phi0, chi2_0, d = _phi(o, W, d_obs, wd, m, m_ref, lam)
        r = wd * (d - d_obs).ravel()
        grad = o.jtvp((wd * r).reshape(d.shape)) + lam * (W.T @ (W @ (m - m_ref)))
        mv, rmv = gn_operator(o, W, wd, lam)
        dm = lsqr(mv, rmv, gn_rhs(d, d_obs, wd, W, m, m_ref, lam), n_lsqr)[0]
        gd = float(grad @ dm)
        eta, trials, margins = 1.0, 0, []
        while True:
            mt = m + eta * dm
            o.set_model(mt)
            trials += 1
            phi_t, chi2_t, _ = _phi(o, W, d_obs, wd, mt, m_ref, lam)
            bound = phi0 + c1 * eta * gd
            margins.append((phi_t - bound) / abs(bound))   # > 0: Armijo fails
            if phi_t <= bound or eta <= eta_min:
                break
            a = (phi_t - phi0 - gd * eta) / (eta * eta)
            nxt = eta / 2
            if a > 0 and eta_min <= -gd / (2 * a) <= eta / 2:
                nxt = -gd / (2 * a)
            eta = max(nxt, eta_min)
        m = mt
        rec = {"it": it, "lam": lam, "phi0": phi0, "phi": phi_t, "chi2": chi2_t, "eta": eta, "trials": trials,
               "margins": margins}
        if (phi0 - phi_t) < conv_tol * phi0 and chi2_t > 1.05:
            lam *= cool
        hist.append(rec)
        if chi2_t <= 1.05:   # the data are fitted within their errors (chi^2 ~ 1): stop
            break
    return m, hist
