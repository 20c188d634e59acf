"""Gauss-Newton inversion on the library's calls (Section 3.3).

Each iteration at the model m:
  1. factor the shifted matrices at m and form the data (tem_factor, tem_forward);
  2. the GN direction dm from LSQR on eq. (lsqr) (tem_lsqr, n_lsqr iterations);
  3. the objective phi(m) and its gradient's projection grad . dm (tem_gn_eval);
  4. backtracking line search from eta = 1: the trial m + eta dm (tem_model_step)
     is factored and evaluated until the Armijo condition
       phi(m + eta dm) <= phi(m) + c1 eta grad . dm,   c1 = 1e-4,
     holds; eta is halved, or set to the minimiser of the quadratic model of phi
     along dm through phi(m), grad . dm and phi(m + eta dm) when that lies in
     [eta_min, eta / 2] (the heuristic of Section 3.3), and never goes below the
     lower bound eta_min (at eta_min the step is taken: the safeguard);
  5. lambda cooling: once phi stops decreasing for the current lambda (relative
     decrease below conv_tol) and the data misfit chi^2 = ||W_d r||^2 / n_data is
     not yet ~1, lambda is halved.
The accepted trial is already factored, so the next iteration starts at step 2.
The state (model, lambda, iteration count, history) is written to a
checkpoint after every iteration and a run can resume from it.
"""
from __future__ import annotations

import json

import numpy as np

from . import tem


class GaussNewton:
    def __init__(self, model, d_obs, wd, m_ref, m0, lam=10.0, n_lsqr=30, c1=1e-4, eta_min=1.0 / 16,
                 cool=0.5, conv_tol=0.05, chi2_target=1.0, checkpoint=None):
        import torch
        self.torch = torch
        self.model = model
        self.d_obs, self.wd, self.m_ref = d_obs.contiguous(), wd.contiguous(), m_ref.contiguous()
        self.m = m0.detach().clone().contiguous()
        self.lam = float(lam)
        self.n_lsqr, self.c1, self.eta_min = int(n_lsqr), float(c1), float(eta_min)
        self.cool, self.conv_tol, self.chi2_target = float(cool), float(conv_tol), float(chi2_target)
        self.checkpoint = checkpoint
        self.it = 0
        self.history = []
        self._at_m = False          # the context holds factors and data at self.m
        self._grad = torch.empty_like(self.m)
        self._trial = torch.empty_like(self.m)

    # -- state ------------------------------------------------------------------
    def save(self, path=None):
        path = path or self.checkpoint
        if path is None:
            return
        np.savez(path, m=self.m.cpu().numpy(), lam=self.lam, it=self.it,
                 history=json.dumps(self.history))

    @classmethod
    def resume(cls, path, model, d_obs, wd, m_ref, **kw):
        import torch
        z = np.load(path, allow_pickle=False)
        gn = cls(model, d_obs, wd, m_ref, torch.as_tensor(z["m"], device=d_obs.device), lam=float(z["lam"]),
                 checkpoint=path, **kw)
        gn.it = int(z["it"])
        gn.history = json.loads(str(z["history"]))
        return gn

    def converged(self):
        return bool(self.history) and self.history[-1]["chi2"] <= 1.05 * self.chi2_target

    # -- one iteration --------------------------------------------------------------
    def _eval(self, dm=None):
        g = self._grad if dm is not None else None
        return tem.tem_gn_eval(self.model.ctx, self.d_obs, self.wd, self.m_ref, self.lam, dm, g)

    def step(self):
        mdl = self.model
        if not self._at_m:
            mdl.factor(self.m)
            mdl.forward()
        dm = mdl.lsqr(self.d_obs, self.wd, self.m_ref, self.lam, self.n_lsqr)
        phi0, _, _, chi2_0, gd = self._eval(dm)
        eta, trials, margins = 1.0, 0, []
        while True:
            tem.tem_model_step(mdl.ctx, self.m, dm, eta, self._trial)
            mdl.factor(self._trial)
            mdl.forward()
            trials += 1
            phi_t, _, reg_t, chi2_t, _ = self._eval()
            bound = phi0 + self.c1 * eta * gd
            margins.append((phi_t - bound) / abs(bound))   # > 0: Armijo fails
            if phi_t <= bound or eta <= self.eta_min:
                break
            a = (phi_t - phi0 - gd * eta) / (eta * eta)   # quadratic model phi0 + gd e + a e^2
            nxt = eta / 2
            if a > 0:
                eq = -gd / (2 * a)
                if self.eta_min <= eq <= eta / 2:
                    nxt = eq
            eta = max(nxt, self.eta_min)
        self.m, self._trial = self._trial, self.m
        self._at_m = True
        rec = {"it": self.it, "lam": self.lam, "phi0": phi0, "phi": phi_t, "chi2_0": chi2_0, "chi2": chi2_t,
               "eta": eta, "trials": trials, "grad_dm": gd, "margins": margins}
        if (phi0 - phi_t) < self.conv_tol * phi0 and chi2_t > 1.05 * self.chi2_target:
            self.lam *= self.cool
            rec["cooled"] = True
        self.history.append(rec)
        self.it += 1
        self.save()
        return rec

    def run(self, n_iter):
        for _ in range(int(n_iter)):
            if self.converged():
                break
            self.step()
        return self.history
