"""Oracle: shifted solves, residue sums and the implicit Jacobian products.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Definitions followed (paper sections):
  Section 2.3:   u(t_j) ~ 2 Re sum_i alpha_i^[j] (K - xi_i M)^-1 f
  Section 3, data equation:   d_j = Q u(t_j), stacked per channel
  Section 3.1:   g_i = A_i^-1 f, A_i = K - xi_i M(m),  dA_i/dm = -xi_i dM/dm
                 J_j v = 2 Re sum_i alpha_i^[j] xi_i Q A_i^-1 [(dM/dm) g_i v]
                 J^T w = sum_j J_j^T w_j
                       = 2 Re sum_i xi_i [(dM/dm) g_i]^T A_i^-1 Q^T (sum_j alpha_i^[j] w_j)
Readings: m = ln(sigma) on the earth cells, so dM/dm_e = sigma_e M1_e (the
chain-rule factor of the log parametrisation); A_i is complex symmetric
(A^T = A, no conjugation), so A_i^-T = A_i^-1 and the same factors serve both
products.  The solve step is the oracle's own plain sparse LDL^T (ldlt.c)
under a coordinate-bisection ordering; the poles are independent, so they are
factored and solved on separate host threads (results combined in pole order).

Array layouts match the GPU library: data d[x][r][j] (transmitter, receiver,
time), model vectors over the earth cells in tet order.
"""
from __future__ import annotations

import os

import numpy as np
import scipy.sparse as sp
from concurrent.futures import ThreadPoolExecutor

from .fem import FEModel
from .sparse_ldlt import LDLT, nested_dissection
from .survey import loop_source, observation_operator


class Oracle:
    def __init__(self, xyz, tets, sigma, is_param, loops, rx, xi, alpha, threads=None):
        self.fe = FEModel(xyz, tets)
        fe = self.fe
        self.sigma_fixed = np.asarray(sigma, dtype=np.float64).copy()
        self.param = np.asarray(is_param).astype(bool)
        self.pidx = np.nonzero(self.param)[0]
        self.F = np.stack([loop_source(fe, lp) for lp in loops], axis=1)   # [N, n_x]
        self.Q = observation_operator(fe, rx)                               # [n_r, N]
        self.xi = np.asarray(xi, dtype=np.complex128)                       # [m]
        self.alpha = np.asarray(alpha, dtype=np.complex128)                 # [m, K]
        T = fe.tdof.shape[0]
        # scatter operator from element-local values [T, 6] to unknowns
        mask = fe.tdof >= 0
        cols = np.arange(T * 6).reshape(T, 6)[mask]
        self.S = sp.csr_matrix((np.ones(cols.size), (fe.tdof[mask], cols)), shape=(fe.N, T * 6))
        self.lu = None
        cent = fe.xyz[fe.tv].mean(axis=1)
        self.perm = nested_dissection(fe.tdof, fe.N, cent)
        self.threads = threads if threads else min(len(self.xi), os.cpu_count() or 1)

    @property
    def forward_shape(self):
        return (self.F.shape[1], self.Q.shape[0], self.alpha.shape[1])

    # -- model ---------------------------------------------------------------
    def set_model(self, log_sigma):
        """Factor every shifted matrix A_i = K - xi_i M(sigma) and solve A_i g_i = f."""
        s = self.sigma_fixed.copy()
        s[self.pidx] = np.exp(np.asarray(log_sigma, dtype=np.float64))
        self.sigma = s
        M = self.fe.mass(s)
        self.M = M

        def one(x):
            lu = LDLT((self.fe.K - x * M).astype(np.complex128), self.perm)
            return lu, lu.solve(self.F.astype(np.complex128))           # [N, n_x]

        with ThreadPoolExecutor(self.threads) as ex:
            res = list(ex.map(one, self.xi))
        self.lu = [r[0] for r in res]
        self.g = [r[1] for r in res]
        return self

    def shifted_matrix(self, i):
        return (self.fe.K - self.xi[i] * self.M).tocsr()

    # -- helpers ---------------------------------------------------------------
    def _local(self, u):
        """Gather unknown vectors [N, n] into element-local [T, 6, n] (0 on PEC)."""
        td = self.fe.tdof
        out = np.where((td >= 0)[:, :, None], u[np.maximum(td, 0)], 0.0)
        return out

    def _residue_sum(self, y):
        """y: list over poles of [n_r, n_x] complex -> d[x][r][j] = 2 Re sum_i alpha_ij y_i."""
        Y = np.stack(y, axis=0)                                    # [m, n_r, n_x]
        d = 2.0 * np.real(np.einsum("ij,irx->xrj", self.alpha, Y))
        return d

    # -- products -----------------------------------------------------------------
    def forward(self):
        """Predicted data d[x][r][j] (Algorithm 1 followed by the observation Q)."""
        return self._residue_sum([self.Q @ g for g in self.g])

    def dM_apply(self, i, v):
        """xi_i (dM/dm) g_i v: element-local sigma_e v_e M1_e (P_e g_i), assembled."""
        fe = self.fe
        ve = np.zeros(fe.tdof.shape[0])
        ve[self.pidx] = np.asarray(v, dtype=np.float64)
        gl = self._local(self.g[i])                                # [T, 6, n_x]
        loc = np.einsum("tab,tbx->tax", fe.Me1, gl) * (ve * self.sigma)[:, None, None]
        return self.xi[i] * (self.S @ loc.reshape(-1, gl.shape[2]))

    def _per_pole(self, fn):
        """fn(i) for every pole on the host threads, results in pole order (the
        poles are independent; the solves release the GIL)."""
        with ThreadPoolExecutor(self.threads) as ex:
            return list(ex.map(fn, range(len(self.lu))))

    def jvp(self, v):
        """J v -> [n_x][n_r][K]."""
        def one(i):
            return self.Q @ self.lu[i].solve(self.dM_apply(i, v))
        return self._residue_sum(self._per_pole(one))

    def jtvp(self, w):
        """J^T w, w[x][r][j] -> [P]."""
        w = np.asarray(w, dtype=np.float64)
        fe = self.fe

        def one(i):
            what = np.einsum("j,xrj->rx", self.alpha[i], w)          # [n_r, n_x] complex
            z = self.lu[i].solve((self.Q.T @ what).astype(np.complex128))     # [N, n_x]
            zl = self._local(z)
            gl = self._local(self.g[i])
            b = np.einsum("tax,tab,tbx->t", zl, fe.Me1, gl)
            return 2.0 * np.real(self.xi[i] * b) * self.sigma

        grad = np.zeros(fe.tdof.shape[0])
        for part in self._per_pole(one):   # summed in pole order
            grad += part
        return grad[self.pidx]

    def residual_norms(self, i, X, B):
        """||A_i X - B|| / ||B|| per column, with the oracle's own A_i (FP64 SpMV)."""
        R = self.shifted_matrix(i) @ X - B
        return np.linalg.norm(R, axis=0) / np.maximum(np.linalg.norm(B, axis=0), 1e-300)
