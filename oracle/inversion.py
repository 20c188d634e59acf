"""Oracle: RT0 smoothness regulariser and LSQR (Section 3.2, Section 3.3).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Regulariser (Section 3.2): R(m) = 1/2 (m - m_ref)^T L (m - m_ref), L = D M_div^-1 D^T,
with D the cell-face divergence of unit-flux RT0 face functions and M_div
lumped.  Reading: the lumped RT0 mass of face f between earth cells a and b
is d_f/|f| (d_f = distance between the cell centroids, |f| = face area), so
L is the two-point-flux Laplacian; faces touching air or the outer boundary
carry no flux (Neumann).  This L is singular (constants), so instead of a
Cholesky factor the rectangular root W = M_div^-1/2 D^T is used: W^T W = L
exactly, and ||sqrt(lambda) W dm|| gives the same least-squares term as
sqrt(lambda) L^1/2 dm in eq. (lsqr).

LSQR (Section 3.3, Paige & Saunders 1982): Golub-Kahan bidiagonalisation of the
operator A = [W_d J; sqrt(lambda) W] with right-hand side
b = -[W_d (d - d_obs); sqrt(lambda) W (m - m_ref)], run for a fixed number of
iterations with no stopping test.  One iteration applies A once and A^T once.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def regulariser(xyz, tets, is_param):
    """W = M_div^-1/2 D^T as a sparse [n_faces, P] matrix over the earth cells."""
    tv = np.sort(np.asarray(tets, dtype=np.int64), axis=1)
    param = np.asarray(is_param).astype(bool)
    pidx = -np.ones(tv.shape[0], dtype=np.int64)
    pidx[param] = np.arange(int(param.sum()))
    faces = []
    owners = []
    for (a, b, c) in ((0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)):
        faces.append(tv[:, [a, b, c]])
        owners.append(np.arange(tv.shape[0]))
    faces = np.concatenate(faces)
    owners = np.concatenate(owners)
    uf, inv, cnt = np.unique(faces, axis=0, return_inverse=True, return_counts=True)
    inv = inv.ravel()
    order = np.argsort(inv, kind="stable")
    inv_s, own_s = inv[order], owners[order]
    first = np.searchsorted(inv_s, np.arange(len(uf)))
    interior = cnt == 2
    fa = own_s[first[interior]]
    fb = own_s[first[interior] + 1]
    keep = param[fa] & param[fb]
    fa, fb = fa[keep], fb[keep]
    fv = uf[interior][keep]
    X = np.asarray(xyz, dtype=np.float64)
    cen = X[tv].mean(axis=1)
    dist = np.linalg.norm(cen[fa] - cen[fb], axis=1)
    p0, p1, p2 = X[fv[:, 0]], X[fv[:, 1]], X[fv[:, 2]]
    area = 0.5 * np.linalg.norm(np.cross(p1 - p0, p2 - p0), axis=1)
    wgt = np.sqrt(area / dist)
    nf = len(fa)
    rows = np.concatenate([np.arange(nf), np.arange(nf)])
    cols = np.concatenate([pidx[fa], pidx[fb]])
    vals = np.concatenate([wgt, -wgt])
    return sp.csr_matrix((vals, (rows, cols)), shape=(nf, int(param.sum())))


def lsqr(matvec, rmatvec, b, n_iter):
    """Paige-Saunders LSQR for min ||A x - b||, x0 = 0, exactly n_iter steps.
    Returns x and the list of iterates."""
    b = np.asarray(b, dtype=np.float64)
    beta = np.linalg.norm(b)
    u = b / beta
    v = rmatvec(u)
    alpha = np.linalg.norm(v)
    v = v / alpha
    w = v.copy()
    x = np.zeros_like(v)
    phibar, rhobar = beta, alpha
    iterates = []
    for _ in range(n_iter):
        u = matvec(v) - alpha * u
        beta = np.linalg.norm(u)
        if beta > 0:
            u = u / beta
        v = rmatvec(u) - beta * v
        alpha = np.linalg.norm(v)
        if alpha > 0:
            v = v / alpha
        rho = np.hypot(rhobar, beta)
        c, s = rhobar / rho, beta / rho
        theta = s * alpha
        rhobar = -c * alpha
        phi = c * phibar
        phibar = s * phibar
        x = x + (phi / rho) * w
        w = v - (theta / rho) * w
        iterates.append(x.copy())
    return x, iterates


def gn_operator(oracle, W, wd, lam):
    """matvec / rmatvec of A = [W_d J; sqrt(lam) W] with data flattened x-r-j."""
    shape = oracle.forward_shape
    nd = int(np.prod(shape))
    sl = np.sqrt(lam)

    def matvec(v):
        return np.concatenate([wd * oracle.jvp(v).ravel(), sl * (W @ v)])

    def rmatvec(u):
        return oracle.jtvp((wd * u[:nd]).reshape(shape)) + sl * (W.T @ u[nd:])

    return matvec, rmatvec


def gn_rhs(d, d_obs, wd, W, m, m_ref, lam):
    return -np.concatenate([wd * (d - d_obs).ravel(), np.sqrt(lam) * (W @ (m - m_ref))])


def noise_weights(d_obs, eps_r=0.03, eps_a_frac=1e-4):
    """W_d = diag(1/sigma(d)), sigma(d) = |d| eps_r + eps_a (Section 4.2 error model);
    eps_a = eps_a_frac * max|d_obs| per transmitter (reading: the paper prints no
    values)."""
    d_obs = np.asarray(d_obs)
    eps_a = eps_a_frac * np.abs(d_obs).reshape(d_obs.shape[0], -1).max(axis=1)
    sd = np.abs(d_obs) * eps_r + eps_a[:, None, None]
    return 1.0 / sd
