"""Oracle: lowest-order Nedelec (Whitney) edge elements on tetrahedra.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Section 2.2 of the paper: the curl-curl operator gives the stiffness matrix K and the
conductivity-weighted L2 product gives the mass matrix M(sigma); the outer
boundary carries the PEC condition n x e = 0 (Section 2.1, boundary condition),
so edge unknowns lying on the outer boundary are removed.

Whitney basis of the edge (a, b) of a tetrahedron with barycentric coordinates
lambda:  N_ab = lambda_a grad(lambda_b) - lambda_b grad(lambda_a),
curl N_ab = 2 grad(lambda_a) x grad(lambda_b).
Element matrices (exact, from int_T lambda_a lambda_c = |T|(1 + delta_ac)/20):
  K_e[i, j] = |T| / mu0 * curl N_i . curl N_j
  M1_e[i, j] = int_T N_i . N_j            (unit conductivity)
Global edge orientation: from the lower to the higher vertex index.  With the
vertices of each tetrahedron sorted ascending, every local edge (a < b) is
oriented like its global edge.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

MU0 = 4e-7 * np.pi
LOCAL_EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))


def barycentric_gradients(X):
    """X: [T, 4, 3] vertex coordinates -> grad lambda [T, 4, 3], volume [T]."""
    B = X[:, 1:, :] - X[:, :1, :]                     # rows x_k - x_0
    det = np.linalg.det(B)
    Binv = np.linalg.inv(B)                            # grad lambda_k = column k of B^-1
    g = np.empty((X.shape[0], 4, 3))
    g[:, 1:, :] = np.transpose(Binv, (0, 2, 1))
    g[:, 0, :] = -g[:, 1:, :].sum(axis=1)
    return g, np.abs(det) / 6.0


def element_matrices(X):
    """Whitney element stiffness (with 1/mu0) and unit-conductivity mass matrices."""
    g, vol = barycentric_gradients(X)
    T = X.shape[0]
    curl = np.empty((T, 6, 3))
    for i, (a, b) in enumerate(LOCAL_EDGES):
        curl[:, i, :] = 2.0 * np.cross(g[:, a, :], g[:, b, :])
    Ke = vol[:, None, None] / MU0 * np.einsum("tik,tjk->tij", curl, curl)
    G = np.einsum("tak,tbk->tab", g, g)               # grad lambda_a . grad lambda_b
    Me = np.empty((T, 6, 6))
    for i, (a, b) in enumerate(LOCAL_EDGES):
        for j, (c, d) in enumerate(LOCAL_EDGES):
            dac, dad, dbc, dbd = float(a == c), float(a == d), float(b == c), float(b == d)
            Me[:, i, j] = vol / 20.0 * ((1 + dac) * G[:, b, d] - (1 + dad) * G[:, b, c]
                                        - (1 + dbc) * G[:, a, d] + (1 + dbd) * G[:, a, c])
    return Ke, Me, vol, curl, g


class FEModel:
    """Edge numbering, PEC removal and the element data of one tetrahedral mesh."""

    def __init__(self, xyz, tets):
        self.xyz = np.asarray(xyz, dtype=np.float64)
        self.tv = np.sort(np.asarray(tets, dtype=np.int64), axis=1)
        nv = self.xyz.shape[0]
        T = self.tv.shape[0]
        pairs = self.tv[:, LOCAL_EDGES]                # [T, 6, 2]
        key = pairs[..., 0] * nv + pairs[..., 1]
        uk, inv = np.unique(key.ravel(), return_inverse=True)
        self.edges = np.stack([uk // nv, uk % nv], axis=1)
        self.tedge = inv.reshape(T, 6)
        # PEC: an edge is on the outer boundary when both end points lie on the
        # same face plane of the bounding box.
        lo, hi = self.xyz.min(axis=0), self.xyz.max(axis=0)
        tol = 1e-9 * (hi - lo).max()
        pa, pb = self.xyz[self.edges[:, 0]], self.xyz[self.edges[:, 1]]
        bnd = np.zeros(len(self.edges), dtype=bool)
        for ax in range(3):
            for v in (lo[ax], hi[ax]):
                bnd |= (np.abs(pa[:, ax] - v) < tol) & (np.abs(pb[:, ax] - v) < tol)
        self.pec = bnd
        self.dof = -np.ones(len(self.edges), dtype=np.int64)
        self.dof[~bnd] = np.arange(int((~bnd).sum()))
        self.N = int((~bnd).sum())
        self.tdof = self.dof[self.tedge]               # [T, 6], -1 on PEC edges
        X = self.xyz[self.tv]
        self.Ke, self.Me1, self.vol, self.curl, self.grad = element_matrices(X)
        # COO pattern of all element entries between interior unknowns
        r = np.repeat(self.tdof[:, :, None], 6, axis=2)
        c = np.repeat(self.tdof[:, None, :], 6, axis=1)
        self._mask = (r >= 0) & (c >= 0)
        self._rows = r[self._mask]
        self._cols = c[self._mask]
        self._tet_of = np.broadcast_to(np.arange(T)[:, None, None], r.shape)[self._mask]
        self.K = self._assemble(self.Ke[self._mask])

    def _assemble(self, data):
        return sp.csr_matrix((data, (self._rows, self._cols)), shape=(self.N, self.N))

    def mass(self, sigma):
        """M(sigma) = sum_e sigma_e P_e^T M1_e P_e."""
        s = np.asarray(sigma, dtype=np.float64)
        return self._assemble((s[:, None, None] * self.Me1)[self._mask])

    def edge_id(self, p, q):
        """Global edge index of the edge joining vertices p and q (or -1)."""
        nv = self.xyz.shape[0]
        a, b = min(p, q), max(p, q)
        key = self.edges[:, 0] * nv + self.edges[:, 1]
        i = np.searchsorted(key, a * nv + b)
        if i < len(key) and key[i] == a * nv + b:
            return int(i)
        return -1

    def interpolate(self, field):
        """Whitney interpolant of a vector field: u_e = int_e E . dl (exact for
        affine fields along a straight edge: midpoint rule)."""
        pa, pb = self.xyz[self.edges[:, 0]], self.xyz[self.edges[:, 1]]
        mid = 0.5 * (pa + pb)
        val = np.einsum("ek,ek->e", field(mid), pb - pa)
        return val[~self.pec]

    def gradient_matrix(self):
        """Node-to-interior-edge incidence G (u = G phi is a discrete gradient)."""
        ne = len(self.edges)
        rows = np.concatenate([np.arange(ne), np.arange(ne)])
        cols = np.concatenate([self.edges[:, 1], self.edges[:, 0]])
        vals = np.concatenate([np.ones(ne), -np.ones(ne)])
        G = sp.csr_matrix((vals, (rows, cols)), shape=(ne, self.xyz.shape[0]))
        return G[~self.pec]
