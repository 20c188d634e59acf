"""Pins of the oracle's sparse LDL^T and of the rational time response (CPU only).

* the plain LDL^T solve equals dense LU (numpy) and SuperLU (scipy) solves;
* complex symmetry without conjugation: <A^-1 b, c> = <b, A^-1 c> (bilinear);
* the sparse residue sum 2 Re sum_i alpha_i (K - xi_i M)^-1 f equals the same
  rational function applied to the dense generalised eigen-decomposition of
  (K, M), and lies within the approximant's measured error of the exact
  exp(-t M^-1 K) M^-1 f (Section 2.2 eq. expm);
* the stored approximant table meets the error it records against exp(-t z).
"""
import numpy as np
import pytest
import scipy.linalg as sla
from scipy.sparse.linalg import splu

from oracle import rational
from oracle.fem import FEModel
from oracle.sparse_ldlt import LDLT, nested_dissection
from oracle.tem import Oracle
from paper_2605_19951_gb300 import inputs


def _tiny(n, n_air=1):
    xyz, tets, sig, earth = inputs.tiny_box(n, 100.0, n_air)
    return FEModel(xyz, tets), sig


@pytest.mark.parametrize("n", [2, 3, 4])
def test_ldlt_matches_dense_and_superlu(n):
    fe, sig = _tiny(n)
    xi, _ = inputs.load_rational(8, inputs.times_log(16))
    perm = nested_dissection(fe.tdof, fe.N, fe.xyz[fe.tv].mean(axis=1), leaf=8)
    M = fe.mass(sig)
    rng = np.random.default_rng(n)
    B = rng.standard_normal((fe.N, 3)) + 1j * rng.standard_normal((fe.N, 3))
    for x in (xi[0], xi[3], xi[-1]):
        A = (fe.K - x * M).astype(np.complex128)
        X = LDLT(A, perm).solve(B)
        Xd = np.linalg.solve(A.toarray(), B)
        Xs = splu(A.tocsc()).solve(B)
        sc = np.abs(Xd).max()
        assert np.abs(X - Xd).max() < 1e-8 * sc      # A is ill-conditioned on air gradients
        assert np.abs(X - Xs).max() < 1e-8 * sc
        # backward error of the LDL^T solve
        R = A @ X - B
        be = np.linalg.norm(R) / (sla.norm(A.toarray(), 2) * np.linalg.norm(X))
        assert be < 1e-14


def test_ldlt_complex_symmetry_c1():
    s = inputs.make_config(1)
    fe = FEModel(s.xyz, s.tets)
    xi, _ = inputs.load_rational(8, s.times)
    perm = nested_dissection(fe.tdof, fe.N, fe.xyz[fe.tv].mean(axis=1))
    A = (fe.K - xi[2] * fe.mass(s.sigma)).astype(np.complex128)
    lu = LDLT(A, perm)
    rng = np.random.default_rng(11)
    b = rng.standard_normal(fe.N) + 1j * rng.standard_normal(fe.N)
    c = rng.standard_normal(fe.N) + 1j * rng.standard_normal(fe.N)
    lhs = lu.solve(b) @ c
    rhs = b @ lu.solve(c)
    assert abs(lhs - rhs) <= 1e-9 * abs(lhs)


def test_rational_table_error():
    for m in (8, 10):
        for K in (16, 24, 40):
            t = inputs.times_log(K)
            xi, al = inputs.load_rational(m, t)
            assert np.all(xi.real < 0) and np.all(xi.imag > 0)
            z = rational.check_points(5000)
            for j in range(K):
                r = 2.0 * np.real((1.0 / (z[:, None] - xi[None, :])) @ al[:, j])
                err = np.max(np.abs(r - np.exp(-t[j] * z)))
                assert err < (4e-4 if m == 8 else 8e-5)


@pytest.mark.parametrize("n,n_air", [(3, 1), (4, 1)])
def test_rational_response_vs_dense_eigen(n, n_air):
    # a less resistive "air" keeps the dense generalised eigenproblem well
    # conditioned (with 1e-8 S/m its own residual is ~1e-9)
    xyz, tets, sig, earth = inputs.tiny_box(n, 100.0, n_air, sigma_air=1e-3)
    times = inputs.times_log(16)
    xi, al = inputs.load_rational(8, times)
    loop = inputs.square_loop(n, n_air, 1, 1, n - 2)
    rx = xyz[loop[0]][None] * np.array([[1.0, 1.0, 0.0]])
    o = Oracle(xyz, tets, sig, earth, [loop], rx, xi, al, threads=2)
    o.set_model(np.log(sig[earth.astype(bool)]))
    K = o.fe.K.toarray()
    M = o.M.toarray()
    lam, V = sla.eigh(K, M)                      # V^T M V = I
    f = o.F[:, 0]
    c = V.T @ f
    # sparse pipeline: u_j = 2 Re sum_i alpha_ij g_i
    G = np.stack([g[:, 0] for g in o.g], axis=1)          # [N, m]
    U = 2.0 * np.real(G @ al)                             # [N, K]
    for j, t in enumerate(times):
        r = 2.0 * np.real((1.0 / (lam[:, None] - xi[None, :])) @ al[:, j])
        u_rat = V @ (r * c)
        # compare in the M-norm (||V y||_M = ||y||_2) against the size of the
        # individual partial fractions (the residue sum cancels)
        pf = 2.0 * (np.abs(1.0 / (lam[:, None] - xi[None, :])) @ np.abs(al[:, j]))
        dr = U[:, j] - u_rat
        assert np.sqrt(abs(dr @ M @ dr)) <= 1e-12 * np.linalg.norm(pf * np.abs(c))
        # exact exp(-t M^-1 K) M^-1 f, in the M-norm
        u_exp = V @ (np.exp(-t * np.maximum(lam, 0.0)) * c)
        eps = np.max(np.abs(r - np.exp(-t * np.maximum(lam, 0.0))))
        dm = U[:, j] - u_exp
        assert np.sqrt(abs(dm @ M @ dm)) <= eps * np.linalg.norm(c) * (1 + 1e-8) + 1e-12 * np.linalg.norm(c)
    assert lam.max() < rational.check_points()[-1]
