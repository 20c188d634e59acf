"""Pins of the oracle's regulariser and LSQR (CPU only).

* LSQR (Paige & Saunders 1982) run for n steps on a full-rank n-column
  least-squares problem reaches the normal-equation solution (numpy lstsq);
* the rectangular root W of the two-point RT0 Laplacian satisfies W^T W = L
  with L symmetric positive semidefinite, constants in its kernel (Neumann)
  and only face neighbours coupled (Section 3.2);
* the Gauss-Newton operator's matvec and rmatvec are adjoint (Section 3.3).
"""
import numpy as np

from oracle.inversion import gn_operator, lsqr, regulariser
from oracle.tem import Oracle
from paper_2605_19951_gb300 import inputs


def test_lsqr_matches_lstsq():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((60, 12))
    b = rng.standard_normal(60)
    x, its = lsqr(lambda v: A @ v, lambda u: A.T @ u, b, 12)   # exact in n steps
    xr = np.linalg.lstsq(A, b, rcond=None)[0]
    assert np.linalg.norm(x - xr) <= 1e-12 * np.linalg.norm(xr)
    A = rng.standard_normal((60, 25)) @ np.diag(np.logspace(0, 1.5, 25))
    x, its = lsqr(lambda v: A @ v, lambda u: A.T @ u, b, 75)   # rounding delays it
    xr = np.linalg.lstsq(A, b, rcond=None)[0]
    assert np.linalg.norm(x - xr) <= 1e-10 * np.linalg.norm(xr)
    assert len(its) == 75
    # the residual norm decreases monotonically along the iterates
    res = [np.linalg.norm(A @ xi - b) for xi in its]
    assert np.all(np.diff(res) <= 1e-12)


def test_lsqr_iterates_match_scipy():
    """Every iterate equals scipy's independent LSQR run for the same count."""
    from scipy.sparse.linalg import lsqr as sp_lsqr
    rng = np.random.default_rng(3)
    A = rng.standard_normal((40, 30)) @ np.diag(np.logspace(0, 2, 30))
    b = rng.standard_normal(40)
    _, its = lsqr(lambda v: A @ v, lambda u: A.T @ u, b, 10)
    # rounding differences grow with the iteration count (condition 1e2)
    for k, tol in ((1, 1e-14), (2, 1e-14), (4, 1e-13), (10, 1e-8)):
        ref = sp_lsqr(A, b, atol=0, btol=0, conlim=0, iter_lim=k)[0]
        assert np.linalg.norm(its[k - 1] - ref) <= tol * np.linalg.norm(ref)


def test_regulariser_properties():
    s = inputs.make_config(1)
    W = regulariser(s.xyz, s.tets, s.is_param)
    P = s.n_param
    L = (W.T @ W).toarray()
    assert L.shape == (P, P)
    assert np.allclose(L, L.T)
    assert np.abs(L @ np.ones(P)).max() < 1e-12 * np.abs(L).max()
    ev = np.linalg.eigvalsh(L)
    assert ev.min() > -1e-10 * ev.max()
    assert np.sum(ev < 1e-10 * ev.max()) == 1          # earth is one connected block
    off = (np.abs(L) > 0).sum(axis=1) - 1
    assert off.max() <= 4                              # a tet has four faces
    # each row of W couples exactly two cells with opposite weights
    Wd = W.toarray()
    assert np.all((Wd != 0).sum(axis=1) == 2)
    assert np.allclose(Wd.sum(axis=1), 0.0)


def test_gn_operator_adjoint():
    s = inputs.make_config(1)
    xi, al = inputs.load_rational(s.m, s.times)
    o = Oracle(s.xyz, s.tets, s.sigma, s.is_param, s.loops, s.rx, xi, al)
    o.set_model(s.log_sigma())
    W = regulariser(s.xyz, s.tets, s.is_param)
    rng = np.random.default_rng(2)
    wd = 1.0 / (0.03 * np.abs(o.forward()).ravel() + 1e-8)
    mv, rmv = gn_operator(o, W, wd, 10.0)
    v = rng.standard_normal(s.n_param)
    u = rng.standard_normal(wd.size + W.shape[0])
    a, b = u @ mv(v), v @ rmv(u)
    assert abs(a - b) <= 1e-11 * max(abs(a), abs(b))
