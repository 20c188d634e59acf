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


def _share_face(tets):
    """Pairs of tetrahedra that share three vertices (computed from the vertex
    sets alone, independently of the regulariser's face matching)."""
    sets = [set(int(v) for v in t) for t in tets]
    return {(a, b) for a in range(len(sets)) for b in range(a + 1, len(sets)) if len(sets[a] & sets[b]) == 3}


def test_regulariser_weights_one_cube():
    """Hand-computed pin of the two-point RT0 weights (Section 3.2).  One cube
    of side h cut into the six Kuhn tetrahedra: the interior faces are the six
    triangles (v000, v_e, v111) through the main diagonal, each of area
    |(1,0,0) x (1,1,1)| h^2 / 2 = h^2 / sqrt(2); the centroids of the two
    tetrahedra on such a face, e.g. (3/4, 1/2, 1/4) h and (3/4, 1/4, 1/2) h,
    are h sqrt(2) / 4 apart.  So every row of W is +-sqrt(|f| / d_f) =
    +-sqrt(2 h), and W^T W is 2 h times the Laplacian of the six-cell ring."""
    h = 3.0
    xyz, tets = inputs.kuhn_box(1, h, 0)
    W = regulariser(xyz, tets, np.ones(len(tets), dtype=np.uint8))
    assert W.shape == (6, 6)
    assert np.allclose(np.abs(W.data), np.sqrt(2.0 * h), rtol=1e-13)
    ring = _share_face(tets)
    assert len(ring) == 6
    lap = np.zeros((6, 6))
    for a, b in ring:
        lap[a, a] += 1
        lap[b, b] += 1
        lap[a, b] = lap[b, a] = -1
    assert np.allclose((W.T @ W).toarray(), 2.0 * h * lap, rtol=1e-13, atol=1e-13 * h)


def test_regulariser_weights_two_cubes():
    """Two unit cubes side by side along x (Kuhn cut, conforming on x = 1).
    Inside each cube the six diagonal faces weigh sqrt(2) (the single-cube case
    with h = 1).  On the shared square x = 1 the two triangles, e.g.
    (1,0,0), (1,1,0), (1,1,1) of area 1/2, join the tetrahedra with centroids
    (3/4, 1/2, 1/4) and (5/4, 3/4, 1/2), sqrt(6) / 4 apart, so they weigh
    sqrt((1/2) / (sqrt(6) / 4)) = sqrt(2 / sqrt(6)).  Cells of the second cube
    marked as air drop every face that touches them (Neumann)."""
    xyz, tets = inputs.kuhn_grid([0.0, 1.0, 2.0], [0.0, 1.0], [0.0, 1.0])
    W = regulariser(xyz, tets, np.ones(len(tets), dtype=np.uint8))
    w = np.sort(np.abs(W.toarray()).max(axis=1))
    expect = np.sort(np.r_[np.full(12, np.sqrt(2.0)), np.full(2, np.sqrt(2.0 / np.sqrt(6.0)))])
    assert w.shape == expect.shape
    assert np.allclose(w, expect, rtol=1e-13)
    assert len(_share_face(tets)) == 14
    half = np.zeros(len(tets), dtype=np.uint8)
    half[:6] = 1                                     # cube 0 earth, cube 1 air
    W0 = regulariser(xyz, tets, half)
    assert W0.shape == (6, 6)
    assert np.allclose(np.abs(W0.data), np.sqrt(2.0), rtol=1e-13)
